"""Writes profiles/stage_flops_torus_jet_256.txt: algorithmic FP64 flops per zone-stage of the RK stage on the
256^3 torus-and-jet workload (WENO-Z, Schwarzschild M = 0.1, Gamma = 4/3), part by part and per kernel unit,
counted by the oracle's flop-counting scalar.  Calls only the oracle.

Counting convention (+ - * / sqrt one flop each; x^1.5 one product and one square root; arithmetic whose operands
are all constants -- literals, parameters and the frozen metric, its interpolation included -- is not counted,
because a frozen metric's arithmetic is done once, not every stage):
  * the oracle evaluates each formula in the paper's order, so a product such as T^00 beta^i beta^j K_ij is
    charged as three products of data although beta^i beta^j K_ij is constant, and symmetric contractions are
    summed over all nine (j, k) pairs; the right-hand side's cell part (flux divergence and sources) is
    therefore an upper estimate of the work an implementation that folds those constants needs;
  * the oracle is literal, so it repeats some steps an implementation does once: u = W v is formed for each of
    the three directions, every cell is reconstructed for both of its faces, every PPM interface of the edge
    fields for both edges that share the face value, and the right-hand side forms the face and centre field
    again after the recovery.  Each of these is charged once (thirds, halves, and the recovery's field);
  * the extreme roots of the magnetosonic quartic (Sec. 3.3 cites the quartic without a solver): each root is
    charged one Newton iteration (one evaluation of the quartic and its derivative and the update), the least
    any iterative solver spends on it; further iterations are the solver's overhead, not the method's work;
  * the recovery's Noble Newton iterations and Palenzuela's Brent iterations are charged as executed: the
    starting guess (the previous primitives) and the tolerance are part of the recovery (Sec. 3.5), and the
    library runs the same iterations.

Sampling: 64 sub-blocks of 8^3 interior cells on a regular 4 x 4 x 4 lattice over the 256^3 block (so the torus,
the jet and the atmosphere enter in proportion to their volume), each advanced one oracle RK4 step (to a state
whose recovery guess is the previous step's primitives, as in a run), then counted over the four stages of the
next step.  Per-unit costs (per interior cell, per padded cell, per face, per edge, per vertex) are scaled to the
256^3 block's unit counts.

    python oracle/count_stage_flops.py [--n 256] [--sub 8] [--lattice 4]
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2406_11669_gb300 import workloads as W  # noqa: E402


def total(d):
    return d["add"] + d["mul"] + d["div"] + d["sqrt"]


def units(n):
    """Unit counts of one stage on a block of n = (nx, ny, nz) interior cells with 3 ghosts."""
    g = 3
    N = [m + 2 * g for m in n]
    faces = sum((n[d] + 1) * N[(d + 1) % 3] * N[(d + 2) % 3] for d in range(3))
    recon_cells = sum((n[d] + 2) * N[(d + 1) % 3] * N[(d + 2) % 3] for d in range(3))
    edges = sum(n[e] * (n[(e + 1) % 3] + 1) * (n[(e + 2) % 3] + 1) for e in range(3))
    return {"cells": n[0] * n[1] * n[2], "padded_cells": N[0] * N[1] * N[2],
            "padded_vertices": (N[0] + 1) * (N[1] + 1) * (N[2] + 1), "faces": faces, "recon_cells": recon_cells,
            "potential_vertices": N[0] * N[1] * N[2], "edges": edges,
            "owned_vertices": (n[0] + 1) * (n[1] + 1) * (n[2] + 1),
            "ghost_area": N[0] * N[1] + N[1] * N[2] + N[2] * N[0]}


def count_block(w):
    """Per-unit algorithmic flops summed over the four stages of one RK4 step (after one step from the initial
    data); returns (sums of algorithmic flops per part, unit counts x 4 stages, diagnostics)."""
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    U, _ = O.rk4_step(w, M, U, P)
    O.ghost_fill_state(w, U)
    u = units(w.n)
    part = {k: 0.0 for k in ("ghost", "recovery_field", "recovery", "uvel", "recon", "face_solve", "face_solve_lit",
                             "hydro_cells", "potentials", "edges", "psi", "combine")}
    diag = {k: 0.0 for k in ("speed_iters", "faces_solved", "noble_iters", "n_noble", "n_fallback", "n_atm",
                             "n_failed", "div_face_solve", "faces_other")}
    Un = U.copy()
    Uacc = np.zeros_like(U)
    Us = U
    for s in range(4):
        r = O.stage_flops(w, M, Us, P.copy(), stage=s)
        per_iter = r["speed_loop_flops"] / max(r["speed_iters"], 1)
        extra_iters = r["speed_iters"] - 4 * r["faces_solved"]  # four roots per face, one iteration each charged
        part["ghost"] += total(r["ghost_state"]) + total(r["ghost_prims"])
        part["recovery_field"] += r["recovery_field_flops"]
        part["recovery"] += total(r["recovery"]) - r["recovery_field_flops"]
        part["uvel"] += r["cellvar_flops"] / 3.0
        part["recon"] += r["recon_flops"] / 2.0
        part["face_solve"] += r["facesolve_flops"] - extra_iters * per_iter
        part["face_solve_lit"] += r["facesolve_flops"]
        diag["faces_other"] += total(r["faces"]) - r["cellvar_flops"] - r["recon_flops"] - r["facesolve_flops"]
        part["hydro_cells"] += total(r["hydro_cells"])
        part["potentials"] += total(r["potentials"])
        part["edges"] += total(r["edges"]) - r["edge_ppm_flops"] / 2.0
        part["psi"] += total(r["psi"])
        part["combine"] += total(r["combine"])
        for k in ("speed_iters", "faces_solved", "noble_iters", "n_noble", "n_fallback", "n_atm", "n_failed"):
            diag[k] += r[k]
        Unext = Us.copy()
        O.rk_stage(w, M, s, w.dt, Un, Us, Unext, Uacc, P)
        Us = Unext
    return part, {k: 4 * v for k, v in u.items()}, diag


# unit each part is charged per
PART_UNIT = {"ghost": "ghost_area", "recovery_field": "padded_vertices", "recovery": "cells", "uvel": "padded_cells",
             "recon": "recon_cells", "face_solve": "faces", "face_solve_lit": "faces", "hydro_cells": "cells",
             "potentials": "potential_vertices", "edges": "edges", "psi": "owned_vertices", "combine": "cells"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--sub", type=int, default=8)
    ap.add_argument("--lattice", type=int, default=4)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    O.set_threads(args.threads)
    full = W.torus_jet(n=(args.n,) * 3)
    step = args.n // args.lattice
    off = (step - args.sub) // 2
    sums = {k: 0.0 for k in PART_UNIT}
    usum = {}
    dsum = {}
    for kz in range(args.lattice):
        for ky in range(args.lattice):
            for kx in range(args.lattice):
                lo = (off + kx * step, off + ky * step, off + kz * step)
                w = W.sub_block(full, lo, (args.sub,) * 3, name="sample")
                part, u, diag = count_block(w)
                for k in sums:
                    sums[k] += part[k]
                for k, v in u.items():
                    usum[k] = usum.get(k, 0.0) + v
                for k, v in diag.items():
                    dsum[k] = dsum.get(k, 0.0) + v
    per_unit = {k: sums[k] / usum[PART_UNIT[k]] for k in sums}
    ufull = units((args.n,) * 3)
    per_zone = {k: per_unit[k] * ufull[PART_UNIT[k]] / ufull["cells"] for k in sums}
    alg = sum(v for k, v in per_zone.items() if k != "face_solve_lit")
    lit = alg - per_zone["face_solve"] + per_zone["face_solve_lit"]
    out = os.path.join(ROOT, "profiles", f"stage_flops_torus_jet_{args.n}.txt")
    nsamp = args.lattice ** 3
    with open(out, "w") as f:
        f.write(f"# Algorithmic FP64 flops per zone-stage of the RK stage on the {args.n}^3 torus-and-jet workload\n")
        f.write(f"# (WENO-Z, HLLE, UCT, Lorenz gauge, Schwarzschild M = 0.1), counted with the oracle's flop-counting\n")
        f.write(f"# scalar on {nsamp} sub-blocks of {args.sub}^3 cells (a {args.lattice}^3 lattice), over the four stages\n")
        f.write("# of the second RK4 step, scaled per unit to the full block.  Conventions in oracle/count_stage_flops.py.\n")
        f.write(f"# Command: python oracle/count_stage_flops.py --n {args.n} --sub {args.sub} --lattice {args.lattice}\n")
        f.write("# part: flops per unit (unit), flops per zone-stage of the full block\n")
        for k in sums:
            f.write(f"#   {k:15s} {per_unit[k]:10.2f} per {PART_UNIT[k]:18s} {per_zone[k]:10.1f} per zone-stage\n")
        f.write(f"# sample recovery mix per stage: Noble {dsum['n_noble']:.0f}, Palenzuela {dsum['n_fallback']:.0f}, "
                f"atmosphere {dsum['n_atm']:.0f}, failed {dsum['n_failed']:.0f}; Noble iterations per Noble cell "
                f"{dsum['noble_iters'] / max(dsum['n_noble'], 1):.2f}\n")
        f.write(f"# speed iterations per face (oracle, Newton from the light cone): "
                f"{dsum['speed_iters'] / dsum['faces_solved']:.2f}; charged: 4\n")
        f.write(f"# flops of the faces part outside u, reconstruction and face solve: {dsum['faces_other']:.0f}\n")
        f.write(f"flops_per_zone_stage = {alg:.1f}\n")
        f.write(f"flops_per_zone_stage_literal_speed_iterations = {lit:.1f}\n")
        f.write(f"face_solve_flops_per_face = {per_unit['face_solve']:.1f}\n")
        f.write(f"face_solve_flops_per_face_literal = {per_unit['face_solve_lit']:.1f}\n")
        f.write(f"recon_flops_per_cell_direction = {per_unit['recon']:.1f}\n")
        f.write(f"recovery_flops_per_cell = {per_unit['recovery']:.1f}\n")
        f.write(f"edge_flops_per_edge = {per_unit['edges']:.1f}\n")
        f.write(f"hydro_cell_flops_per_cell = {per_unit['hydro_cells']:.1f}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
