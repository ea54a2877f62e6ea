"""Writes profiles/face_flops_balsara_schwarzschild_128.txt: the algorithmic FP64 flops per face of the face solve for the
benchmark workload (128^3 WENO-Z block of Balsara-1 data in the Schwarzschild slice), counted by the oracle's
flop-counting scalar (+, -, *, /, sqrt each one flop) on the central 128x16x16 slab of the same data (the data
are uniform in y and z, so the slab has the block's per-face mix).  Calls only the oracle.

    python oracle/count_face_flops.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2406_11669_gb300 import workloads as W  # noqa: E402


def main():
    full = W.balsara_schwarzschild(n=(128, 128, 128))
    w = W.sub_block(full, (0, 56, 56), (128, 16, 16), name="slab")
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    O.con2prim(w, M, U, P)
    O.ghost_fill_prims(w, P)
    rows = []
    for d in range(3):
        c = O.face_flops(w, M, U, P, d, stride=3)
        tot = c["add"] + c["mul"] + c["div"] + c["sqrt"]
        rows.append((d, c, tot / c["faces"]))
    mean = sum(r[2] for r in rows) / 3.0
    out = os.path.join(ROOT, "profiles", "face_flops_balsara_schwarzschild_128.txt")
    with open(out, "w") as f:
        f.write("# Algorithmic FP64 flops per face of the face solve (k_single<Faces<D>>), counted with the oracle's\n")
        f.write("# flop-counting scalar on the central 128x16x16 slab of the 128^3 WENO-Z Schwarzschild workload\n")
        f.write("# (every 3rd face of each direction).  + - * / sqrt count one flop each; metric interpolation\n")
        f.write("# is excluded (frozen metric, precomputed once).  Command: python oracle/count_face_flops.py\n")
        for d, c, per in rows:
            f.write(f"# dir {'xyz'[d]}: faces {int(c['faces'])} add {int(c['add'])} mul {int(c['mul'])} "
                    f"div {int(c['div'])} sqrt {int(c['sqrt'])} speed_iters/face {c['speed_iters'] / c['faces']:.2f} "
                    f"flops/face {per:.1f}\n")
        f.write(f"flops_per_face = {mean:.1f}\n")
        divs = sum(r[1]["div"] for r in rows) / sum(r[1]["faces"] for r in rows)
        sqrts = sum(r[1]["sqrt"] for r in rows) / sum(r[1]["faces"] for r in rows)
        f.write(f"div_per_face = {divs:.2f}\nsqrt_per_face = {sqrts:.2f}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
