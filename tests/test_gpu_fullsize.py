"""Parity at the full sizes of the workloads, in the launch configuration the benchmark times: the CUDA path
runs the whole block (or the whole 512-block batch) and the oracle recomputes sampled parts of the output.

A stage's output at a cell depends on its inputs within a few cells (reconstruction, face solve, the UCT's PPM
along the transverse faces: at most 6 cells per stage), so the oracle run on a sub-block cut from the same input
arrays (ghost layers included) reproduces the full-grid output in the sub-block's inner part; a margin keeps
out the cells near the cut, where the sub-block's own ghost fill or its shifted metric stencils differ from the
full grid.  Independent blocks of the batch are recomputed whole.  Tolerances are those of the small-block
parity tests: 1e-12 of the field group's magnitude for the right-hand side and the stage, 1e-10 for the
recovered primitives where rho > 10 rho_atm.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import CELL_LIKE, GROUPS, GpuCase
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def potentials_and_prims(w):
    """Inputs as the generator gives them: A, Psi in a state array (hydro fields zero), primitives, metric."""
    U = np.zeros((9,) + w.shape)
    U[5], U[6], U[7], U[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
    return U, O.prims_array(w), O.metric_array(w)


def padded_slice(w, lo, n):
    g = w.g
    return tuple(slice(lo[d], lo[d] + n[d] + 2 * g + 1) for d in (2, 1, 0))


def inner(w, lo, n, v, margin, full):
    """Index ranges of field v in the sub-block's interior shrunk by `margin`: in full-grid indices if `full`,
    else in the sub-block's own."""
    g = w.g
    sl = []
    for a in (2, 1, 0):
        hi = g + n[a] - 1 if CELL_LIKE[v][a] else g + n[a]
        off = lo[a] if full else 0
        sl.append(slice(off + g + margin, off + hi - margin + 1))
    return tuple(sl)


def sub_workload(w, lo, n):
    return W.sub_block(w, lo, n)


def check_fields(gpu_full, ref_subs, w, samples, n, margin, tol, fields=range(9), abs_allow=None, floors=None):
    """Max difference over the samples' inner parts, per field, against the group magnitude over the samples
    (or floors[v], when given and larger)."""
    for v in fields:
        scale = 0.0 if floors is None else floors[v]
        for (lo, ref) in zip(samples, ref_subs):
            for u in GROUPS[v]:
                scale = max(scale, np.abs(ref[u][inner(w, lo, n, u, margin, False)]).max())
        if scale == 0.0:
            continue
        for (lo, ref) in zip(samples, ref_subs):
            a = gpu_full[v][inner(w, lo, n, v, margin, True)]
            r = ref[v][inner(w, lo, n, v, margin, False)]
            err = np.abs(a - r)
            if abs_allow is not None and v < 5:
                err = np.maximum(err - abs_allow, 0.0)
            assert err.max() <= tol * scale, (v, lo, err.max() / scale)


SAMPLES = {
    # the 128^3 benchmark block: corner, across the Riemann interface at x = 0, an upper corner
    "balsara_schwarzschild": (W.balsara_schwarzschild, [(0, 0, 0), (58, 40, 70), (116, 116, 0), (60, 116, 116)]),
    # the 256^3 torus with its jet: atmosphere corner, jet axis, torus ring, mixed
    "torus_jet": (W.torus_jet, [(0, 0, 0), (122, 122, 60), (200, 122, 122), (170, 60, 200)]),
}


@pytest.mark.parametrize("name", list(SAMPLES))
def test_rhs_full_size(name):
    """asterx_rhs over the whole block against the oracle's right-hand side of 12^3 sub-blocks (inner 8^3)."""
    need_gpu()
    make, samples = SAMPLES[name]
    w = make()
    U, P, M = potentials_and_prims(w)
    case = GpuCase(w)
    dU = case.solver.zeros_state()
    case.solver.rhs(case.dev(U), case.dev(P), dU, w.dt)
    dUg = case.host(dU)
    del dU
    n = (12, 12, 12)
    refs = []
    floors = np.zeros(9)
    for lo in samples:
        sl = padded_slice(w, lo, n)
        ws = sub_workload(w, lo, n)
        d, _ = O.rhs(ws, np.ascontiguousarray(M[(slice(None),) + sl]), np.ascontiguousarray(U[(slice(None),) + sl]),
                     np.ascontiguousarray(P[(slice(None),) + sl]), dt=w.dt)
        refs.append(d)
        # the hydro right-hand sides are differences of fluxes of size up to |U| / dx; where they nearly cancel
        # (the rotating torus is close to equilibrium) they are compared against that size
        Uc, _ = O.initial_state(ws)
        for v in range(5):
            grp = max(np.abs(Uc[u][inner(w, lo, n, u, 2, False)]).max() for u in GROUPS[v])
            floors[v] = max(floors[v], grp / min(w.dx))
    check_fields(dUg, refs, w, samples, n, margin=2, tol=1e-12, floors=floors)


@pytest.mark.parametrize("name", list(SAMPLES))
def test_con2prim_full_size(name):
    """prim->cons and recovery over the whole block (CUDA) against the oracle's own prim->cons and recovery on
    sub-blocks: the recovered primitives agree where rho > 10 rho_atm, and so do the recovery flags (a cell whose
    D~ sits exactly at the atmosphere threshold may take either branch; at most 1e-4 of the cells)."""
    need_gpu()
    make, samples = SAMPLES[name]
    w = make()
    U, P, M = potentials_and_prims(w)
    case = GpuCase(w)
    s = case.solver
    Ud, Pd = case.dev(U), case.dev(P)
    s.fill_ghosts(Ud)
    s.prim2con(Ud, Pd)
    fl = case.flags()
    s.con2prim(Ud, Pd, flags=fl)
    Pg, flg = case.host(Pd), case.host(fl)
    del Ud, Pd
    n = (10, 10, 10)
    rho_atm = w.params["rho_atm"]
    flips, total = 0, 0
    for lo in samples:
        ws = sub_workload(w, lo, n)
        Mo = O.metric_array(ws)
        Uo, Po = O.initial_state(ws)
        O.ghost_fill_state(ws, Uo)
        flo, _ = O.con2prim(ws, Mo, Uo, Po)
        io = inner(w, lo, n, 0, 1, False)
        ig = inner(w, lo, n, 0, 1, True)
        same = flo[io] == flg[ig]
        flips += int((~same).sum())
        total += same.size
        dense = same & (Po[0][io] > 10 * rho_atm)
        for r in range(5):
            a, b = Pg[r][ig][dense], Po[r][io][dense]
            if r < 2:
                err = np.abs(a - b) / np.abs(b)
            else:
                err = np.abs(a - b)
            assert err.max(initial=0.0) <= 1e-10, (r, lo, err.max(initial=0.0))
    assert flips <= 1e-4 * total + 1, (flips, total)


def test_rk_stage_full_size():
    """One RK stage (stage 0: ghost fill, recovery, right-hand side, combine) over the whole 128^3 block against
    the oracle's stage on 22^3 sub-blocks (inner 8^3: influence reaches at most 6 cells per stage)."""
    need_gpu()
    make, samples = SAMPLES["balsara_schwarzschild"]
    w = make()
    U, P, M = potentials_and_prims(w)
    case = GpuCase(w)
    s = case.solver
    Ud, Pd = case.dev(U), case.dev(P)
    s.fill_ghosts(Ud)
    s.prim2con(Ud, Pd)
    Unext = Ud.clone()
    acc = s.zeros_state()
    s.rk_stage(0, w.dt, Ud, Ud, Unext, acc, Pd)
    Ug = case.host(Unext)
    del Ud, Pd, Unext, acc
    n = (22, 22, 22)
    samples = [tuple(min(c, 128 - n[0]) for c in lo) for lo in samples]
    refs = []
    for lo in samples:
        ws = sub_workload(w, lo, n)
        Mo = O.metric_array(ws)
        Uo, Po = O.initial_state(ws)
        O.ghost_fill_state(ws, Uo)
        Un = Uo.copy()
        O.rk_stage(ws, Mo, 0, w.dt, Un, Un, Uo, np.zeros_like(Uo), Po)
        refs.append(Uo)
    check_fields(Ug, refs, w, samples, n, margin=7, tol=1e-12)


def test_batched_step_full_size():
    """The 512-block batch of the magnetised star in one asterx_batched_step (as the benchmark runs it); three of
    its blocks recomputed whole by the oracle's RK4 step.  Cells reset to the atmosphere right at the threshold
    may differ by a few sqrt(gamma) rho_atm (the allowance of the small-block RK4 test)."""
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    lay = W.star_layout(nblocks=512)
    entries = []
    for nn, o in lay:
        w = W.star_block(nn, o)
        U, P, M = potentials_and_prims(w)
        Ud, Pd, Md = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (U, P, M))
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, Md, Ud, Pd))
        params, dt = w.params, w.dt
    batch = A.Batch(params, entries)
    batch.prepare()
    batch.prim2con()
    batch.step(dt, nsteps=1)
    torch.cuda.synchronize()
    sizes = [int(np.prod(nn)) for nn, _ in lay]
    picks = [int(np.argmin(sizes)), len(lay) // 2, len(lay) - 1]
    for i in picks:
        w = W.star_block(*lay[i])
        Mo = O.metric_array(w)
        Uo, Po = O.initial_state(w)
        O.ghost_fill_state(w, Uo)
        U1, st = O.rk4_step(w, Mo, Uo, Po)
        Ug = entries[i][6].cpu().numpy()
        allow = 100.0 * w.params["rho_atm"] * float(Mo[4:10].max()) ** 1.5 if st["n_atm"] else 0.0
        check_fields(Ug, [U1], w, [(0, 0, 0)], w.n, margin=0, tol=1e-12, abs_allow=allow)
    del batch, entries


def test_adjoint_full_size():
    """asterx_rhs_adjoint over a whole 64^3 block (the adjoint workload's size; smooth data in every field and a
    general metric, since the adjoint workload's uniform pressure puts the PPM limiter exactly on its switching
    surface, where the derivative is one-sided), with weights on an interior 6^3 region, against central
    differences of the oracle's stage operator on a sub-block around that region (margin 8)."""
    need_gpu()
    w = W.smooth_general(n=(64, 64, 64))
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    case = GpuCase(w)
    rng = W.Rng(3301)
    mu = np.zeros_like(U)
    reg = (slice(33, 39),) * 3  # cells 30..35 of the interior (z, y, x)
    for v in range(9):
        mu[(v,) + reg] = rng.uniform(216, -1.0, 1.0).reshape(6, 6, 6)
    lam_d = case.solver.zeros_state()
    case.solver.rhs_adjoint(case.dev(U), case.dev(P), case.dev(mu), lam_d, w.dt)
    lam = case.host(lam_d)
    lo, n = (22, 22, 22), (22, 22, 22)
    sl = padded_slice(w, lo, n)
    ws = sub_workload(w, lo, n)
    Ms = np.ascontiguousarray(M[(slice(None),) + sl])
    Us = np.ascontiguousarray(U[(slice(None),) + sl])
    Ps = np.ascontiguousarray(P[(slice(None),) + sl])
    mus = np.ascontiguousarray(mu[(slice(None),) + sl])

    def J(X):
        Y = X.copy()
        O.ghost_fill_state(ws, Y)
        Pw = Ps.copy()
        O.con2prim(ws, Ms, Y, Pw)
        O.ghost_fill_prims(ws, Pw)
        dU, _ = O.rhs(ws, Ms, Y, Pw, dt=w.dt)
        return float(np.sum(mus * dU))

    lmax = np.abs(lam).max()
    for v in range(9):
        scale = max(np.abs(U[v]).max(), 1e-3)
        for idx_full in ((34, 35, 36), (31, 37, 33)):
            idx_sub = tuple(i - l for i, l in zip(idx_full, (lo[2], lo[1], lo[0])))
            ad = lam[(v,) + idx_full]
            best = None
            for h in (1e-6, 1e-7):
                d = np.zeros_like(Us)
                d[(v,) + idx_sub] = h * scale
                fd = (J(Us + d) - J(Us - d)) / (2.0 * h * scale)
                if best is None or abs(fd - ad) < abs(best - ad):
                    best = fd
            assert abs(ad - best) <= 1e-6 * lmax, (v, idx_full, ad, best, lmax)
