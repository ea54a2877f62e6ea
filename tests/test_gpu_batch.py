"""The batched step (asterx_batched_step) against per-block single steps and the oracle.

Several uneven blocks of the magnetised-star workload (floors firing) advance together with one launch per
kernel; each block must end exactly where asterx_rk4_step on that block alone ends (the same kernel bodies
run in both modes), and one block is also compared with the oracle's RK4 step.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, rel_field_err
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (8, 12, 16, 20)


def _blocks(nb=7, seed=303):
    lay = W.star_layout(nblocks=nb, seed=seed, sizes=SIZES, dx=1.0 / 64.0)
    return [W.star_block(n, o, dx=1.0 / 64.0) for n, o in lay]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _inputs(w):
    M = O.metric_array(w)
    P = O.prims_array(w)
    U = np.zeros((9,) + w.shape)
    U[5], U[6], U[7], U[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
    return M, U, P


def test_batched_step_equals_single_block_steps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    ws = _blocks()
    params = ws[0].params
    dt = ws[0].dt
    # batched
    entries = []
    for w in ws:
        M, U, P = _inputs(w)
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, _dev(M), _dev(U), _dev(P)))
    batch = A.Batch(params, entries)
    batch.prepare()
    batch.prim2con()
    st_b = torch.zeros(5, dtype=torch.int64, device="cuda")
    batch.step(dt, nsteps=2, stats=st_b)
    torch.cuda.synchronize()
    # single blocks
    st_s = torch.zeros(5, dtype=torch.int64, device="cuda")
    for w, e in zip(ws, entries):
        M, U, P = _inputs(w)
        s = A.Solver.for_workload(w)
        Md, Ud, Pd = _dev(M), _dev(U), _dev(P)
        s.prepare(Md)
        s.fill_ghosts(Ud)
        s.prim2con(Ud, Pd)
        s.rk4_step(Ud, Pd, dt, stats=st_s)
        s.rk4_step(Ud, Pd, dt, stats=st_s)
        torch.cuda.synchronize()
        Ub, Ug = e[6].cpu().numpy(), Ud.cpu().numpy()
        for v in range(9):
            err, _ = rel_field_err(Ub, Ug, w, v)
            assert err <= 1e-14, (w.n, v, err)
        Pb, Pg = e[7].cpu().numpy(), Pd.cpu().numpy()
        g, n = w.g, w.n
        sl = (slice(None), slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
        assert np.allclose(Pb[sl], Pg[sl], rtol=1e-13, atol=0)
    assert st_b.tolist() == st_s.tolist()


def test_batched_block_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    ws = _blocks(nb=3, seed=304)
    params, dt = ws[0].params, ws[0].dt
    entries = []
    for w in ws:
        M, U, P = _inputs(w)
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, _dev(M), _dev(U), _dev(P)))
    batch = A.Batch(params, entries)
    batch.prepare()
    batch.prim2con()
    batch.step(dt, nsteps=1)
    torch.cuda.synchronize()
    for w, e in zip(ws, entries):
        U, P = O.initial_state(w)
        O.ghost_fill_state(w, U)
        M = O.metric_array(w)
        U1, st = O.rk4_step(w, M, U, P)
        Ub = e[6].cpu().numpy()
        allow = 100.0 * w.params["rho_atm"] * float(M[4:10].max()) ** 1.5
        for v in range(9):
            err, _ = rel_field_err(Ub, U1, w, v, abs_allow=allow if v < 5 else 0.0)
            assert err <= 1e-12, (w.n, v, err)


def test_batched_step_graph_replay_matches_direct_launches():
    """Repeated asterx_batched_step calls replay the step graph the first call cached; inside the caller's own
    stream capture the step launches its kernels directly (and the captured graph replays them).  Both end
    bit-identical after three steps."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    ws = _blocks(nb=4, seed=404)
    params, dt = ws[0].params, ws[0].dt

    def make():
        entries = []
        for w in ws:
            M, U, P = _inputs(w)
            entries.append((w.n, w.g, w.x0, w.dx, w.bc, _dev(M), _dev(U), _dev(P)))
        b = A.Batch(params, entries)
        b.prepare()
        b.prim2con()
        return b, entries

    b1, e1 = make()
    for _ in range(3):
        b1.step(dt, nsteps=1)
    b2, e2 = make()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b2.step(dt, nsteps=3)
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip(e1, e2):
        assert torch.equal(x[6], y[6]) and torch.equal(x[7], y[7])
    b1.release()
    b2.release()
