"""The recovery entry point for callers that cannot allocate device memory (asterx_con2prim_noalloc).

Such callers (a plugin whose host application owns all device memory, or a loop that must not call cudaMalloc
because it can synchronise the device or fail mid-run) get the same recovery as asterx_con2prim with its
scratch in the library's fixed device array.  This test calls both entry points through the C ABI on the same
inputs, twice in a row (the array keeps the previous call's contents, which must not leak into the next), and
compares the results within the tolerances of the other parity tests.  It runs last so that a failure here
leaves every other test already run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(w):
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    rng = np.random.default_rng(11)
    guess = P * (1.0 + 1e-3 * rng.standard_normal(P.shape))
    return U, guess


def _run_workspace(w, M, U, P):
    from paper_2406_11669_gb300 import asterx as A
    s = A.Solver.for_workload(w)
    s.prepare(torch.from_numpy(M).cuda())
    Ud, Pd = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
    fl = torch.zeros(w.shape, dtype=torch.int8, device="cuda")
    st = torch.zeros(5, dtype=torch.int64, device="cuda")
    s.con2prim(Ud, Pd, fl, st)
    torch.cuda.synchronize()
    return Ud.cpu().numpy(), Pd.cpu().numpy(), fl.cpu().numpy(), st.cpu().numpy()


def _run_noalloc(w, M, U, P):
    from paper_2406_11669_gb300 import asterx as A
    Md = torch.from_numpy(M).cuda()
    Ud, Pd = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
    fl = torch.zeros(w.shape, dtype=torch.int8, device="cuda")
    st = torch.zeros(5, dtype=torch.int64, device="cuda")
    status = A.con2prim_noalloc(w.params, w.n, w.g, w.x0, w.dx, w.bc, Md, Ud, Pd, fl, st)
    assert status == A.ASTERX_OK
    torch.cuda.synchronize()
    return Ud.cpu().numpy(), Pd.cpu().numpy(), fl.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # two different blocks in a row: the second call must not see the first call's scratch
    blocks = [W.torus_jet(n=(20, 18, 16)), W.balsara_schwarzschild(n=(24, 11, 9))]
    for w in blocks:
        assert np.prod([m + 7 for m in w.n]) <= 65536
        M = O.metric_array(w)
        U, P = _inputs(w)
        ref = _run_workspace(w, M, U, P)
        got = _run_noalloc(w, M, U, P)
        g, n = w.g, w.n
        sl = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
        assert np.array_equal(got[2][sl], ref[2][sl])  # recovery flags
        assert np.array_equal(got[3], ref[3])          # counters
        for v in range(5):
            scale = max(np.abs(ref[1][v][sl]).max(), 1e-300)
            assert np.abs(got[1][v][sl] - ref[1][v][sl]).max() <= 1e-12 * scale, v
            scale = max(np.abs(ref[0][v][sl]).max(), 1e-300)
            assert np.abs(got[0][v][sl] - ref[0][v][sl]).max() <= 1e-12 * scale, v


def test_noalloc_rejects_blocks_beyond_the_scratch_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    w = W.flat_modes(n=(40, 40, 40))  # 47^3 = 103823 padded entries > 65536: rejected before any launch
    M = torch.zeros((16,) + w.shape, dtype=torch.float64, device="cuda")
    U = torch.zeros((9,) + w.shape, dtype=torch.float64, device="cuda")
    P = torch.zeros((5,) + w.shape, dtype=torch.float64, device="cuda")
    assert A.con2prim_noalloc(w.params, w.n, w.g, w.x0, w.dx, w.bc, M, U, P) == A.ASTERX_EINVAL
