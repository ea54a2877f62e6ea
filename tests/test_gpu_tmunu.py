"""The stress-energy tensor at vertices (asterx_tmunu) and the RK4 step over a time-dependent metric
(asterx_rk4_step_metrics) through the C ABI, against the oracle on the same seeded inputs.

T_{mu nu} is compared per component group (tt | ti | ij) on the owned vertices at 1e-13 of the group's magnitude:
both sides average the same cell values and differ only in rounding order.  The metric step is compared per
field like the RK4 parity tests (1e-12 of the field group's magnitude).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, rel_field_err, small_workloads
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_GROUPS = [(0,), (1, 2, 3), (4, 5, 6, 7, 8, 9)]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def owned_vertices(w):
    g, n = w.g, w.n
    return (slice(g, g + n[2] + 1), slice(g, g + n[1] + 1), slice(g, g + n[0] + 1))


def compare_T(Tg, Tr, w, tol=1e-13):
    sl = owned_vertices(w)
    mask = np.zeros(w.shape, bool)
    mask[sl] = True
    for grp in T_GROUPS:
        scale = max(np.abs(Tr[q][sl]).max() for q in grp)
        for q in grp:
            err = np.abs(Tg[q][sl] - Tr[q][sl]).max()
            assert err <= tol * scale, (q, err / scale)
    assert np.all(Tg[:, ~mask] == 0.0)  # nothing written outside the owned vertices


CASES = dict(small_workloads())
CASES["smooth_general"] = W.smooth_general(n=(9, 8, 7))


@pytest.mark.parametrize("name", list(CASES))
def test_tmunu_matches_oracle(name):
    need_gpu()
    w = CASES[name]
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    O.ghost_fill_prims(w, P)
    M = O.metric_array(w)
    Tr = O.tmunu(w, M, U, P)
    case = GpuCase(w)
    Td = torch.zeros((10,) + w.shape, dtype=torch.float64, device="cuda")
    case.solver.tmunu(case.dev(U), case.dev(P), Td)
    compare_T(case.host(Td), Tr, w)


def test_tmunu_of_a_stage_state():
    """After asterx_rk_stage the stage state U_s and the primitives have their ghosts filled, so T_{mu nu} of the
    stage state follows directly (the coupling order of a spacetime solver's right-hand side)."""
    need_gpu()
    w = W.star_block((14, 12, 16), (0.3515625, -0.0390625, -0.0234375), name="star_block_surface")
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    M = O.metric_array(w)
    case = GpuCase(w)
    Ud, Pd = case.dev(U), case.dev(P)
    Unext, Uacc = Ud.clone(), torch.zeros_like(Ud)
    case.solver.rk_stage(0, w.dt, Ud, Ud, Unext, Uacc, Pd)
    Td = torch.zeros((10,) + w.shape, dtype=torch.float64, device="cuda")
    case.solver.tmunu(Ud, Pd, Td)
    Ur, Pr = U.copy(), P.copy()
    O.rk_stage(w, M, 0, w.dt, Ur, Ur, Ur.copy(), np.zeros_like(Ur), Pr)
    compare_T(case.host(Td), O.tmunu(w, M, Ur, Pr), w, tol=1e-12)


def test_tmunu_full_size():
    """The whole 128^3 block (in the benchmark's launch configuration) against the oracle on 10^3 sub-blocks cut
    from the same arrays: T at a vertex reads cells within one cell and the metric within two, so the sub-block's
    vertices one layer in from its cut agree."""
    need_gpu()
    w = W.balsara_schwarzschild()
    U = np.zeros((9,) + w.shape)
    U[5], U[6], U[7], U[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
    P, M = O.prims_array(w), O.metric_array(w)
    case = GpuCase(w)
    Td = torch.zeros((10,) + w.shape, dtype=torch.float64, device="cuda")
    case.solver.tmunu(case.dev(U), case.dev(P), Td)
    Tg = case.host(Td)
    del Td
    n, g = (10, 10, 10), w.g
    for lo in [(0, 0, 0), (60, 40, 70), (118, 118, 0), (61, 118, 118)]:
        sl = tuple(slice(lo[d], lo[d] + n[d] + 2 * g + 1) for d in (2, 1, 0))
        ws = W.sub_block(w, lo, n)
        Tr = O.tmunu(ws, np.ascontiguousarray(M[(slice(None),) + sl]), np.ascontiguousarray(U[(slice(None),) + sl]),
                     np.ascontiguousarray(P[(slice(None),) + sl]))
        m = 1
        inner_sub = tuple(slice(g + m, g + n[d] + 1 - m) for d in (2, 1, 0))
        inner_full = tuple(slice(lo[d] + g + m, lo[d] + g + n[d] + 1 - m) for d in (2, 1, 0))
        for grp in T_GROUPS:
            scale = max(np.abs(Tr[q][inner_sub]).max() for q in grp)
            for q in grp:
                err = np.abs(Tg[q][inner_full] - Tr[q][inner_sub]).max()
                assert err <= 1e-13 * scale, (lo, q, err / scale)


def stage_metrics(w):
    """Four metrics of a time-dependent spacetime sampled at the RK4 stage times: the workload's metric with its
    lapse and shift changed from stage to stage (the two middle stages share a time)."""
    M = O.metric_array(w)
    out = []
    for s, f in enumerate((0.0, 0.5, 0.5, 1.0)):
        X = M.copy()
        X[0] = M[0] * (1.0 + 0.08 * f)
        X[1] = M[1] + 0.01 * f
        X[3] = M[3] - 0.02 * f
        out.append(X)
    return out


@pytest.mark.parametrize("name", ["star", "smooth_general", "balsara_schwarzschild"])
def test_rk4_step_metrics_matches_oracle(name):
    need_gpu()
    w = CASES[name]
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    Ms = stage_metrics(w)
    ref, st = O.rk4_step_metrics(w, Ms, U.copy(), P.copy())
    case = GpuCase(w)
    Ud, Pd = case.dev(U), case.dev(P)
    stats = case.stats()
    case.solver.rk4_step_metrics(Ud, Pd, w.dt, [case.dev(X) for X in Ms], stats=stats)
    got = case.host(Ud)
    # cells whose D~ sits at the atmosphere threshold after an earlier stage may take either branch on either
    # side (both valid), moving a hydro value by at most a few sqrt(gamma) rho_atm
    abs_allow = 100.0 * w.params["rho_atm"] * float(Ms[0][4:10].max()) ** 1.5 if st["n_atm"] else 0.0
    for v in range(9):
        err, _ = rel_field_err(got, ref, w, v, abs_allow=abs_allow if v < 5 else 0.0)
        assert err <= 1e-12, (v, err)


def test_rk4_step_metrics_with_one_metric_is_the_frozen_step():
    need_gpu()
    w = CASES["weak_field_modes"]
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    case = GpuCase(w)
    a, pa = case.dev(U), case.dev(P)
    b, pb = case.dev(U), case.dev(P)
    case.solver.rk4_step_metrics(a, pa, w.dt, [case.Md] * 4)
    case.solver.rk4_step(b, pb, w.dt)
    assert torch.equal(a, b) and torch.equal(pa, pb)
