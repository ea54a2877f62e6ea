"""The paper's alternative schemes on the CUDA path against the oracle: the Lax-Friedrichs flux (Eq. LxFfluxes),
flux constrained transport for the edge electric field (Sec. 3.4), and the RK2 step (explicit midpoint).

Same tolerances as the default scheme's parity tests: the right-hand side and the stepped state within 1e-12 of
each field group's magnitude on the owned ranges (with the atmosphere-threshold allowance of chained stages).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, rel_field_err, small_workloads
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SWITCHES = {"lxf_uct": (W.FLUX_LXF, W.EFIELD_UCT), "hlle_fct": (W.FLUX_HLLE, W.EFIELD_FCT),
            "lxf_fct": (W.FLUX_LXF, W.EFIELD_FCT)}
WORKLOADS = dict(small_workloads())
WORKLOADS["smooth_general"] = W.smooth_general(n=(9, 8, 7))
NAMES = ["flat_modes", "balsara_schwarzschild", "star", "torus_jet", "smooth_general"]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def with_switch(w, sw):
    flux, efield = SWITCHES[sw]
    return dict(w.params, flux=flux, efield=efield)


@pytest.mark.parametrize("sw", list(SWITCHES))
@pytest.mark.parametrize("name", NAMES)
def test_rhs_parity(name, sw):
    need_gpu()
    w = WORKLOADS[name]
    params = with_switch(w, sw)
    case = GpuCase(w, params)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    O.con2prim(w, case.M, U, P, params=params)
    O.ghost_fill_prims(w, P)
    ref, _ = O.rhs(w, case.M, U, P, params=params)
    dU = case.solver.zeros_state()
    case.solver.rhs(case.dev(U), case.dev(P), dU, w.dt)
    got = case.host(dU)
    for v in range(9):
        e, scale = rel_field_err(got, ref, w, v)
        if scale < 1e-300:
            continue
        assert e <= 1e-12, (v, e)


def allowance(w, M, st):
    return 100.0 * w.params["rho_atm"] * float(M[4:10].max()) ** 1.5 if st["n_atm"] else 0.0


@pytest.mark.parametrize("sw", list(SWITCHES))
@pytest.mark.parametrize("name", ["flat_modes", "star", "smooth_general"])
def test_rk4_step_parity(name, sw):
    need_gpu()
    w = WORKLOADS[name]
    params = with_switch(w, sw)
    case = GpuCase(w, params)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    Ud, Pd = case.dev(U), case.dev(P)
    case.solver.rk4_step(Ud, Pd, w.dt)
    ref, st = O.rk4_step(w, case.M, U, P, params=params)
    got = case.host(Ud)
    allow = allowance(w, case.M, st)
    for v in range(9):
        e, scale = rel_field_err(got, ref, w, v, abs_allow=allow if v < 5 else 0.0)
        if scale < 1e-300:
            continue
        assert e <= 1e-12, (v, e)


@pytest.mark.parametrize("sw", [None, "lxf_fct"])
@pytest.mark.parametrize("name", ["flat_modes", "star", "weak_field_modes"])
def test_rk2_step_parity(name, sw):
    need_gpu()
    w = WORKLOADS[name]
    params = with_switch(w, sw) if sw else dict(w.params)
    case = GpuCase(w, params)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    Ud, Pd = case.dev(U), case.dev(P)
    stats = case.stats()
    case.solver.rk2_step(Ud, Pd, w.dt, stats=stats)
    ref, st = O.rk2_step(w, case.M, U, P, params=params)
    got = case.host(Ud)
    allow = allowance(w, case.M, st)
    for v in range(9):
        e, scale = rel_field_err(got, ref, w, v, abs_allow=allow if v < 5 else 0.0)
        if scale < 1e-300:
            continue
        assert e <= 1e-12, (v, e)
    assert int(stats[1]) == st["n_fallback"] and int(stats[3]) == st["n_failed"]


def test_batched_step_with_switches_matches_single_blocks():
    """The batched launch takes the switches from the same parameters: each block ends bit-identical to the
    single-block step with the same switches."""
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    blocks = [W.star_block(n, o) for n, o in (((12, 16, 10), (0.3515625, -0.0390625, -0.0234375)),
                                                   ((16, 12, 14), (-0.1, 0.05, 0.02)))]
    params = dict(blocks[0].params, flux=W.FLUX_LXF, efield=W.EFIELD_FCT)
    entries, singles = [], []
    for w in blocks:
        U, P = O.initial_state(w)
        O.ghost_fill_state(w, U)
        M = torch.from_numpy(O.metric_array(w)).cuda()
        Ub, Pb = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, M, Ub, Pb))
        s = A.Solver(params, w.n, w.g, w.x0, w.dx, w.bc)
        s.prepare(M)
        Us, Ps = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
        s.rk4_step(Us, Ps, blocks[0].dt)
        singles.append(Us)
    batch = A.Batch(params, entries)
    batch.prepare()
    batch.step(blocks[0].dt)
    torch.cuda.synchronize()
    for e, Us in zip(entries, singles):
        assert torch.equal(e[6], Us)
    batch.release()
