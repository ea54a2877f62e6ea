"""MP5 reconstruction (Sec. 3.3 lists it among the reconstruction methods; Suresh & Huynh 1997) on the CUDA path
against the oracle: the right-hand side on every workload kind (ragged blocks; the torus with its jet, the star
with its atmosphere, the Balsara jump), RK4 steps, the batched launch (bit-identical to single blocks) and the
adjoint of the stage and of the RK4 step against the oracle's dual-number derivative.  Tolerances as for the
other schemes: 1e-12 of each field group's magnitude on the owned ranges; the adjoint to 1e-11 of sum |mu J d|."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, field_scale, owned, rel_field_err, small_workloads
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOADS = dict(small_workloads())
WORKLOADS["smooth_general"] = W.smooth_general(n=(9, 8, 7))


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mp5(w):
    return dict(w.params, recon=W.RECON_MP5)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_rhs_parity(name):
    need_gpu()
    w = WORKLOADS[name]
    params = mp5(w)
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
        # where a right-hand side is pure rounding (MP5 reproduces flat data exactly, so the Alfven wave's D~ has
        # none), it is measured against the size of the flux differences it is made of, |U| / dx
        sl = owned(w, v)
        floor = np.abs(U[v][sl]).max() / min(w.dx)
        err = np.abs(got[v][sl] - ref[v][sl]).max()
        scale = max(field_scale(ref, w, v), 1e-3 * floor)
        assert err <= 1e-12 * max(scale, 1e-300), (v, err, scale)


def allowance(w, M, st):
    return 100.0 * w.params["rho_atm"] * float(M[4:10].max()) ** 1.5 if st["n_atm"] else 0.0


@pytest.mark.parametrize("name", ["flat_modes", "balsara_schwarzschild", "star", "torus_jet", "smooth_general"])
def test_rk4_step_parity(name):
    need_gpu()
    w = WORKLOADS[name]
    params = mp5(w)
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


def test_batched_step_matches_single_blocks():
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    blocks = [W.star_block(n, o) for n, o in (((12, 16, 10), (0.3515625, -0.0390625, -0.0234375)),
                                                   ((16, 12, 14), (-0.1, 0.05, 0.02)))]
    params = mp5(blocks[0])
    entries, singles = [], []
    for w in blocks:
        U, P = O.initial_state(w)
        O.ghost_fill_state(w, U)
        M = torch.from_numpy(O.metric_array(w)).cuda()
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, M, torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()))
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


def test_adjoint_equals_the_oracle_jvp():
    need_gpu()
    from test_gpu_adjoint import Problem, check_against_jvp
    w = W.smooth_general(n=(9, 8, 10), recon=W.RECON_MP5)
    prob = Problem(w, seed=2211)
    mu = prob.mu_for(prob.stage_rhs(prob.U))
    case = GpuCase(w)
    lam_d = case.solver.zeros_state()
    case.solver.rhs_adjoint(case.dev(prob.U), case.dev(prob.P), case.dev(mu), lam_d, w.dt)
    worst = check_against_jvp(prob, mu, case.host(lam_d),
                              lambda d: O.stage_jvp(w, prob.M, prob.U, d, prob.P.copy())[1])
    mu = prob.mu_for(prob.rk4(prob.U))
    lam_d = case.dev(mu)
    case.solver.rk4_step_adjoint(case.dev(prob.U), case.dev(prob.P), lam_d, w.dt)
    worst = max(worst, check_against_jvp(prob, mu, case.host(lam_d),
                                         lambda d: O.rk4_jvp(w, prob.M, prob.U, d, prob.P.copy())[1],
                                         entries_full=False))
    print(f"MP5 adjoint: largest relative difference {worst:.2e}")
