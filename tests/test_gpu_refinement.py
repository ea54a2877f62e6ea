"""Two refinement levels on the CUDA path against the oracle: prolongation (to the ghost points and to every point
of a nested fine block), the two-level RK4 step (coarse stage, prolongation of its stage state to the fine
ghosts, fine stage, restriction after the step) and the subcycled two-level step (one coarse step, two fine
steps of half its size with ghost data interpolated in time from the coarse step).  Prolongation within 1e-13
of each field's magnitude (the same arithmetic, rounding aside); the two-level steps within 1e-12 of each field
group's magnitude."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, rel_field_err
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = (3, 4, 3)
M = (4, 3, 5)


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def levels(n=(12, 12, 12), **kw):
    wc = W.smooth_general(n=n, bc=W.BC_COPY, **kw)
    wfd = W.smooth_general(n=tuple(2 * v for v in n), bc=W.BC_COPY, **kw)
    wf = W.sub_block(wfd, tuple(2 * v for v in L), tuple(2 * v for v in M))
    return wc, wf


@pytest.mark.parametrize("rough", [False, True])
@pytest.mark.parametrize("all_points", [False, True])
def test_prolongation_matches_oracle(rough, all_points):
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    wc, wf = levels()
    if rough:  # the limited fallback acts often
        rng = np.random.default_rng(11)
        Uc = rng.uniform(0.5, 1.5, (9,) + wc.shape)
        Pc = rng.uniform(0.5, 1.5, (5,) + wc.shape)
    else:
        Uc, Pc = O.initial_state(wc)
        O.ghost_fill_state(wc, Uc)
        O.ghost_fill_prims(wc, Pc)
    Uf0 = np.full((9,) + wf.shape, 7.0)
    Pf0 = np.full((5,) + wf.shape, 7.0)
    Uf, Pf = Uf0.copy(), Pf0.copy()
    O.prolong(wc, wf, L, Uc, Pc, Uf, Pf, all_points=all_points)
    cc, cf = GpuCase(wc), GpuCase(wf)
    Ufd, Pfd = cf.dev(Uf0), cf.dev(Pf0)
    A.prolong(cc.solver, cf.solver, cc.dev(Uc), cc.dev(Pc), Ufd, Pfd, all_points=all_points)
    Ug, Pg = cf.host(Ufd), cf.host(Pfd)
    for v in range(9):
        assert np.abs(Ug[v] - Uf[v]).max() <= 1e-13 * np.abs(Uf[v]).max(), v
    for v in range(5):
        assert np.abs(Pg[v] - Pf[v]).max() <= 1e-13 * np.abs(Pf[v]).max(), v


@pytest.mark.parametrize("recon", [W.RECON_PPM, W.RECON_WENOZ])
def test_two_level_step_matches_oracle(recon):
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    wc, wf = levels(recon=recon)
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Uf, Pf = O.initial_state(wf)
    Mc, Mf = O.metric_array(wc), O.metric_array(wf)
    dt = wf.dt
    cc, cf = GpuCase(wc), GpuCase(wf)
    Ucd, Pcd, Ufd, Pfd = cc.dev(Uc), cc.dev(Pc), cf.dev(Uf), cf.dev(Pf)
    stats = cc.stats()
    for _ in range(2):
        A.rk4_step_refined(cc.solver, cf.solver, Ucd, Pcd, Ufd, Pfd, dt, stats=stats)
    rc, rf = Uc.copy(), Uf.copy()
    pc, pf = Pc.copy(), Pf.copy()
    for _ in range(2):
        rc, rf = O.refined_rk4_step(wc, Mc, rc, pc, wf, Mf, rf, pf, L, dt)
        O.ghost_fill_state(wc, rc)
    gc, gf = cc.host(Ucd), cf.host(Ufd)
    for v in range(9):
        e, s = rel_field_err(gc, rc, wc, v)
        assert s == 0.0 or e <= 1e-12, ("coarse", v, e)
        e, s = rel_field_err(gf, rf, wf, v)
        assert s == 0.0 or e <= 1e-12, ("fine", v, e)
    # the coarse points under the fine box hold the restricted fine values
    g = wf.g
    kids = gf[0][g:g + 2 * M[2], g:g + 2 * M[1], g:g + 2 * M[0]].reshape(M[2], 2, M[1], 2, M[0], 2).mean(axis=(1, 3, 5))
    par = gc[0][wc.g + L[2]:wc.g + L[2] + M[2], wc.g + L[1]:wc.g + L[1] + M[1], wc.g + L[0]:wc.g + L[0] + M[0]]
    assert np.abs(kids - par).max() <= 1e-14 * np.abs(par).max()


@pytest.mark.parametrize("recon", [W.RECON_PPM, W.RECON_WENOZ])
def test_subcycled_step_matches_oracle(recon):
    """Two coarse steps of the subcycled two-level step (each: one coarse RK4 step, two fine ones of half the
    size with time-interpolated ghost data) against the oracle, within the parity tolerance on both levels."""
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    wc, wf = levels(recon=recon)
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Uf, Pf = O.initial_state(wf)
    Mc, Mf = O.metric_array(wc), O.metric_array(wf)
    dt = 2.0 * wf.dt
    cc, cf = GpuCase(wc), GpuCase(wf)
    Ucd, Pcd, Ufd, Pfd = cc.dev(Uc), cc.dev(Pc), cf.dev(Uf), cf.dev(Pf)
    stats = cc.stats()
    for _ in range(2):
        A.rk4_step_subcycled(cc.solver, cf.solver, Ucd, Pcd, Ufd, Pfd, dt, stats=stats)
    rc, rf = Uc.copy(), Uf.copy()
    pc, pf = Pc.copy(), Pf.copy()
    for _ in range(2):
        rc, rf = O.subcycled_rk4_step(wc, Mc, rc, pc, wf, Mf, rf, pf, L, dt)
    gc, gf = cc.host(Ucd), cf.host(Ufd)
    for v in range(9):
        e, s = rel_field_err(gc, rc, wc, v)
        assert s == 0.0 or e <= 1e-12, ("coarse", v, e)
        e, s = rel_field_err(gf, rf, wf, v)
        assert s == 0.0 or e <= 1e-12, ("fine", v, e)
    assert int(stats[3]) == 0


@pytest.mark.parametrize("bc", [W.BC_COPY, W.BC_PERIODIC])
def test_subcycled_step_with_the_box_on_the_boundary_matches_oracle(bc):
    """The fine box touching the coarse block's boundary (low x, high y, high z): the interpolated coarse state
    is then formed and recovered along whole axes there, and its ghost fill (copy or periodic) feeds the
    prolongation.  One subcycled step against the oracle, both levels within 1e-12."""
    need_gpu()
    from paper_2406_11669_gb300 import asterx as A
    Lb = (0, 9, 7)  # with M = (4, 3, 5) coarse cells under the box: L + M = (4, 12, 12)
    n = (12, 12, 12)
    wc = W.smooth_general(n=n, bc=bc, recon=W.RECON_WENOZ)
    wfd = W.smooth_general(n=tuple(2 * v for v in n), bc=bc, recon=W.RECON_WENOZ)
    wf = W.sub_block(wfd, tuple(2 * v for v in Lb), tuple(2 * v for v in M))
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Uf, Pf = O.initial_state(wf)
    Mc, Mf = O.metric_array(wc), O.metric_array(wf)
    dt = 2.0 * wf.dt
    cc, cf = GpuCase(wc), GpuCase(wf)
    Ucd, Pcd, Ufd, Pfd = cc.dev(Uc), cc.dev(Pc), cf.dev(Uf), cf.dev(Pf)
    A.rk4_step_subcycled(cc.solver, cf.solver, Ucd, Pcd, Ufd, Pfd, dt)
    rc, rf = O.subcycled_rk4_step(wc, Mc, Uc.copy(), Pc.copy(), wf, Mf, Uf.copy(), Pf.copy(), Lb, dt)
    gc, gf = cc.host(Ucd), cf.host(Ufd)
    for v in range(9):
        e, s = rel_field_err(gc, rc, wc, v)
        assert s == 0.0 or e <= 1e-12, ("coarse", v, e)
        e, s = rel_field_err(gf, rf, wf, v)
        assert s == 0.0 or e <= 1e-12, ("fine", v, e)
