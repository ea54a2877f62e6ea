"""Pins of the oracle's subcycled two-level step (the fine level takes two RK4 steps of half the coarse step; its
ghost values at every fine stage come from the coarse step by time interpolation, with no buffer zones: the
subcycling of Sec. 3.10, here in the stage-consistent form of Mongwane 2015).

Closed forms: the continuous extension of RK4 reproduces u(0) = u_n and u(h) = u_{n+1}, integrates quadratic
right-hand sides u' = f(t) exactly at every theta, and its derivative rows are the derivatives of its weights.
Order: for the linear problem u' = lambda u the ghost states match the stage states of a fine RK4 step started
from the exact solution to O(h^4) (error ratio about 16 when h halves; a wrong weight drops it to 8 or below).
The two-level subcycled step keeps a uniform state uniform, and on a smooth wave it differs from both levels
stepping with the fine step by an amount that falls at least twelvefold when the step halves.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W


def test_dense_output_end_points_and_weights():
    assert np.array_equal(O.rk4_dense_weights(0.0)[0], np.zeros(4))
    assert np.allclose(O.rk4_dense_weights(1.0)[0], [1 / 6, 1 / 3, 1 / 3, 1 / 6], rtol=0, atol=1e-16)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_dense_output_integrates_quadratics_exactly(deg):
    """u' = f(t) = t^deg on [0, h]: the RK4 slopes are f(0), f(h/2), f(h/2), f(h), and the continuous extension
    must give the integral (theta h)^(deg+1) / (deg+1) at every theta."""
    h = 0.7
    f = lambda t: t ** deg
    k = np.array([f(0.0), f(0.5 * h), f(0.5 * h), f(h)])
    for theta in np.linspace(0.0, 1.0, 11):
        p = h * O.rk4_dense_weights(theta)[0] @ k
        assert abs(p - (theta * h) ** (deg + 1) / (deg + 1)) <= 1e-15


def test_dense_output_derivative_rows():
    """Rows 1..3 are the theta-derivatives of row 0 (central differences of a cubic: exact for the first and
    third derivative up to the known delta^2 term, which is checked away with two step sizes)."""
    for theta in (0.0, 0.3, 0.5, 1.0):
        B = O.rk4_dense_weights(theta)
        for order in (1, 2, 3):
            ests = []
            for dlt in (1e-2, 5e-3):
                r = lambda x: O.rk4_dense_weights(x)[order - 1]
                ests.append((r(theta + dlt) - r(theta - dlt)) / (2 * dlt))
            rich = (4 * ests[1] - ests[0]) / 3
            assert np.abs(rich - B[order]).max() <= 1e-9, (theta, order)


def _ghost_errors(lam, h):
    """Errors of the ghost states against the fine RK4 stage states from the exact solution of u' = lam u."""
    u0 = 1.0 + 0.0j
    # one coarse RK4 step, exact arithmetic on the linear problem
    k1 = lam * u0
    Y1 = u0 + 0.5 * h * k1
    k2 = lam * Y1
    Y2 = u0 + 0.5 * h * k2
    k3 = lam * Y2
    Y3 = u0 + h * k3
    k4 = lam * Y3
    U1 = u0 + h * (k1 + 2 * k2 + 2 * k3 + k4) / 6
    errs = np.zeros((2, 4))
    hf = 0.5 * h
    for m in range(2):
        u = np.exp(lam * m * hf) * u0
        z = lam * hf
        fine = [u, (1 + z / 2) * u, (1 + z / 2 + z * z / 4) * u, (1 + z + z * z / 2 + z ** 3 / 4) * u]
        for s in range(4):
            errs[m, s] = abs(O.subcycle_ghost_state(u0, Y1, Y2, Y3, U1, m, s) - fine[s])
    return errs


@pytest.mark.parametrize("lam", [-1.3, 2.1j, -0.4 + 1.7j])
def test_ghost_states_are_fourth_order(lam):
    e1 = _ghost_errors(lam, 0.1)
    e2 = _ghost_errors(lam, 0.05)
    for m in range(2):
        for s in range(4):
            if e1[m, s] <= 1e-15:  # exact (the first stages of the first substep)
                assert e2[m, s] <= 1e-15
                continue
            assert e1[m, s] / e2[m, s] >= 13.0, (m, s, e1[m, s], e2[m, s])


@pytest.mark.parametrize("Lr", [(2, 2, 1), (0, 4, 2)])  # inside; touching the coarse boundary at low x, high y, z
def test_subcycled_step_keeps_a_uniform_state(Lr):
    from test_oracle_grid import _uniform_workload
    wc = _uniform_workload(W.RECON_PPM, "flat")
    wf = W.Workload("fine", (8, 6, 8), wc.g, tuple(wc.x0[d] + Lr[d] * wc.dx[d] for d in range(3)),
                    tuple(h / 2 for h in wc.dx), wc.bc, wc.params, wc.dt / 2, {}, {}, None, {})
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Mc = O.metric_array(wc)
    Uf = np.zeros((9,) + wf.shape)
    Pf = np.zeros((5,) + wf.shape)
    O.prolong(wc, wf, Lr, Uc, Pc, Uf, Pf, all_points=True)
    Mf = np.stack([np.full(wf.shape, Mc[q].flat[0]) for q in range(16)])
    Uc0, Uf0 = Uc.copy(), Uf.copy()
    Uc1, Uf1 = O.subcycled_rk4_step(wc, Mc, Uc.copy(), Pc.copy(), wf, Mf, Uf.copy(), Pf.copy(), Lr, wc.dt)
    g = wf.g
    for v in range(5):
        sl = (slice(g, g + wf.n[2]), slice(g, g + wf.n[1]), slice(g, g + wf.n[0]))
        assert np.abs(Uf1[v][sl] - Uf0[v][sl]).max() <= 1e-13 * max(np.abs(Uf0[v][sl]).max(), 1.0), v
        slc = (slice(wc.g, wc.g + wc.n[2]), slice(wc.g, wc.g + wc.n[1]), slice(wc.g, wc.g + wc.n[0]))
        assert np.abs(Uc1[v][slc] - Uc0[v][slc]).max() <= 1e-13 * max(np.abs(Uc0[v][slc]).max(), 1.0), v


def _same_step_levels(wc, Mc, Uc, Pc, wf, Mf, Uf, Pf, L, dt, nsteps, params):
    """Both levels step together with the fine step dt (ghosts from the coarse stage states, as the two-level
    step without subcycling does), restricting only after the last step, so that the coarse data feeding the
    fine ghosts evolve on the coarse grid alone, as in the subcycled step."""
    for n in range(nsteps):
        Ua_c, Ua_f = np.zeros_like(Uc), np.zeros_like(Uf)
        Us_c, Us_f = Uc, Uf
        for s in range(4):
            Un_c = Us_c.copy()
            O.rk_stage(wc, Mc, s, dt, Uc, Us_c, Un_c, Ua_c, Pc, params)
            O.prolong(wc, wf, L, Us_c, Pc, Us_f, Pf)
            Un_f = Us_f.copy()
            O.rk_stage_given_ghosts(wf, Mf, s, dt, Uf, Us_f, Un_f, Ua_f, Pf, params)
            Us_c, Us_f = Un_c, Un_f
        Uc, Uf = Us_c, Us_f
    O.restrict(wc, wf, L, Uc, Uf)
    return Uc, Uf


def _alfven_levels(nc=(16, 4, 4), Lr=(4, 1, 1), nf=(16, 4, 4)):
    """The circularly polarised Alfven wave (smooth, an exact nonlinear solution) with WENO-Z on a coarse block
    and a fine box of half the spacing over coarse cells Lr .. Lr + nf / 2 - 1."""
    wc = W.alfven_wave(nc[0], recon=W.RECON_WENOZ, ny=nc[1], nz=nc[2])
    wfd = W.alfven_wave(2 * nc[0], recon=W.RECON_WENOZ, ny=2 * nc[1], nz=2 * nc[2])
    wf = W.sub_block(wfd, tuple(2 * v for v in Lr), nf)
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Uf, Pf = O.initial_state(wf)
    return wc, wf, Lr, O.metric_array(wc), O.metric_array(wf), Uc, Pc, Uf, Pf


def _subcycling_difference(dt, xi):
    wc, wf, Lr, Mc, Mf, Uc, Pc, Uf, Pf = _alfven_levels()
    params = dict(wc.params, xi_lorenz=xi)  # the same Psi damping rate for every step size
    Uc_s, Uf_s = O.subcycled_rk4_step(wc, Mc, Uc.copy(), Pc.copy(), wf, Mf, Uf.copy(), Pf.copy(), Lr, dt, params)
    Uc_r, Uf_r = _same_step_levels(wc, Mc, Uc.copy(), Pc.copy(), wf, Mf, Uf.copy(), Pf.copy(), Lr, 0.5 * dt, 2,
                                   params)
    g = wf.g
    sl = (slice(None), slice(g, g + wf.n[2]), slice(g, g + wf.n[1]), slice(g, g + wf.n[0]))
    return np.abs(Uf_s[sl] - Uf_r[sl]).max(), np.abs(Uf_r[sl] - Uf[sl]).max()


def test_subcycled_step_approaches_same_step_levels():
    """After one coarse step (two fine steps) the fine interior differs from both levels stepping with the fine
    step only through the coarse level's larger step and the time interpolation of its ghost data, both
    high-order in the step: on the smooth Alfven wave with WENO-Z (no limiter kinks) the difference falls at
    least twelvefold per halving of the step (measured 23-53; first order without the stage-consistent ghost
    states would give 2).  The Psi damping rate is fixed, since its default 1.5 / dt differs between the runs
    by design."""
    dt0 = _alfven_levels()[0].dt
    d = []
    for q in range(3):
        dq, ch = _subcycling_difference(dt0 / 2 ** q, 1.5 / dt0)
        d.append(dq)
        assert dq < 1e-3 * ch
    print("differences", ["%.3e" % v for v in d])
    assert d[0] / d[1] >= 12.0 and d[1] / d[2] >= 12.0
