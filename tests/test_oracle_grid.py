"""Grid-level pins of the oracle's RK stage: structure the discretisation must have whatever the data.

* div B~ = 0 to round-off after a stage (B~ = curl A on faces, Sec. 3.4, Eq. divB2).
* volume integrals of D~, S~_i, tau~ conserved on a periodic flat box (flux form, Eq. fluxconseqs).
* a uniform state in a uniform (non-flat) metric has a zero hydro right-hand side, and curl(dA/dt) = 0.
* A_z advected by a uniform flow moves toward +x (fixes the sign of E = -v~ x B~, Eq. eq3.20 vs the
  induction equation) with second-order error.
* the circularly polarised Alfven wave of Sec. 4.2 travels at v_A = 0.5 and converges at ~2nd order.
* ghost fill: periodic copies are exact images; copy BCs copy hydro and extrapolate A linearly.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W


def interior(w):
    g, n = w.g, w.n
    return (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))


def div_B(w, U):
    Bf = O.face_B(w, U)
    g, n, dx = w.g, w.n, w.dx
    k, j, i = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    k1, j1, i1 = (slice(g + 1, g + n[2] + 1), slice(g + 1, g + n[1] + 1), slice(g + 1, g + n[0] + 1))
    return ((Bf[0][k, j, i1] - Bf[0][k, j, i]) / dx[0] + (Bf[1][k, j1, i] - Bf[1][k, j, i]) / dx[1] +
            (Bf[2][k1, j, i] - Bf[2][k, j, i]) / dx[2]), np.abs(Bf).max()


@pytest.mark.parametrize("maker", [lambda: W.flat_modes(n=(12, 10, 8)), lambda: W.balsara_schwarzschild(n=(12, 8, 8)),
                                   lambda: W.torus_jet(n=(12, 12, 10))])
def test_divB_zero_after_step(maker):
    w = maker()
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    U1, _ = O.rk4_step(w, M, U, P)
    O.ghost_fill_state(w, U1)
    d, bmax = div_B(w, U1)
    assert np.abs(d).max() <= 1e-13 * max(bmax, 1e-30) / min(w.dx)


def test_conservation_periodic_flat():
    w = W.flat_modes(n=(12, 10, 8))
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    sl = interior(w)
    tot0 = np.array([U[v][sl].sum() for v in range(5)])
    scale = np.array([np.abs(U[v][sl]).sum() for v in range(5)])
    for _ in range(2):
        U, st = O.rk4_step(w, M, U, P)
        assert st["n_atm"] == 0 and st["n_failed"] == 0
    tot1 = np.array([U[v][sl].sum() for v in range(5)])
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)


def test_conservation_of_D_curved_periodic():
    """Weak-field lapse (the adjoint workload's metric): only D~ is conserved (the others have sources)."""
    w = W.weak_field_modes(n=(10, 8, 8))
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    sl = interior(w)
    d0 = U[0][sl].sum()
    U1, _ = O.rk4_step(w, M, U, P)
    assert abs(U1[0][sl].sum() - d0) <= 1e-13 * np.abs(U1[0][sl]).sum()
    assert abs(U1[4][sl].sum() - U[4][sl].sum()) > 1e-12 * np.abs(U[4][sl]).sum()


def _uniform_workload(recon, metric_kind):
    n = (8, 7, 6)
    g = 3
    x0 = (-0.3, 0.1, 0.2)
    dx = (0.05, 0.06, 0.07)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    full = lambda v: np.full(shape, v)
    metric = W.flat_metric(shape)
    if metric_kind == "curved":
        metric["alp"][...] = 0.8
        metric["betax"][...] = 0.1
        metric["betay"][...] = -0.05
        metric["betaz"][...] = 0.02
        metric["gxx"][...] = 1.3
        metric["gyy"][...] = 1.2
        metric["gzz"][...] = 1.4
        metric["gxy"][...] = 0.1
        metric["gxz"][...] = -0.05
        metric["gyz"][...] = 0.07
    Bt = np.array([0.3, -0.2, 0.5])  # densitised uniform field from A = (B~ x r)/2
    A = {}
    for name, st, comp in (("Ax", W.XEDGE, 0), ("Ay", W.YEDGE, 1), ("Az", W.ZEDGE, 2)):
        X, Y, Z = W.positions(n, g, x0, dx, st)
        r = [np.broadcast_to(X, shape), np.broadcast_to(Y, shape), np.broadcast_to(Z, shape)]
        a1, a2 = (comp + 1) % 3, (comp + 2) % 3
        A[name] = 0.5 * (Bt[a1] * r[a2] - Bt[a2] * r[a1])
    prims = dict(rho=full(0.7), press=full(0.4), velx=full(0.2), vely=full(-0.1), velz=full(0.15))
    params = W.default_params(gamma=5.0 / 3.0, recon=recon)
    return W.Workload("uniform", n, g, x0, dx, (W.BC_COPY,) * 3, params, 0.01, prims, A, full(0.0), metric)


@pytest.mark.parametrize("recon", [W.RECON_MINMOD, W.RECON_PPM, W.RECON_WENOZ])
@pytest.mark.parametrize("metric_kind", ["flat", "curved"])
def test_uniform_state_is_steady(recon, metric_kind):
    w = _uniform_workload(recon, metric_kind)
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    O.con2prim(w, M, U, P)
    O.ghost_fill_prims(w, P)
    dU, _ = O.rhs(w, M, U, P)
    sl = interior(w)
    for v in range(5):
        assert np.abs(dU[v][sl]).max() <= 1e-13 * max(np.abs(U[v][sl]).max(), 1.0)
    # dB~/dt = curl(dA/dt) = 0: apply the face curl to dA/dt (with its owned range only)
    g, n = w.g, w.n
    Ad = np.zeros_like(U)
    Ad[5:8] = dU[5:8]
    Bf = O.face_B(w, Ad)
    k, j, i = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    assert np.abs(Bf[:, k, j, i]).max() <= 1e-12


def _advection_workload(nx, v, amp=1e-4):
    n = (nx, 1, 1)
    g = 3
    x0 = (0.0, 0.0, 0.0)
    h = 1.0 / nx
    dx = (h, h, h)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    full = lambda q: np.full(shape, q)
    X, _, _ = W.positions(n, g, x0, dx, W.ZEDGE)
    Az = np.broadcast_to(amp * np.sin(2 * math.pi * X), shape).copy()
    prims = dict(rho=full(1.0), press=full(1.0), velx=full(v), vely=full(0.0), velz=full(0.0))
    params = W.default_params(gamma=5.0 / 3.0, recon=W.RECON_MINMOD)
    return W.Workload("advect", n, g, x0, dx, (W.BC_PERIODIC,) * 3, params, 0.25 * h, prims,
                      dict(Ax=full(0.0), Ay=full(0.0), Az=Az), full(0.0), W.flat_metric(shape))


def _advect(nx, v, T):
    w = _advection_workload(nx, v)
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    steps = int(round(T / w.dt))
    for _ in range(steps):
        U, _ = O.rk4_step(w, M, U, P)
        O.ghost_fill_state(w, U)
    g = w.g
    X, _, _ = W.positions(w.n, g, w.x0, w.dx, W.ZEDGE)
    x = X[0, 0, g:g + nx]
    a = U[7][g, g, g:g + nx]
    t = steps * w.dt
    fwd = np.abs(a - 1e-4 * np.sin(2 * math.pi * (x - v * t))).max()
    bwd = np.abs(a - 1e-4 * np.sin(2 * math.pi * (x + v * t))).max()
    return fwd, bwd


def test_vector_potential_advects_downstream():
    fwd, bwd = _advect(16, 0.3, 0.5)
    assert fwd < 0.1 * bwd
    fwd2, _ = _advect(32, 0.3, 0.5)
    assert math.log2(fwd / fwd2) >= 1.7


def _alfven_run(nx, T, recon):
    """L2 error of B^y against the exact translated wave, and the fitted amplitude and phase shift."""
    w = W.alfven_wave(nx, recon=recon)
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    steps = int(round(T / w.dt))
    for _ in range(steps):
        U, st = O.rk4_step(w, M, U, P)
        O.ghost_fill_state(w, U)
        assert st["n_fallback"] == 0 and st["n_atm"] == 0
    t = steps * w.dt
    Bf = O.face_B(w, U)
    g = w.g
    By = 0.5 * (Bf[1][g, g, g:g + nx] + Bf[1][g, g + 1, g:g + nx])
    Xc, _, _ = W.positions(w.n, g, w.x0, w.dx, W.CELL)
    x = Xc[0, 0, g:g + nx]
    exact = np.cos(2 * math.pi * (x - 0.5 * t))
    c = 2.0 / nx * np.sum(By * np.cos(2 * math.pi * x))
    s_ = 2.0 / nx * np.sum(By * np.sin(2 * math.pi * x))
    shift = math.atan2(s_, c) / (2 * math.pi)
    return math.sqrt(np.mean((By - exact) ** 2)), shift, t


def test_alfven_wave_convergence_and_speed():
    """Sec. 4.2: with rho = 1, p = 0.5, Gamma = 5/3, B^x = 1, A0 = 1 the wave travels at v_A = 0.5 (this also
    fixes the reading p = 0.5 of the garbled text).  PPM converges at >= 2nd order; minmod's error decreases
    (its clipping of the cos/sin extrema slows the approach to 2nd order at these resolutions)."""
    T = 0.25
    e16, shift16, t = _alfven_run(16, T, W.RECON_PPM)
    e32, shift32, _ = _alfven_run(32, T, W.RECON_PPM)
    assert math.log2(e16 / e32) >= 2.0
    assert abs(shift32 / t - 0.5) < 2e-3
    m16, _, _ = _alfven_run(16, T, W.RECON_MINMOD)
    m32, _, _ = _alfven_run(32, T, W.RECON_MINMOD)
    assert math.log2(m16 / m32) >= 1.0


def test_ghost_fill_periodic_and_copy():
    w = W.flat_modes(n=(6, 5, 4))
    U, _ = O.initial_state(w)
    O.ghost_fill_state(w, U)
    g, n = w.g, w.n
    # periodic: index i and i + n are the same object for every staggering
    assert np.array_equal(U[:, :, :, 0:g], U[:, :, :, n[0]:n[0] + g])
    assert np.array_equal(U[:, :, 0:g, :], U[:, :, n[1]:n[1] + g, :])
    w2 = W.balsara_schwarzschild(n=(6, 5, 4))
    U2, _ = O.initial_state(w2)
    O.ghost_fill_state(w2, U2)
    # copy: hydro ghosts equal the nearest owned cell; A_z (vertex-like along x) extrapolates linearly
    assert np.array_equal(U2[0][:, :, 0], U2[0][:, :, g])
    a = U2[7][g, g, :]
    assert a[0] == pytest.approx(a[g] - g * (a[g + 1] - a[g]), rel=1e-14)
    hi = g + n[0]
    assert a[hi + 2] == pytest.approx(a[hi] + 2 * (a[hi] - a[hi - 1]), rel=1e-14)


def test_balsara1_robustness_smoke():
    """Table 1 test 1 states (the bench workload's data) in the Schwarzschild slice: one step, no recovery
    failure."""
    w = W.balsara_schwarzschild(n=(24, 6, 6))
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    U1, st = O.rk4_step(w, M, U, P)
    assert st["n_failed"] == 0 and st["n_atm"] == 0
    assert np.all(np.isfinite(U1[:, w.g:w.g + 6, w.g:w.g + 6, w.g:w.g + 24]))


def test_loop_advection_moves_with_the_flow():
    """Magnetic loop advection (Sec. 4) on a coarse 16^2 grid for t = 0.75: the loop's magnetic energy
    centroid moves by v t = (1, 1/2) cells (periodic centroid), and minmod keeps most of its energy.  An
    induction update of the wrong sign would carry the loop the other way."""
    n, T = 16, 0.75
    w = W.loop_advection(n)
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    g = w.g

    def energy(U):
        Bf = O.face_B(w, U)
        bx = 0.5 * (Bf[0][g, g:g + n, g:g + n] + Bf[0][g, g:g + n, g + 1:g + n + 1])
        by = 0.5 * (Bf[1][g, g:g + n, g:g + n] + Bf[1][g, g + 1:g + n + 1, g:g + n])
        return bx ** 2 + by ** 2

    def centroid(e):
        ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        cx = np.angle((e * np.exp(2j * np.pi * (xs + 0.5) / n)).sum()) / (2 * np.pi) * n
        cy = np.angle((e * np.exp(2j * np.pi * (ys + 0.5) / n)).sum()) / (2 * np.pi) * n
        return np.array([cx, cy])

    e0 = energy(U)
    for _ in range(int(round(T / w.dt))):
        U, _ = O.rk4_step(w, M, U, P)
    e1 = energy(U)
    shift = centroid(e1) - centroid(e0)
    shift = (shift + n / 2) % n - n / 2
    assert np.allclose(shift, [T / 12 * n, T / 24 * n], atol=0.1), shift
    assert 0.6 < e1.sum() / e0.sum() <= 1.0
