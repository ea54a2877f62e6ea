"""Pins of the paper's alternative schemes in the oracle: the Lax-Friedrichs flux (Eq. LxFfluxes), flux
constrained transport for the edge electric field (Sec. 3.4, Balsara & Spicer 1999), and the RK2 integrator the
performance section compares with RK4 (Sec. 5; read as the explicit midpoint method).

Face level, against the separately pinned point prim->cons map, fluxes and wave speeds: equal states give the
physical flux for either solver (and the induction fluxes v~^d B~^a - v~^a B~^d); a symmetric wave fan (both
states at rest, c_max = c_min) makes Lax-Friedrichs and HLLE coincide; for a supersonic flow HLLE is the upwind
flux while Lax-Friedrichs keeps the average minus c_wave / 2 times the jump with c_wave the faster side.  Grid
level: a uniform state stays steady, div B~ stays zero and the conserved sums stay constant with either switch,
and flux constrained transport still moves A downstream.  Time integration: on the linear gauge wave of the
potentials (a pure-gauge A = grad chi over a uniform fluid at rest, where nothing else moves) the global error
falls as dt^4 for RK4 and dt^2 for RK2.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
GEN = np.array([0.83, 0.05, -0.03, 0.02, 1.2, 0.1, -0.05, 1.1, 0.07, 1.3, 0, 0, 0, 0, 0, 0], float)
FLAT = np.array([1, 0, 0, 0, 1, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0], float)


def params(flux, efield=W.EFIELD_FCT, **kw):
    return W.default_params(gamma=5.0 / 3.0, flux=flux, efield=efield, **kw)


def metric3(m16):
    g = np.array([[m16[4 + SYM[a][b]] for b in range(3)] for a in range(3)])
    return m16[0], np.array(m16[1:4]), g, math.sqrt(np.linalg.det(g))


def side(m16, rho, p, v, B):
    _, _, g, _ = metric3(m16)
    v = np.asarray(v, float)
    W_ = 1.0 / math.sqrt(1.0 - v @ g @ v)
    return np.array([rho, p, *(W_ * v), *B], float)


def physical(prm, m16, rho, p, v, B, d):
    """Conserved variables and flux along d (both densitised) from the pinned point prim->cons."""
    cons, fl = O.point_prim2con(prm, m16, np.array([rho, p, *v], float), np.asarray(B, float))
    return cons, fl[d]


@pytest.mark.parametrize("flux", [W.FLUX_HLLE, W.FLUX_LXF])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_equal_states_give_the_physical_flux(flux, d):
    prm = params(flux)
    alp, beta, g, sqg = metric3(GEN)
    rho, p, v = 0.7, 0.3, np.array([0.2, -0.15, 0.1])
    B = np.array([0.4, -0.25, 0.3])
    s = side(GEN, rho, p, v, B)
    out = O.point_face(prm, GEN, s, s, sqg * B[d], d)
    _, F = physical(prm, GEN, rho, p, v, B, d)
    assert np.abs(out["F"] - F).max() <= 1e-14 * np.abs(F).max()
    vt = alp * v - beta
    Bt = sqg * B
    for a in range(3):
        ref = 0.0 if a == d else vt[d] * Bt[a] - vt[a] * Bt[d]
        assert abs(out["Fb"][a] - ref) <= 1e-14 * np.abs(Bt).max(), a


def test_lxf_equals_hlle_for_a_symmetric_fan():
    L = side(FLAT, 1.0, 1.0, [0, 0, 0], [0.0, 0.3, -0.2])
    R = side(FLAT, 0.125, 0.1, [0, 0, 0], [0.0, -0.3, 0.1])
    h = O.point_face(params(W.FLUX_HLLE), FLAT, L, R, 0.5, 0)
    x = O.point_face(params(W.FLUX_LXF), FLAT, L, R, 0.5, 0)
    assert h["cmax"] == h["cmin"]
    assert np.abs(h["F"] - x["F"]).max() <= 1e-15 * np.abs(h["F"]).max()
    assert np.abs(h["Fb"] - x["Fb"]).max() <= 1e-15 * np.abs(h["Fb"]).max()


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_supersonic_face_upwind_hlle_and_lxf_dissipation(sign):
    """Cold fast flow along x (all wave speeds of one sign): HLLE returns the upwind side's flux; Lax-Friedrichs
    returns the average minus c_wave / 2 times the jump, c_wave the faster of c_max and c_min."""
    BL, BR = [0.05, 0.1, 0.0], [0.05, -0.05, 0.08]
    vL, vR = [sign * 0.9, 0.05, 0.0], [sign * 0.85, 0.0, -0.05]
    L = side(FLAT, 1.0, 0.01, vL, BL)
    R = side(FLAT, 0.5, 0.02, vR, BR)
    prm = params(W.FLUX_HLLE)
    UL, FL = physical(prm, FLAT, 1.0, 0.01, vL, BL, 0)
    UR, FR = physical(prm, FLAT, 0.5, 0.02, vR, BR, 0)
    lam = [O.point_wave_speeds(prm, FLAT, np.array([r, p, *v]), np.array(B), 0)
           for r, p, v, B in ((1.0, 0.01, vL, BL), (0.5, 0.02, vR, BR))]
    cmax = max(0.0, lam[0][1], lam[1][1])
    cmin = -min(0.0, lam[0][0], lam[1][0])
    h = O.point_face(prm, FLAT, L, R, 0.05, 0)
    up = FL if sign > 0 else FR
    assert (cmin == 0.0) if sign > 0 else (cmax == 0.0)
    assert np.abs(h["F"] - up).max() <= 1e-14 * np.abs(up).max()
    x = O.point_face(params(W.FLUX_LXF), FLAT, L, R, 0.05, 0)
    cw = max(cmax, cmin)
    ref = 0.5 * (FL + FR - cw * (UR - UL))
    assert np.abs(x["F"] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(x["F"] - up).max() > 1e-3 * np.abs(up).max()  # and it is not the upwind flux


def variant(w, flux, efield):
    w.params = dict(w.params, flux=flux, efield=efield)
    return w


SWITCHES = [(W.FLUX_LXF, W.EFIELD_UCT), (W.FLUX_HLLE, W.EFIELD_FCT), (W.FLUX_LXF, W.EFIELD_FCT)]


@pytest.mark.parametrize("flux,efield", SWITCHES)
def test_switches_keep_divB_conservation_and_steady_states(flux, efield):
    from test_oracle_grid import _uniform_workload, div_B, interior
    w = variant(W.flat_modes(n=(10, 8, 6)), flux, efield)
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    sl = interior(w)
    tot0 = np.array([U[v][sl].sum() for v in range(5)])
    scale = np.array([np.abs(U[v][sl]).sum() for v in range(5)])
    U1, st = O.rk4_step(w, M, U, P)
    assert st["n_atm"] == 0 and st["n_failed"] == 0
    O.ghost_fill_state(w, U1)
    d, bmax = div_B(w, U1)
    assert np.abs(d).max() <= 1e-13 * bmax / min(w.dx)
    tot1 = np.array([U1[v][sl].sum() for v in range(5)])
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)
    assert np.abs(U1 - U)[:5].max() > 1e-6  # the flow does evolve
    for kind in ("flat", "curved"):
        u = variant(_uniform_workload(W.RECON_PPM, kind), flux, efield)
        X, Pu = O.initial_state(u)
        Mu = O.metric_array(u)
        O.ghost_fill_state(u, X)
        O.con2prim(u, Mu, X, Pu)
        O.ghost_fill_prims(u, Pu)
        dU, _ = O.rhs(u, Mu, X, Pu)
        s2 = interior(u)
        for v in range(5):
            assert np.abs(dU[v][s2]).max() <= 1e-13 * max(np.abs(X[v][s2]).max(), 1.0), (kind, v)
        Ad = np.zeros_like(X)
        Ad[5:8] = dU[5:8]
        Bf = O.face_B(u, Ad)
        g, n = u.g, u.n
        assert np.abs(Bf[:, g:g + n[2], g:g + n[1], g:g + n[0]]).max() <= 1e-12, kind


def test_fct_moves_A_downstream():
    """A_z(x - v t) in a uniform flow along x: with flux constrained transport the wave still travels toward +x
    (the sign of E in the four-face average)."""
    import test_oracle_grid as G

    def advect(nx):
        w = G._advection_workload(nx, 0.3)
        w.params = dict(w.params, efield=W.EFIELD_FCT)
        U, P = O.initial_state(w)
        M = O.metric_array(w)
        O.ghost_fill_state(w, U)
        steps = int(round(0.25 / w.dt))
        for _ in range(steps):
            U, _ = O.rk4_step(w, M, U, P)
            O.ghost_fill_state(w, U)
        g = w.g
        X, _, _ = W.positions(w.n, g, w.x0, w.dx, W.ZEDGE)
        x = X[0, 0, g:g + nx]
        a = U[7][g, g, g:g + nx]
        t = steps * w.dt
        return (np.abs(a - 1e-4 * np.sin(2 * math.pi * (x - 0.3 * t))).max(),
                np.abs(a - 1e-4 * np.sin(2 * math.pi * (x + 0.3 * t))).max())

    fwd, bwd = advect(16)
    assert fwd < 0.1 * bwd


def _edge_rhs_error(nx, efield):
    """dA_z/dt on the z-edges for A_z = eps sin(2 pi x) cos(2 pi y) carried by a uniform flow v = (0.3, 0, 0) in
    flat space (algebraic gauge, so dA/dt = -E = v~ x B~): the exact value is -v^x dA_z/dx at the edge.  Returns
    the mean absolute error over the owned edges, relative to the mean exact magnitude."""
    n = (nx, nx, 1)
    g, h, eps, vx = 3, 1.0 / nx, 1e-4, 0.3
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    full = lambda q: np.full(shape, q)
    X, Y, _ = W.positions(n, g, (0.0, 0.0, 0.0), (h, h, h), W.ZEDGE)
    Az = np.broadcast_to(eps * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y), shape).copy()
    prims = dict(rho=full(1.0), press=full(1.0), velx=full(vx), vely=full(0.0), velz=full(0.0))
    prm = W.default_params(gamma=5.0 / 3.0, recon=W.RECON_WENOZ, gauge=W.GAUGE_ALGEBRAIC, efield=efield)
    w = W.Workload("edge", n, g, (0.0, 0.0, 0.0), (h, h, h), (W.BC_PERIODIC,) * 3, prm, 0.25 * h, prims,
                   dict(Ax=full(0.0), Ay=full(0.0), Az=Az), full(0.0), W.flat_metric(shape))
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    O.ghost_fill_prims(w, P)
    dU, _ = O.rhs(w, M, U, P)
    sl = (slice(g, g + 1), slice(g, g + nx), slice(g, g + nx))
    exact = -vx * eps * 2 * math.pi * np.cos(2 * math.pi * X) * np.cos(2 * math.pi * Y)
    exact = np.broadcast_to(exact, shape)[sl]
    return np.abs(dU[7][sl] - exact).mean() / np.abs(exact).mean()


@pytest.mark.parametrize("efield", [W.EFIELD_UCT, W.EFIELD_FCT])
def test_edge_field_is_second_order_in_two_dimensions(efield):
    """The discrete dA_z/dt of a field varying in x and y converges at second order in the mean: a face pair
    taken half a cell off (for constrained transport, the faces sharing the edge) leaves a first-order error."""
    e1, e2 = _edge_rhs_error(16, efield), _edge_rhs_error(32, efield)
    assert e1 < 0.05 and math.log2(e1 / e2) >= 1.7, (e1, e2)


def gauge_wave(n=(4, 4, 1), eps=1e-3):
    """Uniform fluid at rest in flat space with a pure-gauge potential A = grad chi (discrete gradient of a vertex
    chi, so the discrete curl B~ is zero) and Psi = 0: the Lorenz-gauge potentials then obey the linear damped
    wave system dA/dt = -grad Psi, dPsi/dt = -div A - xi Psi while the fluid stays put."""
    w = W.flat_modes(n=n)
    w.params = dict(w.params, recon=W.RECON_PPM, xi_lorenz=2.0)
    g, N = w.g, w.N
    x = [w.x0[a] + (np.arange(N[a] + 2) - g) * w.dx[a] for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    chi = eps * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y)
    sh = w.shape
    w.A = dict(Ax=(chi[:-1, :-1, 1:] - chi[:-1, :-1, :-1])[:sh[0], :sh[1], :sh[2]] / w.dx[0],
               Ay=(chi[:-1, 1:, :-1] - chi[:-1, :-1, :-1])[:sh[0], :sh[1], :sh[2]] / w.dx[1],
               Az=np.zeros(sh))
    for k in ("rho", "press"):
        w.prims[k] = np.ones(sh)
    for k in ("velx", "vely", "velz"):
        w.prims[k] = np.zeros(sh)
    return w


def test_rk4_and_rk2_orders_on_the_gauge_wave():
    w = gauge_wave()
    M = O.metric_array(w)
    U0, P0 = O.initial_state(w)
    O.ghost_fill_state(w, U0)
    T = 4.0 * w.dt

    def run(step, N):
        U, P = U0.copy(), P0.copy()
        for _ in range(N):
            U, _ = step(w, M, U, P, T / N)
            O.ghost_fill_state(w, U)
        return U

    ref = run(O.rk4_step, 32)
    g, n = w.g, w.n
    sl = (slice(5, 9), slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    scale = np.abs(U0[sl]).max()
    assert np.abs(ref[sl] - U0[sl]).max() > 0.05 * scale  # the potentials do evolve
    e4 = [np.abs(run(O.rk4_step, N)[sl] - ref[sl]).max() / scale for N in (4, 8, 16)]
    e2 = [np.abs(run(O.rk2_step, N)[sl] - ref[sl]).max() / scale for N in (4, 8, 16)]
    r4 = [e4[0] / e4[1], e4[1] / e4[2]]
    r2 = [e2[0] / e2[1], e2[1] / e2[2]]
    assert all(13.0 < r < 19.0 for r in r4), (e4, r4)
    assert all(3.4 < r < 4.6 for r in r2), (e2, r2)
