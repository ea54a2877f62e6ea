"""Pointwise pins of the oracle: each check uses a route independent of the oracle's own formulas.

* prim -> cons and the fluxes (Eqs. cons, grmhdeqs) against the stress-energy tensor T^{mu nu} of Eq. tmunu
  built here from u^mu and b^mu:  D~ = sqrt(-g) rho u^0,  S~_j = sqrt(-g) T^0_j,  tau~ = sqrt(gamma)(alpha^2 T^00
  - D), and the fluxes sqrt(-g) rho u^i, sqrt(-g) T^i_j, sqrt(-g)(alpha T^{0i} - rho u^i).  In flat space they
  also reduce to the textbook special-relativistic MHD forms (Mignone & Bodo 2006).
* Magnetosonic speeds (Sec. 3.3) against closed forms: sound speeds for b = 0, the perpendicular and parallel
  fast speeds at rest, a boost along B, the lapse/shift scaling at rest, and causality.
* Reconstruction (Sec. 3.3, ReconX unit-test properties): exactness on linear data, design order on smooth
  cell averages, no new extrema at a jump.
* Source terms (Eq. grmhdsrc): the oracle's 3+1 form against the paper's 4-covariant form evaluated from the
  Christoffel symbols of an analytic static 4-metric (complex-step derivatives), with K_ij consistent with
  d_t gamma_ij = 0; and 4th-order convergence of the grid sources built from vertex samples (Sec. 3.2).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

SYMIDX = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}


def m16_from(alp, beta, g, K=None):
    m = np.zeros(16)
    m[0] = alp
    m[1:4] = beta
    for (a, b), k in SYMIDX.items():
        m[k] = g[a][b]
        if K is not None:
            m[k + 6] = K[a][b]
    return m


def four_vectors(alp, beta, g, prim, B, gamma):
    """u^mu, b^mu, rho h, p, and the inverse 4-metric, from the definitions of Sec. 2.2."""
    rho, p = prim[0], prim[1]
    v = np.asarray(prim[2:5])
    B = np.asarray(B)
    g = np.asarray(g)
    beta = np.asarray(beta)
    W_ = 1.0 / math.sqrt(1.0 - v @ g @ v)
    u = np.concatenate([[W_ / alp], W_ * (v - beta / alp)])
    # 4-metric
    g4 = np.zeros((4, 4))
    blow = g @ beta
    g4[0, 0] = -alp ** 2 + beta @ blow
    g4[0, 1:] = blow
    g4[1:, 0] = blow
    g4[1:, 1:] = g
    g4inv = np.linalg.inv(g4)
    # b^mu from the Faraday dual: b^mu = (delta^mu_nu + u^mu u_nu) B^nu / W with B^mu = (0, B^i) for n-observer
    Bmu = np.concatenate([[0.0], B])
    ulow = g4 @ u
    b = (Bmu + u * (ulow @ Bmu)) / W_
    eps = p / ((gamma - 1.0) * rho)
    rhoh = rho * (1.0 + eps) + p
    return u, b, rhoh, p, g4, g4inv


def stress(u, b, rhoh, p, g4inv):
    b2 = b @ np.linalg.inv(g4inv) @ b
    return (rhoh + b2) * np.outer(u, u) + (p + 0.5 * b2) * g4inv - np.outer(b, b), b2


def random_metric(r):
    alp = float(r.uniform(1, 0.5, 1.0)[0])
    beta = r.uniform(3, -0.3, 0.3)
    A = r.uniform(9, -0.15, 0.15).reshape(3, 3)
    g = np.eye(3) * float(r.uniform(1, 1.0, 1.6)[0]) + 0.5 * (A + A.T)
    return alp, beta, g


def random_prim(r, g, vmax=0.9):
    rho = float(10 ** r.uniform(1, -3, 0)[0])
    p = rho * float(10 ** r.uniform(1, -2, 1)[0])
    vd = r.uniform(3, -1, 1)
    v = vd / math.sqrt(vd @ g @ vd) * float(r.uniform(1, 0.0, vmax)[0])
    B = r.uniform(3, -1, 1) * math.sqrt(rho)
    return np.array([rho, p, *v]), B


def test_prim2con_and_flux_match_stress_tensor():
    r = W.Rng(201)
    gamma = 5.0 / 3.0
    params = W.default_params(gamma=gamma)
    for _ in range(200):
        alp, beta, g = random_metric(r)
        prim, B = random_prim(r, g)
        m = m16_from(alp, beta, g)
        cons, fl = O.point_prim2con(params, m, prim, B)
        u, b, rhoh, p, g4, g4inv = four_vectors(alp, beta, g, prim, B, gamma)
        T, _ = stress(u, b, rhoh, p, g4inv)
        Tmixed = T @ g4  # T^mu_nu
        sg = math.sqrt(np.linalg.det(g))
        rho = prim[0]
        D = alp * rho * u[0]
        ref = np.array([sg * D, *(sg * alp * Tmixed[0, 1:]), sg * (alp ** 2 * T[0, 0] - D)])
        np.testing.assert_allclose(cons, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
        for d in range(3):
            fref = alp * sg * np.array([rho * u[1 + d], *Tmixed[1 + d, 1:], alp * T[0, 1 + d] - rho * u[1 + d]])
            np.testing.assert_allclose(fl[d], fref, rtol=1e-11, atol=1e-12 * np.abs(fref).max())


def test_flat_space_reduces_to_srmhd():
    """Flat metric: D = rho W, m = (rho h W^2 + B^2) v - (v.B) B, E = rho h W^2 - p + B^2/2 + (v^2 B^2 - (v.B)^2)/2,
    x-fluxes D v_x, m v_x - (B/W^2 + (v.B) v) B_x + p_t e_x, m_x (for E); tau = E - D."""
    r = W.Rng(202)
    gamma = 4.0 / 3.0
    params = W.default_params(gamma=gamma)
    m = m16_from(1.0, np.zeros(3), np.eye(3))
    for _ in range(200):
        prim, B = random_prim(r, np.eye(3), vmax=0.95)
        rho, p, v = prim[0], prim[1], prim[2:]
        W_ = 1 / math.sqrt(1 - v @ v)
        h = 1 + gamma / (gamma - 1) * p / rho
        vB = v @ B
        B2 = B @ B
        mom = (rho * h * W_ ** 2 + B2) * v - vB * B
        E = rho * h * W_ ** 2 - p + 0.5 * B2 + 0.5 * ((v @ v) * B2 - vB ** 2)
        pt = p + 0.5 * (B2 / W_ ** 2 + vB ** 2)
        cons, fl = O.point_prim2con(params, m, prim, B)
        np.testing.assert_allclose(cons, [rho * W_, *mom, E - rho * W_], rtol=1e-12, atol=1e-14)
        for d in range(3):
            e = np.zeros(3)
            e[d] = 1
            fm = mom * v[d] - (B / W_ ** 2 + vB * v) * B[d] + pt * e
            ref = [rho * W_ * v[d], *fm, mom[d] - rho * W_ * v[d]]
            np.testing.assert_allclose(fl[d], ref, rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------------------------- wave speeds


def _cs2(gamma, rho, p):
    h = 1 + gamma / (gamma - 1) * p / rho
    return gamma * p / (rho * h), rho * h


def test_speeds_hydro_flat_closed_form():
    r = W.Rng(203)
    gamma = 5.0 / 3.0
    params = W.default_params(gamma=gamma)
    m = m16_from(1.0, np.zeros(3), np.eye(3))
    for _ in range(300):
        prim, _ = random_prim(r, np.eye(3), vmax=0.99)
        c2, _ = _cs2(gamma, prim[0], prim[1])
        c = math.sqrt(c2)
        v = prim[2:]
        v2 = v @ v
        for d in range(3):
            vx = v[d]
            root = math.sqrt((1 - v2) * (1 - v2 * c2 - vx * vx * (1 - c2)))
            lp = (vx * (1 - c2) + c * root) / (1 - v2 * c2)
            lm = (vx * (1 - c2) - c * root) / (1 - v2 * c2)
            lo, hi = O.point_wave_speeds(params, m, prim, np.zeros(3), d)
            assert hi == pytest.approx(lp, rel=1e-12, abs=1e-14)
            assert lo == pytest.approx(lm, rel=1e-12, abs=1e-14)


def test_speeds_at_rest_perpendicular_and_parallel():
    gamma = 4.0 / 3.0
    params = W.default_params(gamma=gamma)
    m = m16_from(1.0, np.zeros(3), np.eye(3))
    for rho, p, Bm in [(1.0, 0.1, 0.5), (0.01, 1e-4, 0.3), (1.0, 2.0, 3.0), (1e-3, 1e-3, 1e-2)]:
        c2, rhoh = _cs2(gamma, rho, p)
        cA2 = Bm ** 2 / (rhoh + Bm ** 2)
        prim = np.array([rho, p, 0.0, 0.0, 0.0])
        lo, hi = O.point_wave_speeds(params, m, prim, np.array([0.0, Bm, 0.0]), 0)   # k perpendicular to B
        perp = math.sqrt(c2 + cA2 - c2 * cA2)
        assert hi == pytest.approx(perp, rel=1e-12) and lo == pytest.approx(-perp, rel=1e-12)
        lo, hi = O.point_wave_speeds(params, m, prim, np.array([Bm, 0.0, 0.0]), 0)   # k parallel to B
        par = math.sqrt(max(c2, cA2))
        assert hi == pytest.approx(par, rel=1e-10) and lo == pytest.approx(-par, rel=1e-10)


def test_speeds_boost_along_field():
    """v and B along x: the fast speeds are the rest-frame parallel speed boosted, (V +- c_f)/(1 +- V c_f)."""
    gamma = 5.0 / 3.0
    params = W.default_params(gamma=gamma)
    m = m16_from(1.0, np.zeros(3), np.eye(3))
    for V in (-0.7, -0.2, 0.3, 0.9):
        for Bm in (0.2, 2.0):
            rho, p = 1.0, 0.3
            c2, rhoh = _cs2(gamma, rho, p)
            cf = math.sqrt(max(c2, Bm ** 2 / (rhoh + Bm ** 2)))
            lo, hi = O.point_wave_speeds(params, m, np.array([rho, p, V, 0, 0]), np.array([Bm, 0, 0]), 0)
            assert hi == pytest.approx((V + cf) / (1 + V * cf), rel=1e-10)
            assert lo == pytest.approx((V - cf) / (1 - V * cf), rel=1e-10)


def test_speeds_lapse_shift_at_rest():
    """Fluid at rest with the Eulerian observer (v = 0), b = 0: lambda = -beta^d +- alpha c_s sqrt(gamma^dd)."""
    r = W.Rng(204)
    gamma = 5.0 / 3.0
    params = W.default_params(gamma=gamma)
    for _ in range(100):
        alp, beta, g = random_metric(r)
        m = m16_from(alp, beta, g)
        gu = np.linalg.inv(g)
        rho, p = 0.5, 0.2
        c = math.sqrt(_cs2(gamma, rho, p)[0])
        for d in range(3):
            lo, hi = O.point_wave_speeds(params, m, np.array([rho, p, 0, 0, 0]), np.zeros(3), d)
            assert hi == pytest.approx(-beta[d] + alp * c * math.sqrt(gu[d, d]), rel=1e-12, abs=1e-14)
            assert lo == pytest.approx(-beta[d] - alp * c * math.sqrt(gu[d, d]), rel=1e-12, abs=1e-14)


def test_speeds_causal_and_ordered():
    r = W.Rng(205)
    params = W.default_params(gamma=4.0 / 3.0)
    for _ in range(500):
        alp, beta, g = random_metric(r)
        prim, B = random_prim(r, g, vmax=0.99)
        B = B * float(10 ** r.uniform(1, -2, 1)[0])
        m = m16_from(alp, beta, g)
        gu = np.linalg.inv(g)
        for d in range(3):
            lo, hi = O.point_wave_speeds(params, m, prim, B, d)
            cone = alp * math.sqrt(gu[d, d])
            vt = alp * prim[2 + d] - beta[d]
            assert -beta[d] - cone <= lo < hi <= -beta[d] + cone
            assert lo <= vt <= hi  # the fluid speed lies between the fast speeds


# ------------------------------------------------------------------------------------------- reconstruction


@pytest.mark.parametrize("scheme", [W.RECON_MINMOD, W.RECON_PPM, W.RECON_WENOZ, W.RECON_MP5])
def test_recon_exact_on_linear_and_constant(scheme):
    for a0, s in ((1.3, 0.0), (-2.0, 0.25), (5.0, -1.5)):
        a = a0 + s * np.arange(-2, 3)
        lo, hi = O.point_recon(scheme, a)
        assert lo == pytest.approx(a0 - 0.5 * s, abs=1e-14)
        assert hi == pytest.approx(a0 + 0.5 * s, abs=1e-14)


@pytest.mark.parametrize("scheme,order", [(W.RECON_MINMOD, 1.9), (W.RECON_PPM, 2.9), (W.RECON_WENOZ, 4.5),
                                          (W.RECON_MP5, 4.8)])
def test_recon_design_order_on_smooth_averages(scheme, order):
    def err(n):
        h = 1.0 / n
        xc = (np.arange(-2, n + 2) + 0.5) * h
        avg = (np.exp(xc + h / 2) - np.exp(xc - h / 2)) / h  # exact cell averages of exp(x)
        e = 0.0
        for i in range(2, n + 2):
            lo, hi = O.point_recon(scheme, avg[i - 2:i + 3])
            e = max(e, abs(hi - math.exp(xc[i] + h / 2)), abs(lo - math.exp(xc[i] - h / 2)))
        return e
    e1, e2 = err(32), err(64)
    assert math.log2(e1 / e2) >= order


@pytest.mark.parametrize("scheme", [W.RECON_MINMOD, W.RECON_PPM, W.RECON_WENOZ, W.RECON_MP5])
def test_recon_no_new_extrema_at_jump(scheme):
    data = np.array([1.0] * 6 + [0.125] * 6)
    for i in range(2, 10):
        lo, hi = O.point_recon(scheme, data[i - 2:i + 3])
        window = data[i - 1:i + 2]
        if scheme != W.RECON_WENOZ:  # TVD and monotonicity-preserving schemes: within the neighbouring values
            assert window.min() - 1e-15 <= lo <= window.max() + 1e-15
            assert window.min() - 1e-15 <= hi <= window.max() + 1e-15
        else:  # WENO-Z is essentially non-oscillatory: overshoot tiny against the jump
            assert 0.125 - 1e-3 <= lo <= 1.0 + 1e-3 and 0.125 - 1e-3 <= hi <= 1.0 + 1e-3


def test_mp5_keeps_fifth_order_through_smooth_extrema():
    """MP5's curvature bounds leave smooth extrema unclipped (Suresh & Huynh 1997): on averages of sin 2 pi x,
    whose extrema the cells resolve, the maximum face error over all cells still falls at fifth order, and on
    averages of a monotone quartic the face values are the exact point values (the fifth-order interface
    formula is exact for polynomials of degree four)."""
    def err(n):
        h = 1.0 / n
        xc = (np.arange(-2, n + 2) + 0.5) * h
        avg = (np.cos(2 * math.pi * (xc - h / 2)) - np.cos(2 * math.pi * (xc + h / 2))) / (2 * math.pi * h)
        e = 0.0
        for i in range(2, n + 2):
            lo, hi = O.point_recon(W.RECON_MP5, avg[i - 2:i + 3])
            e = max(e, abs(hi - math.sin(2 * math.pi * (xc[i] + h / 2))),
                    abs(lo - math.sin(2 * math.pi * (xc[i] - h / 2))))
        return e
    e1, e2 = err(32), err(64)
    assert math.log2(e1 / e2) >= 4.8
    h = 0.05
    f = lambda x: 1.0 + x + 0.3 * x ** 2 + 0.2 * x ** 3 + 0.1 * x ** 4
    F = lambda x: x + x ** 2 / 2 + 0.1 * x ** 3 + 0.05 * x ** 4 + 0.02 * x ** 5
    xc = (np.arange(5) + 0.5) * h + 0.5
    avg = (F(xc + h / 2) - F(xc - h / 2)) / h
    lo, hi = O.point_recon(W.RECON_MP5, avg)
    assert hi == pytest.approx(f(xc[2] + h / 2), rel=1e-14)
    assert lo == pytest.approx(f(xc[2] - h / 2), rel=1e-14)


def test_mp5_adds_no_ramp_at_an_isolated_jump():
    """Next to an isolated jump in otherwise flat data the monotonicity-preserving bounds collapse onto the
    cell's own value (the fifth-order value, 0.4 of the jump into the flat cell, lies outside the interval
    [a_i, a_i + minmod(a_i+1 - a_i, 4 (a_i - a_i-1))] = [a_i, a_i]), so every face value is its cell's value."""
    for lo_v, hi_v in ((1.0, 0.125), (0.0, 1.0), (-3.0, 2.5)):
        data = np.array([lo_v] * 6 + [hi_v] * 6)
        for i in range(2, 10):
            lo, hi = O.point_recon(W.RECON_MP5, data[i - 2:i + 3])
            assert abs(lo - data[i]) <= 1e-15 * abs(data[i]) + 1e-300
            assert abs(hi - data[i]) <= 1e-15 * abs(data[i]) + 1e-300


def test_ppm_recovers_parabola_interface_values():
    """Unlimited PPM interface value is the 4th-order (7(a_i + a_i+1) - (a_i-1 + a_i+2))/12: on averages of a
    monotone quadratic it is exact at the interface (all limiter branches inactive)."""
    h = 0.1
    f = lambda x: 1.0 + 2.0 * x + 0.5 * x * x
    F = lambda x: x + x * x + x ** 3 / 6.0
    xc = (np.arange(5) + 0.5) * h + 1.0
    avg = (F(xc + h / 2) - F(xc - h / 2)) / h
    lo, hi = O.point_recon(W.RECON_PPM, avg)
    assert hi == pytest.approx(f(xc[2] + h / 2), rel=1e-13)
    assert lo == pytest.approx(f(xc[2] - h / 2), rel=1e-13)


# ------------------------------------------------------------------------------------------------- sources


def _metric_fn(x):
    """Analytic static 3+1 fields at x (complex-safe): alpha, beta^i, gamma_ij."""
    X, Y, Z = x
    alp = 0.8 + 0.1 * np.sin(X + 2 * Y) + 0.05 * np.cos(Z)
    beta = np.array([0.1 * np.sin(Y), 0.05 * np.cos(Z), 0.1 * np.sin(X + Z)])
    c = 1.0 + 0.2 * np.cos(X * Y)
    g = np.array([[c, 0.05 * np.sin(X), 0.03 * np.cos(Y)],
                  [0.05 * np.sin(X), c + 0.1 * np.sin(Z), 0.02 * np.sin(Y)],
                  [0.03 * np.cos(Y), 0.02 * np.sin(Y), c]])
    return alp, beta, g


def _g4(x):
    alp, beta, g = _metric_fn(x)
    blow = g @ beta
    g4 = np.zeros((4, 4), dtype=np.result_type(alp, complex))
    g4[0, 0] = -alp ** 2 + beta @ blow
    g4[0, 1:] = blow
    g4[1:, 0] = blow
    g4[1:, 1:] = g
    return g4


def _cstep(fn, x, k, h=1e-30):
    xc = np.array(x, dtype=complex)
    xc[k] += 1j * h
    return np.imag(fn(xc)) / h


def _analytic_3p1(x):
    """alpha, beta, gamma, K (static: d_t gamma = 0 => K_ij = (D_i beta_j + D_j beta_i)/(2 alpha)) and the
    spatial derivatives d_i alpha, d_i beta^j, d_i gamma_jk."""
    alp, beta, g = (np.real(q) for q in _metric_fn(np.array(x, dtype=complex)))
    dalp = np.array([_cstep(lambda y: _metric_fn(y)[0], x, k) for k in range(3)])
    dbeta = np.array([_cstep(lambda y: _metric_fn(y)[1], x, k) for k in range(3)])
    dg = np.array([_cstep(lambda y: _metric_fn(y)[2], x, k) for k in range(3)])
    gu = np.linalg.inv(g)
    Gam = 0.5 * (np.einsum("kl,ilj->kij", gu, dg) + np.einsum("kl,jli->kij", gu, dg) -
                 np.einsum("kl,lij->kij", gu, dg))  # Gamma^k_ij
    blow = g @ beta
    dblow = np.einsum("ijk,k->ij", dg, beta) + np.einsum("jk,ik->ij", g, dbeta)  # d_i beta_j
    Dbeta = dblow - np.einsum("kij,k->ij", Gam, blow)
    K = (Dbeta + Dbeta.T) / (2 * alp)
    return alp, beta, g, K, dalp, dbeta, dg


def _covariant_source(x, prim, B, gamma):
    """alpha sqrt(gamma) times Eq. grmhdsrc from Christoffels of the static 4-metric."""
    x = np.asarray(x, float)
    g4 = np.real(_g4(x))
    dg4 = np.zeros((4, 4, 4))  # d_mu g_{nu sigma}, d_t = 0
    for k in range(3):
        dg4[1 + k] = _cstep(_g4, x, k)
    g4inv = np.linalg.inv(g4)
    Gam = 0.5 * (np.einsum("ds,nsm->dnm", g4inv, dg4) + np.einsum("ds,msn->dnm", g4inv, dg4) -
                 np.einsum("ds,snm->dnm", g4inv, dg4))  # Gamma^d_{nm}, indices (delta, nu, mu)
    alp, beta, g = (np.real(q) for q in _metric_fn(x))
    u, b, rhoh, p, _, _ = four_vectors(alp, beta, g, prim, B, gamma)
    T, _ = stress(u, b, rhoh, p, g4inv)
    S = np.zeros(3)
    for j in range(3):
        S[j] = np.einsum("mn,mn->", T, dg4[:, :, 1 + j]) - np.einsum("mn,dnm,d->", T, Gam, g4[:, 1 + j])
    dlnalp = np.concatenate([[0.0], [_cstep(lambda y: _metric_fn(y)[0], x, k) for k in range(3)]]) / alp
    Stau = alp * (T[:, 0] @ dlnalp - np.einsum("mn,nm->", T, Gam[0]))
    sg = math.sqrt(np.linalg.det(g))
    return alp * sg * np.array([0.0, *S, Stau])


def test_sources_3p1_equal_covariant_form():
    r = W.Rng(206)
    gamma = 5.0 / 3.0
    params = W.default_params(gamma=gamma)
    for _ in range(40):
        x = r.uniform(3, -1.0, 1.0)
        alp, beta, g, K, dalp, dbeta, dg = _analytic_3p1(x)
        prim, B = random_prim(r, g, vmax=0.8)
        src = O.point_sources(params, m16_from(alp, beta, g, K), dalp, dbeta.reshape(9), dg.reshape(27), prim, B)
        ref = _covariant_source(x, prim, B, gamma)
        np.testing.assert_allclose(src, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())


def test_grid_sources_fourth_order():
    """Vertex-sampled metric -> 4th-order centre interpolation and derivatives (Sec. 3.2): the grid source
    converges to the analytic one at order ~4."""
    gamma = 5.0 / 3.0

    def run(n):
        g0 = 3
        x0 = (0.1, -0.2, 0.05)
        dx = (0.4 / n,) * 3
        w = W.Workload("src", (n, n, n), g0, x0, dx, (W.BC_COPY,) * 3, W.default_params(gamma=gamma), 0.1,
                       {}, {}, None, {})
        shape = w.shape
        Xv, Yv, Zv = W.positions(w.n, g0, x0, dx, W.VERTEX)
        M = np.zeros((16,) + shape)
        Xb, Yb, Zb = (np.broadcast_to(q, shape) for q in (Xv, Yv, Zv))
        alp, beta, gg = _metric_fn((Xb, Yb, Zb))
        M[0] = alp
        M[1:4] = beta
        for (a, b), k in SYMIDX.items():
            M[k] = gg[a][b]
        # K at vertices is not needed for a consistency check of interpolation; sample it analytically
        Xc, Yc, Zc = W.positions(w.n, g0, x0, dx, W.CELL)
        P = np.zeros((5,) + shape)
        P[0] = 1.0 + 0.1 * np.sin(3 * np.broadcast_to(Xc, shape))
        P[1] = 0.5
        P[2] = 0.1
        P[3] = -0.05
        U = np.zeros((9,) + shape)  # A = 0: B = 0
        src = O.grid_sources(w, M, U, P)
        # analytic source at the centres of a few interior cells (K = 0 in both: vertex K fields are zero)
        err = 0.0
        for (i, j, k) in [(g0, g0, g0), (g0 + n // 2, g0 + n // 3, g0 + n - 1), (g0 + n - 1, g0 + 1, g0 + n // 2)]:
            xc = np.array([x0[0] + (i - g0 + 0.5) * dx[0], x0[1] + (j - g0 + 0.5) * dx[1],
                           x0[2] + (k - g0 + 0.5) * dx[2]])
            a_, b_, g_, _, da, db, dgg = _analytic_3p1(xc)
            prim = P[:, k, j, i]
            ref = O.point_sources(w.params, m16_from(a_, b_, g_, np.zeros((3, 3))), da, db.reshape(9),
                                  dgg.reshape(27), prim, np.zeros(3))
            err = max(err, np.abs(src[:, k, j, i] - ref).max())
        return err

    e1, e2 = run(8), run(16)
    assert math.log2(e1 / e2) >= 3.6
