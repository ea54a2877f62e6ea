"""Pins of the oracle's potential right-hand side on a curved metric (Sec. 3.4, Eqs. recastedAvec and
recastedScalarPot; Sec. 2.3, Eq. scalarpotentialevol2), and of its metric interpolation (Sec. 3.2).

The potentials evolve by dA_i/dt = -E_i - d_i G_A and dPsi/dt = -d_j F^j - xi alpha Psi with
G_A = alpha Psi / sqrt(gamma) - beta^j A_j and F^j = alpha sqrt(gamma) gamma^{jk} A_k - beta^j Psi (Psi is the
densitised scalar potential).  On a constant metric with alpha != 1, beta != 0, a non-diagonal gamma_ij and
sqrt(gamma) != 1, with the fluid at rest and no magnetic field (E = 0), two families of data have closed-form
right-hand sides that the method's stencils reproduce exactly (the vertex average of the edge A, the vertex-to-
edge difference of G_A and the centred vertex difference of F^j are exact for linear functions):

  (i)  A uniform (a_k), Psi = p0 + c.x:      dPsi/dt = beta^j c_j - xi alpha Psi,  dA_i/dt = -(alpha / sqrt(gamma)) c_i
  (ii) Psi = 0, A = grad chi, chi quadratic: dPsi/dt = -alpha sqrt(gamma) gamma^{jk} H_jk,  dA_i/dt = beta^j H_ij
       (H the Hessian of chi; A on the edges is the difference of chi between the edge's vertices, so the
       discrete curl vanishes and E = 0).

The expected values are computed here from numpy's inverse and determinant of gamma_ij.  Each factor of G_A and
F^j appears in one of them: sqrt(gamma) in G_A through (i), sqrt(gamma) and gamma^{jk} in F^j through (ii), the
sign of beta^j Psi through (i), the sign of beta^j A_j through (ii).  Dropping a factor, inverting it or
flipping a sign changes a closed form by O(1).

The metric interpolation to centres and faces is pinned against the plain tensor-product Lagrange sum (weights
(-1, 9, 9, -1)/16 per axis; the derivative stencil (1, -27, 27, -1)/(24 h) along its axis), evaluated exactly
in rational arithmetic: the oracle's fused, x-then-y-then-z summation agrees with that exact sum to rounding,
so the oracle's definition does not depend on the order in which it sums.
"""
from fractions import Fraction

import numpy as np

import oracle as O
from paper_2406_11669_gb300 import workloads as W

ALPHA = 0.8
BETA = np.array([0.11, -0.06, 0.07])
GAMMA = np.array([[1.30, 0.10, -0.05],
                  [0.10, 1.15, 0.08],
                  [-0.05, 0.08, 0.90]])
XI = 3.0


def _constant_metric(shape):
    m = {k: np.zeros(shape) for k in W.METRIC_NAMES}
    m["alp"][...] = ALPHA
    for a, name in enumerate(("betax", "betay", "betaz")):
        m[name][...] = BETA[a]
    for name, (a, b) in zip(("gxx", "gxy", "gxz", "gyy", "gyz", "gzz"),
                            ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        m[name][...] = GAMMA[a, b]
    return m


def _workload(n, A, Psi_fn):
    """A block at rest on the constant metric; A = (Ax, Ay, Az) as functions of the vertex coordinates of each
    edge's two end points (the edge value is computed from them), Psi_fn of the vertex coordinates.  Every
    padded point, ghosts included, is set from the formulas, so no ghost fill is involved."""
    g = 3
    x0 = (-0.3, 0.2, 0.1)
    dx = (0.1, 0.125, 0.08)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    Xv, Yv, Zv = W.positions(n, g, x0, dx, W.VERTEX)
    Xv, Yv, Zv = (np.broadcast_to(a, shape) for a in (Xv, Yv, Zv))
    pos = (Xv, Yv, Zv)
    Aed = {}
    for e, name in enumerate(("Ax", "Ay", "Az")):
        hi = [p.copy() for p in pos]
        hi[e] = hi[e] + dx[e]
        Aed[name] = np.ascontiguousarray(A[e](pos, hi))
    prims = dict(rho=np.full(shape, 1.0), press=np.full(shape, 0.7), velx=np.zeros(shape), vely=np.zeros(shape),
                 velz=np.zeros(shape))
    params = W.default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-9, recon=W.RECON_PPM,
                              xi_lorenz=XI)
    return W.Workload("gauge_pin", tuple(n), g, x0, dx, (W.BC_COPY,) * 3, params, 0.25 * min(dx), prims, Aed,
                      np.ascontiguousarray(Psi_fn(pos)), _constant_metric(shape))


def _rhs(w):
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    dU, _ = O.rhs(w, M, U, P, dt=w.dt)
    return U, dU


def _owned(w, kind):
    """Index ranges of the owned vertices, or of the owned edges along axis e (kind = 'v' or 0, 1, 2)."""
    g, n = w.g, w.n
    sl = []
    for a in (2, 1, 0):
        hi = g + n[a] + (0 if kind == a else 1)
        sl.append(slice(g, hi))
    return tuple(sl)


def test_uniform_potential_and_linear_psi_on_a_general_metric():
    """(i): G_A's factor 1/sqrt(gamma) and the sign of -beta^j Psi in F^j."""
    a = np.array([0.3, -0.2, 0.45])
    p0, c = 0.05, np.array([0.7, -0.4, 0.25])
    A = [lambda lo, hi, e=e: np.full(lo[0].shape, a[e]) for e in range(3)]
    w = _workload((7, 6, 5), A, lambda x: p0 + c[0] * x[0] + c[1] * x[1] + c[2] * x[2])
    U, dU = _rhs(w)
    sqrtg = np.sqrt(np.linalg.det(GAMMA))
    psi = U[8][_owned(w, "v")]
    want_psi = BETA @ c - XI * ALPHA * psi
    scale = np.abs(BETA @ c) + XI * ALPHA * np.abs(psi).max()
    assert np.abs(dU[8][_owned(w, "v")] - want_psi).max() <= 1e-13 * scale
    for e in range(3):
        want = -(ALPHA / sqrtg) * c[e]
        got = dU[5 + e][_owned(w, e)]
        assert np.abs(got - want).max() <= 1e-13 * np.abs(c).max(), e


def test_gradient_potential_with_zero_psi_on_a_general_metric():
    """(ii): F^j's factors alpha sqrt(gamma) gamma^{jk} and the sign of -beta^j A_j in G_A."""
    H = np.array([[0.9, -0.3, 0.2],
                  [-0.3, 0.5, 0.6],
                  [0.2, 0.6, -0.7]])
    b = np.array([0.2, -0.1, 0.3])

    def chi(x):
        q = b[0] * x[0] + b[1] * x[1] + b[2] * x[2]
        for i in range(3):
            for j in range(3):
                q = q + 0.5 * H[i, j] * x[i] * x[j]
        return q

    dx = (0.1, 0.125, 0.08)
    A = [lambda lo, hi, e=e: (chi(hi) - chi(lo)) / dx[e] for e in range(3)]
    w = _workload((6, 7, 5), A, lambda x: np.zeros(x[0].shape))
    assert w.dx == dx
    U, dU = _rhs(w)
    # the discrete curl of a discrete gradient vanishes: no magnetic field
    Bf = O.face_B(w, U)
    assert np.abs(Bf).max() <= 1e-12 * np.abs(U[5:8]).max() / min(dx)
    gu = np.linalg.inv(GAMMA)
    sqrtg = np.sqrt(np.linalg.det(GAMMA))
    want_psi = -ALPHA * sqrtg * np.sum(gu * H)
    assert abs(want_psi) > 0.1
    got_psi = dU[8][_owned(w, "v")]
    assert np.abs(got_psi - want_psi).max() <= 1e-11 * abs(want_psi)
    for e in range(3):
        want = BETA @ H[e]
        got = dU[5 + e][_owned(w, e)]
        assert np.abs(got - want).max() <= 1e-11 * np.abs(H).max(), e


# ------------------------------------------------------------------------------------------------------------
# metric interpolation against the exact tensor-product sum

LAG = [Fraction(-1, 16), Fraction(9, 16), Fraction(9, 16), Fraction(-1, 16)]
DER = [Fraction(1, 24), Fraction(-27, 24), Fraction(27, 24), Fraction(-1, 24)]


def _exact_sum(f, lo, weights):
    """sum_abc w_x[a] w_y[b] w_z[c] f[z0 + c, y0 + b, x0 + a] in rational arithmetic (weights per axis; an axis
    with weights [1] is not interpolated)."""
    acc = Fraction(0)
    for c, wz in enumerate(weights[2]):
        for bb, wy in enumerate(weights[1]):
            for a, wx in enumerate(weights[0]):
                acc += wx * wy * wz * Fraction(float(f[lo[2] + c, lo[1] + bb, lo[0] + a]))
    return acc


def _abs_sum(f, lo, weights):
    return _exact_sum(np.abs(f), lo, [[abs(x) for x in w] for w in weights])


def test_metric_interpolation_equals_the_exact_lagrange_sum():
    w = W.smooth_general(n=(5, 4, 6))
    M = O.metric_array(w)
    C = O.centre_metric(w, M)
    faces = [O.face_metric(w, M, d) for d in range(3)]
    N = w.N
    rng = np.random.default_rng(3)
    # centres whose 4-point stencils are centred (vertex i-1..i+2 along every axis)
    pts = [tuple(int(rng.integers(1, N[d] - 2)) for d in range(3)) for _ in range(12)]
    interp = [(0, 0)] + [(1 + a, 1 + a) for a in range(3)] + [(4 + q, 4 + q) for q in range(6)] + \
             [(10 + q, 17 + q) for q in range(6)]   # (metric field, centre-record field)
    worst = 0.0
    for (i, j, k) in pts:
        lo = (i - 1, j - 1, k - 1)
        for f, r in interp:
            ex = _exact_sum(M[f], lo, [LAG] * 3)
            err = abs(Fraction(float(C[r][k, j, i])) - ex) / _abs_sum(M[f], lo, [LAG] * 3)
            worst = max(worst, float(err))
        # derivatives: d_d alpha (record 23 + d), d_d beta^a (26 + 3d + a), d_d gamma_q (35 + 6d + q)
        for d in range(3):
            ws = [LAG] * 3
            ws[d] = [x / Fraction(w.dx[d]) for x in DER]
            for f, r in [(0, 23 + d)] + [(1 + a, 26 + 3 * d + a) for a in range(3)] + \
                        [(4 + q, 35 + 6 * d + q) for q in range(6)]:
                ex = _exact_sum(M[f], lo, ws)
                err = abs(Fraction(float(C[r][k, j, i])) - ex) / _abs_sum(M[f], lo, ws)
                worst = max(worst, float(err))
        # faces normal to d: vertex index along d, centred stencils across
        for d in range(3):
            ws = [LAG] * 3
            ws[d] = [Fraction(1)]
            flo = list(lo)
            flo[d] = (i, j, k)[d]
            for f, r in [(0, 0)] + [(1 + a, 1 + a) for a in range(3)] + [(4 + q, 4 + q) for q in range(6)]:
                ex = _exact_sum(M[f], flo, ws)
                err = abs(Fraction(float(faces[d][r][k, j, i])) - ex) / _abs_sum(M[f], flo, ws)
                worst = max(worst, float(err))
    # 64 rounded fused multiply-adds: a few units of 2^-53 relative to the sum of the terms' magnitudes
    assert worst <= 1e-15, worst
