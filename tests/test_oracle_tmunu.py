"""Pins of the oracle's stress-energy tensor at vertices (Eq. tmunu, stored at vertices per Sec. 3.1).

A uniform state on a constant, general metric (lapse, shift, non-diagonal gamma_ij) gives the same T_{mu nu} at
every vertex, and its projections must reproduce the oracle's pinned prim->cons map and fluxes: the Eulerian
energy density n^mu n^nu T_{mu nu} = (tau~ + D~) / sqrt(gamma), the momentum density -n^mu T_{mu i} =
S~_i / sqrt(gamma), and the momentum flux T^i_j = (alpha sqrt(gamma) F^i(S_j)) / (alpha sqrt(gamma)).  These
three fix all ten components.  Two invariants hold for any state: the trace g^{mu nu} T_{mu nu} = 4p - rho h
(the field part is traceless), and u^mu u^nu T_{mu nu} = rho (1 + eps) + b^2 / 2.  Linear rho and p at rest
on a static diagonal metric locate the vertex: the average of the eight cells around it is then the value at
the vertex itself, T_tt = alpha^2 (rho + p / (Gamma - 1)) and T_ij = p gamma_ij there.
"""
import numpy as np

import oracle as O
from paper_2406_11669_gb300 import workloads as W

SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
IDX = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def block(n=(5, 4, 6), gamma=5.0 / 3.0):
    w = W.flat_modes(n=n)
    w.params = dict(w.params, gamma=gamma)
    return w


def constant_metric(w, alp, beta, g6, k6=(0.01, 0.0, -0.02, 0.0, 0.03, 0.0)):
    M = np.zeros((16,) + w.shape)
    M[0] = alp
    for a in range(3):
        M[1 + a] = beta[a]
    for a in range(6):
        M[4 + a] = g6[a]
        M[10 + a] = k6[a]
    return M


def vertex_positions(w):
    g = w.g
    x = [w.x0[a] + (np.arange(w.N[a] + 1) - g) * w.dx[a] for a in range(3)]
    return x


def potentials_for(w, Bt):
    """Edge A_i whose discrete curl is the uniform densitised field Bt (A linear: the curl is exact)."""
    x = vertex_positions(w)
    h = [0.5 * w.dx[a] for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    U = np.zeros((9,) + w.shape)
    U[5] = 0.5 * (Bt[1] * Z - Bt[2] * Y)                 # A_x at (x + h, y, z): no x dependence
    U[6] = 0.5 * (Bt[2] * X - Bt[0] * Z)
    U[7] = 0.5 * (Bt[0] * Y - Bt[1] * X)
    del h
    return U


def full4(m16):
    alp, beta = m16[0], np.array(m16[1:4])
    g = np.array([[m16[4 + SYM[a][b]] for b in range(3)] for a in range(3)])
    blow = g @ beta
    gdd = np.zeros((4, 4))
    gdd[0, 0] = -alp ** 2 + blow @ beta
    gdd[0, 1:] = gdd[1:, 0] = blow
    gdd[1:, 1:] = g
    return gdd, np.linalg.inv(gdd), g


def tensor_at(T, v):
    t = np.zeros((4, 4))
    for q, (a, b) in enumerate(IDX):
        t[a, b] = t[b, a] = T[q][v]
    return t


def owned_vertices(w):
    g, n = w.g, w.n
    return (slice(g, g + n[2] + 1), slice(g, g + n[1] + 1), slice(g, g + n[0] + 1))


def test_uniform_state_projections_match_prim2con_and_fluxes():
    w = block()
    m16 = np.array([0.83, 0.05, -0.03, 0.02, 1.2, 0.1, -0.05, 1.1, 0.07, 1.3, 0, 0, 0, 0, 0, 0], float)
    M = constant_metric(w, m16[0], m16[1:4], m16[4:10])
    gdd, guu, g3 = full4(m16)
    sqg = np.sqrt(np.linalg.det(g3))
    prim5 = np.array([0.7, 0.3, 0.2, -0.15, 0.1])
    Bt = np.array([0.4, -0.25, 0.3]) * sqg          # uniform undensitised B = (0.4, -0.25, 0.3)
    P = np.zeros((5,) + w.shape)
    for r in range(5):
        P[r] = prim5[r]
    U = potentials_for(w, Bt)
    T = O.tmunu(w, M, U, P)
    cons, fl = O.point_prim2con(w.params, m16, prim5, Bt / sqg)
    alp, beta = m16[0], m16[1:4]
    n_up = np.array([1.0 / alp, *(-beta / alp)])
    sl = owned_vertices(w)
    idx = np.argwhere(np.ones(T[0][sl].shape, bool))
    assert len(idx) == np.prod([w.n[a] + 1 for a in range(3)])
    ref = tensor_at(T, tuple(s.start for s in sl))
    for q in range(10):  # the same tensor at every owned vertex
        assert np.abs(T[q][sl] - T[q][sl].flat[0]).max() <= 1e-14 * np.abs(ref).max()
    E = n_up @ ref @ n_up
    assert abs(E - (cons[4] + cons[0]) / sqg) <= 1e-13 * abs(E)
    S = -(n_up @ ref)[1:]
    assert np.abs(S - cons[1:4] / sqg).max() <= 1e-13 * np.abs(S).max()
    mixed = guu @ ref  # T^mu_nu
    for i in range(3):
        for j in range(3):
            Fij = fl[i][1 + j] / (alp * sqg)
            assert abs(mixed[1 + i, 1 + j] - Fij) <= 1e-13 * np.abs(fl).max() / (alp * sqg), (i, j)
    # invariants: trace and the comoving energy density
    gam = w.params["gamma"]
    rho, p = prim5[0], prim5[1]
    eps = p / ((gam - 1.0) * rho)
    h = 1.0 + eps + p / rho
    assert abs(np.sum(guu * ref) - (4.0 * p - rho * h)) <= 1e-13 * rho * h
    v = prim5[2:]
    W_ = 1.0 / np.sqrt(1.0 - v @ g3 @ v)
    u_up = np.array([W_ / alp, *(W_ * (v - beta / alp))])
    Bu = Bt / sqg
    Bv = Bu @ g3 @ v
    b0 = W_ * Bv / alp
    b2 = (Bu @ g3 @ Bu + alp ** 2 * b0 ** 2) / W_ ** 2
    assert abs(u_up @ ref @ u_up - (rho * (1.0 + eps) + 0.5 * b2)) <= 1e-13 * rho * h


def test_linear_fields_at_rest_locate_the_vertex():
    w = block(n=(6, 5, 4), gamma=4.0 / 3.0)
    alp = 0.9
    g6 = (1.3, 0.0, 0.0, 1.1, 0.0, 0.95)
    M = constant_metric(w, alp, (0.0, 0.0, 0.0), g6, k6=(0.0,) * 6)
    x = vertex_positions(w)
    c = [xi[:-1] + 0.5 * w.dx[a] for a, xi in enumerate(x)]   # cell centres
    Zc, Yc, Xc = np.meshgrid(np.append(c[2], 0), np.append(c[1], 0), np.append(c[0], 0), indexing="ij")
    rho = 1.0 + 0.3 * Xc - 0.2 * Yc + 0.1 * Zc
    p = 0.5 + 0.1 * Xc + 0.25 * Yc - 0.15 * Zc
    P = np.zeros((5,) + w.shape)
    P[0], P[1] = rho, p
    U = np.zeros((9,) + w.shape)
    T = O.tmunu(w, M, U, P)
    Zv, Yv, Xv = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    rv = 1.0 + 0.3 * Xv - 0.2 * Yv + 0.1 * Zv
    pv = 0.5 + 0.1 * Xv + 0.25 * Yv - 0.15 * Zv
    sl = owned_vertices(w)
    gam = w.params["gamma"]
    assert np.abs(T[0][sl] - alp ** 2 * (rv + pv / (gam - 1.0))[sl]).max() <= 1e-13
    for q, (a, b) in enumerate(IDX):
        if a == 0 and b > 0:
            assert np.abs(T[q][sl]).max() == 0.0
        elif a > 0:
            assert np.abs(T[q][sl] - pv[sl] * g6[SYM[a - 1][b - 1]]).max() <= 1e-13
    # nothing outside the owned vertices
    mask = np.zeros(w.shape, bool)
    mask[sl] = True
    assert np.all(T[:, ~mask] == 0.0)


def test_smooth_state_is_finite_and_symmetric_in_its_inputs():
    """On a general workload T_tt > 0 (the energy density seen by the coordinate observer is positive for a
    static-ish metric) and the spatial block is positive definite (pressure plus a rank-one kinetic part minus a
    field part bounded by the magnetic pressure)."""
    w = W.smooth_general(n=(6, 6, 6))
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    O.ghost_fill_prims(w, P)
    M = O.metric_array(w)
    T = O.tmunu(w, M, U, P)
    sl = owned_vertices(w)
    assert np.all(np.isfinite(T))
    assert np.all(T[0][sl] > 0.0)
    Ts = np.stack([np.stack([T[4 + [0, 1, 2, 1, 3, 4, 2, 4, 5][3 * a + b]][sl] for b in range(3)], -1)
                   for a in range(3)], -2)
    assert np.all(np.linalg.eigvalsh(Ts) > 0.0)
