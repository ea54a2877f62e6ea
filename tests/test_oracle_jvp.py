"""Pins of the oracle's forward-mode derivative: the Jacobian-vector product J dU of the stage operator
L(U) = RHS(ghost fill U, recovery, ghost fill P) and of one classical RK4 step (Sec. 3.12), evaluated with
one-direction dual numbers and, for the recovery, the implicit-function theorem at its root.

The dual evaluation repeats the plain oracle's arithmetic in its value part, so L and the stepped state must
equal the plain path's bit for bit.  Its derivative part must agree with central differences of the plain
oracle (pinned by the other oracle tests) to the truncation and rounding of an extrapolated quotient, and it
must be linear in the direction to rounding.  These make it an exact (rounding-level) reference for the CUDA
adjoint: for outputs weighted by mu, <mu, J d> = <(dL/dU)^T mu, d> for every direction d.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

CELL_LIKE = [(1, 1, 1)] * 5 + [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 0)]
CASES = {
    "ppm_periodic_lorenz": dict(recon=W.RECON_PPM, bc=W.BC_PERIODIC, gauge=W.GAUGE_LORENZ),
    "minmod_copy_lorenz": dict(recon=W.RECON_MINMOD, bc=W.BC_COPY, gauge=W.GAUGE_LORENZ),
    "wenoz_periodic_algebraic": dict(recon=W.RECON_WENOZ, bc=W.BC_PERIODIC, gauge=W.GAUGE_ALGEBRAIC),
    "mp5_copy_lorenz": dict(recon=W.RECON_MP5, bc=W.BC_COPY, gauge=W.GAUGE_LORENZ),
}
GROUPS = [(0,), (1, 2, 3), (1, 2, 3), (1, 2, 3), (4,), (5, 6, 7), (5, 6, 7), (5, 6, 7), (8,)]


def independent(w, v):
    """Owned index range of field v, without the vertex index g+n along periodic axes (the image of g)."""
    g, n = w.g, w.n
    return tuple(slice(g, (g + n[a] - 1 if (CELL_LIKE[v][a] or w.bc[a] == W.BC_PERIODIC) else g + n[a]) + 1)
                 for a in (2, 1, 0))


class Case:
    def __init__(self, name, n=(8, 8, 8), seed=3101):
        w = W.smooth_general(n=n, **CASES[name])
        self.w = w
        self.M = O.metric_array(w)
        U, P = O.initial_state(w)
        O.ghost_fill_state(w, U)
        self.U, self.P = U, P
        self.mask = np.zeros((9,) + w.shape, dtype=bool)
        for v in range(9):
            self.mask[v][independent(w, v)] = True
        scale = np.array([max(np.abs(U[v][self.mask[v]]).max(), 1e-3) for v in range(9)])
        rng = W.Rng(seed)
        self.dirs = [np.where(self.mask, rng.uniform(U.size, -1.0, 1.0).reshape(U.shape), 0.0) *
                     scale[:, None, None, None] for _ in range(2)]

    def stage(self, U):
        X = U.copy()
        O.ghost_fill_state(self.w, X)
        P = self.P.copy()
        O.con2prim(self.w, self.M, X, P)
        O.ghost_fill_prims(self.w, P)
        return O.rhs(self.w, self.M, X, P)[0]

    def rk4(self, U):
        X = U.copy()
        O.ghost_fill_state(self.w, X)
        return O.rk4_step(self.w, self.M, X, self.P.copy())[0]


def richardson(F, U, d, h):
    """Central difference of F at U along d with step h, Richardson-extrapolated from h and 2h: (4 q(h) - q(2h))/3
    cancels the h^2 term of the truncation error (WENO-Z's weights have large third derivatives on smooth data)."""
    def q(k):
        return (F(U + k * d) - F(U - k * d)) / (2.0 * k)
    return (4.0 * q(h) - q(2.0 * h)) / 3.0


def check_against_differences(c, F, JF, d, steps, tol):
    """Each output field on its independent range: max |JF - quotient| <= tol * max |JF| over the field's group,
    for the closest of the step sizes (a switching point of a limiter within h of the state spoils one h)."""
    quot = [richardson(F, c.U, d, h) for h in steps]
    for v in range(9):
        sl = independent(c.w, v)
        scale = max(np.abs(JF[u][independent(c.w, u)]).max() for u in GROUPS[v])
        err = min(np.abs(q[v][sl] - JF[v][sl]).max() for q in quot)
        assert err <= tol * scale, (v, err, scale)


@pytest.mark.parametrize("name", list(CASES))
def test_stage_value_part_is_the_plain_operator(name):
    c = Case(name)
    L, JL = O.stage_jvp(c.w, c.M, c.U, c.dirs[0], c.P.copy())
    ref = c.stage(c.U)
    for v in range(9):
        sl = independent(c.w, v)
        assert np.array_equal(L[v][sl], ref[v][sl]), v
    assert np.all(np.isfinite(JL))


@pytest.mark.parametrize("name", list(CASES))
def test_stage_derivative_matches_central_differences(name):
    c = Case(name)
    _, JL = O.stage_jvp(c.w, c.M, c.U, c.dirs[0], c.P.copy())
    check_against_differences(c, c.stage, JL, c.dirs[0], (1e-6, 2.5e-7), 1e-8)


def test_stage_derivative_of_each_input_group():
    """Directions confined to one input group (D~ | S~ | tau~ | A | Psi): catches a term dropped from one input's
    chain that the all-fields direction could hide behind a larger one."""
    c = Case("ppm_periodic_lorenz", n=(7, 8, 6), seed=3102)
    for grp in [(0,), (1, 2, 3), (4,), (5, 6, 7), (8,)]:
        d = np.zeros_like(c.U)
        for v in grp:
            d[v] = c.dirs[1][v]
        L, JL = O.stage_jvp(c.w, c.M, c.U, d, c.P.copy())
        steps = (4e-6, 1e-6)
        quot = [richardson(c.stage, c.U, d, h) for h in steps]
        total = max(np.abs(JL[v][independent(c.w, v)]).max() for v in range(9))
        for v in range(9):
            sl = independent(c.w, v)
            err = min(np.abs(q[v][sl] - JL[v][sl]).max() for q in quot)
            # the quotient's rounding, eps |L_v| / h, dominates where this group moves L_v only weakly
            floor = 16.0 * np.finfo(float).eps * np.abs(L[v][sl]).max() / steps[0]
            assert err <= 1e-8 * total + floor, (grp, v, err, total, floor)


def test_stage_derivative_is_linear_in_the_direction():
    c = Case("wenoz_periodic_algebraic", seed=3103)
    d1, d2 = c.dirs
    outs = [O.stage_jvp(c.w, c.M, c.U, d, c.P.copy())[1] for d in (d1, d2, 2.0 * d1 - 3.0 * d2)]
    comb = 2.0 * outs[0] - 3.0 * outs[1]
    for v in range(9):
        sl = independent(c.w, v)
        assert np.abs(outs[2][v][sl] - comb[v][sl]).max() <= 1e-12 * np.abs(comb[v][sl]).max(), v
    _, J0 = O.stage_jvp(c.w, c.M, c.U, np.zeros_like(c.U), c.P.copy())
    assert np.all(J0 == 0.0)


@pytest.mark.parametrize("name", ["wenoz_periodic_algebraic", "minmod_copy_lorenz"])
def test_rk4_value_part_and_derivative(name):
    """Over the four stages PPM's monotonicity switches put some stage state within any usable h of a branch
    point (the quotient is then one-sided at every h), so the step is checked with WENO-Z and minmod."""
    c = Case(name, n=(8, 7, 8), seed=3104)
    U1, JU1 = O.rk4_jvp(c.w, c.M, c.U, c.dirs[0], c.P.copy())
    ref = c.rk4(c.U)
    for v in range(9):
        sl = independent(c.w, v)
        assert np.array_equal(U1[v][sl], ref[v][sl]), v
    check_against_differences(c, c.rk4, JU1, c.dirs[0], (1e-6, 2.5e-7), 1e-8)


def test_prim2con_derivative():
    """The initial-data map (A, rho, p, v^i) -> (D~, S~, tau~): the dual evaluation's value part equals the plain
    prim->cons bit for bit, its derivative matches extrapolated central differences of the plain map (smooth and
    pointwise after B~ = curl A, so to 1e-9 of each field's scale), and it is linear in the direction."""
    w = W.smooth_general(n=(8, 7, 6), seed=3105)
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    O.ghost_fill_prims(w, P)
    rng = W.Rng(3106)
    dirs = []
    for _ in range(2):
        dA = rng.uniform(3 * U[0].size, -1.0, 1.0).reshape((3,) + U.shape[1:]) * 0.01
        dP = rng.uniform(P.size, -1.0, 1.0).reshape(P.shape) * np.array([0.05, 0.05, 0.1, 0.1, 0.1])[:, None, None,
                                                                                                        None]
        dirs.append((dA, dP))

    def F(s, dA, dP):
        X = U.copy()
        X[5:8] += s * dA
        O.prim2con(w, M, X, P + s * dP)
        return X[:5]

    X = U.copy()
    J = O.prim2con_jvp(w, M, X, dirs[0][0], P, dirs[0][1])
    ref = F(0.0, *dirs[0])
    owned = (slice(w.g, w.g + w.n[2]), slice(w.g, w.g + w.n[1]), slice(w.g, w.g + w.n[0]))
    assert np.array_equal(X[:5], ref)

    def q(h):
        return (F(h, *dirs[0]) - F(-h, *dirs[0])) / (2.0 * h)
    rich = (4.0 * q(1e-4) - q(2e-4)) / 3.0
    for v in range(5):
        scale = np.abs(J[v][owned]).max()
        assert scale > 0.0, v
        assert np.abs(rich[v][owned] - J[v][owned]).max() <= 1e-9 * scale, v
    # dropping the potentials' direction changes the result (the B~ = curl A chain is live), and the map is linear
    J1 = O.prim2con_jvp(w, M, U.copy(), dirs[1][0], P, dirs[1][1])
    J2 = O.prim2con_jvp(w, M, U.copy(), 2.0 * dirs[0][0] - 3.0 * dirs[1][0], P, 2.0 * dirs[0][1] - 3.0 * dirs[1][1])
    comb = 2.0 * J - 3.0 * J1
    assert np.abs(J2[:, owned[0], owned[1], owned[2]] - comb[:, owned[0], owned[1], owned[2]]).max() <= \
        1e-12 * np.abs(comb[:, owned[0], owned[1], owned[2]]).max()
    Jp = O.prim2con_jvp(w, M, U.copy(), np.zeros_like(dirs[0][0]), P, dirs[0][1])
    assert np.abs(Jp[1:][:, owned[0], owned[1], owned[2]] - J[1:][:, owned[0], owned[1], owned[2]]).max() > \
        1e-6 * np.abs(J[1:][:, owned[0], owned[1], owned[2]]).max()
