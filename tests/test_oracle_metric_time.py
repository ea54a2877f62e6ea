"""Pin of the RK4 step over a time-dependent metric (each stage on the spacetime of its stage time).

In flat space with a lapse that depends on time only (beta = 0, gamma = identity, K = 0, a consistent slicing of
Minkowski space), every term of the right-hand side carries one factor alpha: the fluxes alpha sqrt(gamma) F
and the wave speeds, v~ = alpha v in the electric field, G_A = alpha Psi, F_Psi = alpha A and the damping
-xi alpha Psi, while the sources vanish; so L_alpha(U) = alpha L_1(U).  An RK4 step whose stages run on lapses
a_0..a_3 must then equal classical RK4 written out with the stage slopes a_s L_1(U_s):
U_1 = U_n + dt/2 a_0 L_1(U_n), U_2 = U_n + dt/2 a_1 L_1(U_1), U_3 = U_n + dt a_2 L_1(U_2),
U_{n+1} = U_n + dt/6 (a_0 L_1(U_n) + 2 a_1 L_1(U_1) + 2 a_2 L_1(U_2) + a_3 L_1(U_3)).
A stage that ran on another stage's metric, or a term without its lapse factor, breaks the equality.  (A
convergence test in dt cannot show this cleanly: HLLE's c_max = max(0, lambda_L, lambda_R) switches sides
wherever the two reconstructed speeds cross, so the semi-discrete right-hand side has kinks throughout a
smooth flow and RK4's local error is not O(dt^5) there.)
"""
import numpy as np

import oracle as O
from paper_2406_11669_gb300 import workloads as W

LAPSES = (1.0, 1.21, 0.87, 1.34)


def owned(w, v):
    g, n = w.g, w.n
    cell = [(1, 1, 1)] * 5 + [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 0)]
    return tuple(slice(g, g + n[a] + (0 if cell[v][a] else 1)) for a in (2, 1, 0))


def test_stage_lapses_scale_the_stage_slopes():
    w = W.flat_modes(n=(7, 6, 8))
    w.params = dict(w.params, recon=W.RECON_PPM, xi_lorenz=10.0)
    M1 = O.metric_array(w)
    U0, P0 = O.initial_state(w)
    O.ghost_fill_state(w, U0)
    dt = w.dt
    Ms = []
    for a in LAPSES:
        M = M1.copy()
        M[0] = a
        Ms.append(M)
    got, st = O.rk4_step_metrics(w, Ms, U0.copy(), P0.copy(), dt)
    assert st["n_atm"] == 0 and st["n_failed"] == 0

    P = P0.copy()

    def L1(U):
        X = U.copy()
        O.ghost_fill_state(w, X)
        O.con2prim(w, M1, X, P)
        O.ghost_fill_prims(w, P)
        return O.rhs(w, M1, X, P, dt=dt)[0]

    k0 = LAPSES[0] * L1(U0)
    k1 = LAPSES[1] * L1(U0 + 0.5 * dt * k0)
    k2 = LAPSES[2] * L1(U0 + 0.5 * dt * k1)
    k3 = LAPSES[3] * L1(U0 + dt * k2)
    ref = U0 + dt / 6.0 * (k0 + 2.0 * k1 + 2.0 * k2 + k3)
    for v in range(9):
        sl = owned(w, v)
        scale = np.abs(ref[v][sl] - U0[v][sl]).max()  # the step's increment
        assert np.abs(got[v][sl] - ref[v][sl]).max() <= 1e-11 * scale, v
    # and not the frozen-lapse step
    frozen, _ = O.rk4_step(w, Ms[0], U0.copy(), P0.copy(), dt)
    assert np.abs(frozen[0][owned(w, 0)] - ref[0][owned(w, 0)]).max() > 1e-3 * np.abs(
        ref[0][owned(w, 0)] - U0[0][owned(w, 0)]).max()


def test_constant_stage_metrics_reproduce_the_frozen_step():
    w = W.smooth_general(n=(6, 5, 7))
    M = O.metric_array(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    a, _ = O.rk4_step_metrics(w, [M] * 4, U.copy(), P.copy())
    b, _ = O.rk4_step(w, M, U.copy(), P.copy())
    assert np.array_equal(a, b)
