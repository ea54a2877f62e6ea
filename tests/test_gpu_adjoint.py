"""The adjoint (vector-Jacobian product) of the stage right-hand side and of one RK4 step, against central
differences of the oracle's forward operator on the same inputs.

For a weight mu on the outputs, the CUDA adjoint returns lam = (dL/dU)^T mu.  The oracle gives
J(U) = <mu, L(U)> for any U, so for a direction v the directional derivative <lam, v> must equal
(J(U + h v) - J(U - h v)) / 2h up to O(h^2) truncation and rounding of order eps |L| / h; with h between 1e-8
and 1e-6 in units of each field's magnitude both stay below 1e-8 of sum |lam v|.  The limiters, max/min and
recovery branches make L piecewise smooth: where a switching surface lies within h of the state the quotient is
one-sided at that h, so each check takes the closest of three step sizes (a wrong adjoint is off at all of
them).  Two kinds of check: one direction per field group (all independent entries of D~ | S~ | tau~ | A | Psi at
once), and single entries at the middle and at the ends of every field's independent range (where the ghost zones and
the boundary conditions act).  The workloads vary smoothly in every direction, so that no limiter sits exactly
at a branch point; copy boundary conditions are checked with minmod, whose slopes in the ghost zones are exactly
zero for every state.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, independent
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HS = (1e-6, 1e-7, 1e-8)
RTOL = 1e-6
IN_GROUPS = [(0,), (1, 2, 3), (4,), (5, 6, 7), (8,)]

CASES = {
    "ppm_periodic_lorenz": dict(recon=W.RECON_PPM, bc=W.BC_PERIODIC, gauge=W.GAUGE_LORENZ),
    "minmod_copy_lorenz": dict(recon=W.RECON_MINMOD, bc=W.BC_COPY, gauge=W.GAUGE_LORENZ),
    "wenoz_periodic_algebraic": dict(recon=W.RECON_WENOZ, bc=W.BC_PERIODIC, gauge=W.GAUGE_ALGEBRAIC),
}


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def independent_mask(w):
    m = np.zeros((9,) + w.shape, dtype=bool)
    for v in range(9):
        m[v][independent(w, v)] = True
    return m


class Problem:
    """A workload with its oracle state, primitives and seeded weights."""

    def __init__(self, w, seed):
        self.w = w
        self.M = O.metric_array(w)
        U, P = O.initial_state(w)
        O.ghost_fill_state(w, U)
        self.U, self.P = U, P
        self.mask = independent_mask(w)
        rng = W.Rng(seed)
        self.uscale = np.array([max(np.abs(U[v][independent(w, v)]).max(), 1e-3) for v in range(9)])
        self.r_mu = rng.uniform(9 * int(np.prod(w.shape)), -1.0, 1.0).reshape((9,) + w.shape)
        self.r_v = rng.uniform(9 * int(np.prod(w.shape)), -1.0, 1.0).reshape((9,) + w.shape)

    def stage_rhs(self, U):
        """L(U): the oracle's stage operator from the independent entries of U (ghost fill, recovery warm-started
        from the unperturbed primitives, primitive ghost fill, right-hand side)."""
        w = self.w
        X = U.copy()
        O.ghost_fill_state(w, X)
        P = self.P.copy()
        O.con2prim(w, self.M, X, P)
        O.ghost_fill_prims(w, P)
        dU, _ = O.rhs(w, self.M, X, P)
        return np.where(self.mask, dU, 0.0)

    def rk4(self, U):
        X = U.copy()
        O.ghost_fill_state(self.w, X)
        U1, st = O.rk4_step(self.w, self.M, X, self.P.copy())
        assert st["n_atm"] == 0 and st["n_failed"] == 0
        return np.where(self.mask, U1, 0.0)

    def mu_for(self, out):
        """Weights on the independent outputs, each field scaled by 1 / its magnitude so that all fields count."""
        sc = np.array([max(np.abs(out[v]).max(), 1e-300) for v in range(9)])
        return np.where(self.mask, self.r_mu / sc[:, None, None, None], 0.0)


def directional(F, mu, U, d, h):
    """<mu, (F(U + h d) - F(U - h d)) / 2h>, the difference taken entry by entry before the weighted sum."""
    return float(np.sum(mu * (F(U + h * d) - F(U - h * d)))) / (2.0 * h)


def closest(F, mu, U, d, target, steps):
    return min((directional(F, mu, U, d, h) for h in steps), key=lambda fd: abs(fd - target))


def sample_entries(w, v, full):
    """(z, y, x) indices: the two corners of the field's independent range, and (full) its middle and a mixed
    corner."""
    sl = independent(w, v)
    lo = tuple(s.start for s in sl)
    hi = tuple(s.stop - 1 for s in sl)
    mid = tuple((a + b) // 2 for a, b in zip(lo, hi))
    return [lo, hi, mid, (lo[0], mid[1], hi[2])] if full else [lo, hi]


def check_vjp(prob, F, lam, full_entries=True):
    """Compares lam with central differences of J(U) = <mu, F(U)>: per input group, then per sampled entry."""
    w, U = prob.w, prob.U
    mu = prob.mu_for(F(U))
    for grp in IN_GROUPS:
        d = np.zeros_like(U)
        for v in grp:
            d[v] = np.where(prob.mask[v], prob.r_v[v] * prob.uscale[v], 0.0)
        ad = float(np.sum(lam * d))
        fd = closest(F, mu, U, d, ad, HS)
        scale = float(np.sum(np.abs(lam * d)))
        assert abs(ad - fd) <= RTOL * scale, (grp, ad, fd, scale)
    for v in range(9):
        lmax = np.abs(lam[v][prob.mask[v]]).max()
        for idx in sample_entries(w, v, full_entries):
            d = np.zeros_like(U)
            d[(v,) + idx] = prob.uscale[v]
            ad = lam[(v,) + idx]
            fd = closest(F, mu, U, d, ad * prob.uscale[v], HS[:2]) / prob.uscale[v]
            assert abs(ad - fd) <= RTOL * max(lmax, abs(fd)), (v, idx, ad, fd, lmax)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_adjoint_matches_central_differences(name):
    need_gpu()
    w = W.smooth_general(**CASES[name])
    prob = Problem(w, seed=2201)
    mu = prob.mu_for(prob.stage_rhs(prob.U))
    case = GpuCase(w)
    lam_d = case.solver.zeros_state()
    P_d = case.dev(prob.P)
    case.solver.rhs_adjoint(case.dev(prob.U), P_d, case.dev(mu), lam_d, w.dt)
    lam = case.host(lam_d)
    assert np.all(lam[~prob.mask] == 0.0)
    assert np.all(np.isfinite(lam))
    check_vjp(prob, prob.stage_rhs, lam)


@pytest.mark.parametrize("name", ["ppm_periodic_lorenz", "minmod_copy_lorenz"])
def test_rk4_step_adjoint_matches_central_differences(name):
    need_gpu()
    w = W.smooth_general(n=(10, 9, 8), **CASES[name])
    prob = Problem(w, seed=2202)
    mu = prob.mu_for(prob.rk4(prob.U))
    case = GpuCase(w)
    lam_d = case.dev(mu)
    case.solver.rk4_step_adjoint(case.dev(prob.U), case.dev(prob.P), lam_d, w.dt)
    lam = case.host(lam_d)
    assert np.all(lam[~prob.mask] == 0.0)
    check_vjp(prob, prob.rk4, lam, full_entries=False)


def check_against_jvp(prob, mu, lam, jvp, entries_full=True, rtol=1e-11):
    """<lam, d> against <mu, J d> with J d from the oracle's dual-number derivative (no truncation error: the two
    agree to rounding and the recovery's root tolerance): one random direction over every independent entry, one
    per input group, then unit directions at the sampled entries of every field (lam_i = <mu, J e_i>)."""
    w, U = prob.w, prob.U
    dirs = [np.where(prob.mask, prob.r_v, 0.0) * prob.uscale[:, None, None, None]]
    for grp in IN_GROUPS:
        d = np.zeros_like(U)
        for v in grp:
            d[v] = dirs[0][v]
        dirs.append(d)
    worst = 0.0
    for d in dirs:
        Jd = jvp(d)
        ad, ref = float(np.sum(lam * d)), float(np.sum(mu * Jd))
        scale = max(float(np.sum(np.abs(lam * d))), float(np.sum(np.abs(mu * Jd))), 1e-300)
        worst = max(worst, abs(ad - ref) / scale)
        assert abs(ad - ref) <= rtol * scale, (ad, ref, scale)
    for v in range(9):
        for idx in sample_entries(w, v, entries_full):
            d = np.zeros_like(U)
            d[(v,) + idx] = 1.0
            Jd = jvp(d)
            ad, ref = float(lam[(v,) + idx]), float(np.sum(mu * Jd))
            scale = max(float(np.sum(np.abs(mu * Jd))), 1e-300)
            worst = max(worst, abs(ad - ref) / scale)
            assert abs(ad - ref) <= rtol * scale, (v, idx, ad, ref, scale)
    return worst


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_adjoint_equals_the_oracle_jvp(name):
    need_gpu()
    w = W.smooth_general(**CASES[name])
    prob = Problem(w, seed=2206)
    mu = prob.mu_for(prob.stage_rhs(prob.U))
    case = GpuCase(w)
    lam_d = case.solver.zeros_state()
    case.solver.rhs_adjoint(case.dev(prob.U), case.dev(prob.P), case.dev(mu), lam_d, w.dt)
    lam = case.host(lam_d)
    worst = check_against_jvp(prob, mu, lam, lambda d: O.stage_jvp(w, prob.M, prob.U, d, prob.P.copy())[1])
    print(f"{name}: largest relative difference {worst:.2e}")


@pytest.mark.parametrize("name", list(CASES))
def test_rk4_step_adjoint_equals_the_oracle_jvp(name):
    need_gpu()
    w = W.smooth_general(n=(10, 9, 8), **CASES[name])
    prob = Problem(w, seed=2207)
    mu = prob.mu_for(prob.rk4(prob.U))
    case = GpuCase(w)
    lam_d = case.dev(mu)
    case.solver.rk4_step_adjoint(case.dev(prob.U), case.dev(prob.P), lam_d, w.dt)
    lam = case.host(lam_d)
    worst = check_against_jvp(prob, mu, lam, lambda d: O.rk4_jvp(w, prob.M, prob.U, d, prob.P.copy())[1],
                              entries_full=False)
    print(f"{name}: largest relative difference {worst:.2e}")


SWITCHES = {"lxf": dict(flux=W.FLUX_LXF), "fct": dict(efield=W.EFIELD_FCT),
            "lxf_fct": dict(flux=W.FLUX_LXF, efield=W.EFIELD_FCT)}


@pytest.mark.parametrize("sw", list(SWITCHES))
@pytest.mark.parametrize("name", ["ppm_periodic_lorenz", "minmod_copy_lorenz"])
def test_rhs_adjoint_of_the_scheme_switches_equals_the_oracle_jvp(name, sw):
    """The Lax-Friedrichs and flux-CT switches differentiated: the oracle's dual-number derivative follows the
    switches through the same face solve and electric field code."""
    need_gpu()
    w = W.smooth_general(**CASES[name])
    w.params = dict(w.params, **SWITCHES[sw])
    prob = Problem(w, seed=2208)
    mu = prob.mu_for(prob.stage_rhs(prob.U))
    case = GpuCase(w)
    lam_d = case.solver.zeros_state()
    case.solver.rhs_adjoint(case.dev(prob.U), case.dev(prob.P), case.dev(mu), lam_d, w.dt)
    lam = case.host(lam_d)
    worst = check_against_jvp(prob, mu, lam, lambda d: O.stage_jvp(w, prob.M, prob.U, d, prob.P.copy())[1])
    print(f"{name} {sw}: largest relative difference {worst:.2e}")


def test_rk4_step_adjoint_of_the_scheme_switches_equals_the_oracle_jvp():
    need_gpu()
    w = W.smooth_general(n=(10, 9, 8), **CASES["wenoz_periodic_algebraic"])
    w.params = dict(w.params, flux=W.FLUX_LXF, efield=W.EFIELD_FCT)
    prob = Problem(w, seed=2209)
    mu = prob.mu_for(prob.rk4(prob.U))
    case = GpuCase(w)
    lam_d = case.dev(mu)
    case.solver.rk4_step_adjoint(case.dev(prob.U), case.dev(prob.P), lam_d, w.dt)
    lam = case.host(lam_d)
    worst = check_against_jvp(prob, mu, lam, lambda d: O.rk4_jvp(w, prob.M, prob.U, d, prob.P.copy())[1],
                              entries_full=False)
    print(f"lxf_fct rk4: largest relative difference {worst:.2e}")


def test_rhs_adjoint_is_linear_in_the_weights():
    """J^T (2 mu1 - 3 mu2) = 2 J^T mu1 - 3 J^T mu2 up to the summation order of the atomic accumulations."""
    need_gpu()
    w = W.smooth_general(**CASES["ppm_periodic_lorenz"])
    prob = Problem(w, seed=2203)
    case = GpuCase(w)
    rng = W.Rng(77)
    m1 = np.where(prob.mask, rng.uniform(prob.U.size, -1.0, 1.0).reshape(prob.U.shape), 0.0)
    m2 = np.where(prob.mask, rng.uniform(prob.U.size, -1.0, 1.0).reshape(prob.U.shape), 0.0)
    out = []
    for m in (m1, m2, 2.0 * m1 - 3.0 * m2):
        lam_d = case.solver.zeros_state()
        case.solver.rhs_adjoint(case.dev(prob.U), case.dev(prob.P), case.dev(m), lam_d, w.dt)
        out.append(case.host(lam_d))
    comb = 2.0 * out[0] - 3.0 * out[1]
    for v in range(9):
        scale = np.abs(comb[v]).max()
        assert np.abs(out[2][v] - comb[v]).max() <= 1e-12 * scale, v


def test_loss_gradient_through_steps_and_initial_data():
    """Gradient of J = 1/2 sum_interior (D~_N - T)^2 after N = 2 RK4 steps with respect to the initial primitives,
    and potentials: forward with checkpoints, reverse through the steps and the initial data (prim->cons with
    B~ = curl A), against central differences of the oracle's whole pipeline at sampled entries."""
    need_gpu()
    nsteps = 2
    w = W.smooth_general(n=(9, 8, 10), seed=107, **CASES["ppm_periodic_lorenz"])
    M = O.metric_array(w)
    P0 = O.prims_array(w)
    base = np.zeros((9,) + w.shape)
    base[5], base[6], base[7], base[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
    mask = independent_mask(w)
    g, n = w.g, w.n
    inter = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    rng = W.Rng(2204)
    T = 1.0 + 0.01 * rng.uniform(int(np.prod(w.shape)), -1.0, 1.0).reshape(w.shape)

    def loss(P, pot):
        U = np.where(mask, pot, 0.0)
        O.ghost_fill_state(w, U)
        O.prim2con(w, M, U, P)
        Pw = P.copy()
        for _ in range(nsteps):
            U, st = O.rk4_step(w, M, U, Pw)
            assert st["n_atm"] == 0
        return 0.5 * float(np.sum((U[0][inter] - T[inter]) ** 2))

    case = GpuCase(w)
    s = case.solver
    U = case.dev(base)
    s.fill_ghosts(U)
    P = case.dev(P0)
    s.prim2con(U, P)
    U0 = U.clone()
    ckpt = [s.zeros_state() for _ in range(nsteps)]
    s.rk4_steps_checkpointed(U, P, w.dt, ckpt)
    lam = torch.zeros_like(U)
    Tt = case.dev(T)
    ii = (0,) + inter
    lam[ii] = U[ii] - Tt[inter]
    s.rk4_adjoint_steps(ckpt, P, lam, w.dt)
    lamP = s.zeros_prims()
    s.prim2con_adjoint(U0, case.dev(P0), lam, lamP)
    gP, gU = case.host(lamP), case.host(lam)
    assert np.all(gU[:5] == 0.0) and np.all(gU[~mask] == 0.0)

    def check(ad, gmax, quotient):
        """ad against the difference quotient at h = 1e-5, and at 1e-6 if a switching point spoils the first.
        (J is a sum of squares of small residuals, whose rounding swamps the quotient for h below 1e-6.)"""
        fd = quotient(1e-5)
        if abs(ad - fd) > 1e-6 * max(gmax, abs(fd)):
            fd = quotient(1e-6)
        return abs(ad - fd) <= 1e-6 * max(gmax, abs(fd)), fd

    def perturbed(arr, v, idx, d):
        x = arr.copy()
        x[(v,) + idx] += d
        return x

    lo = tuple(sl.start for sl in inter)
    hi = tuple(sl.stop - 1 for sl in inter)
    mid = tuple((a + b) // 2 for a, b in zip(lo, hi))
    for r in range(5):
        scale = max(np.abs(P0[r][inter]).max(), 0.05)
        gmax = np.abs(gP[r][inter]).max()
        for idx in (lo, mid, hi):
            ok, fd = check(gP[(r,) + idx], gmax, lambda h: (loss(perturbed(P0, r, idx, h * scale), base) -
                                                            loss(perturbed(P0, r, idx, -h * scale), base)) /
                           (2.0 * h * scale))
            assert ok, (r, idx, gP[(r,) + idx], fd)
    # Psi enters the update of A only through the discrete gradient of G_A, which the discrete curl annihilates,
    # so D~ (and J) does not depend on it: its gradient is zero up to rounding
    amax = max(np.abs(gU[v][independent(w, v)]).max() for v in (5, 6, 7))
    assert np.abs(gU[8]).max() <= 1e-12 * amax
    for v in (5, 6, 7):
        sl = independent(w, v)
        scale = max(np.abs(base[v][sl]).max(), 1e-3)
        gmax = np.abs(gU[v][sl]).max()
        lo_v = tuple(x.start for x in sl)
        mid_v = tuple((x.start + x.stop - 1) // 2 for x in sl)
        for idx in (lo_v, mid_v):
            ok, fd = check(gU[(v,) + idx], gmax, lambda h: (loss(P0, perturbed(base, v, idx, h * scale)) -
                                                            loss(P0, perturbed(base, v, idx, -h * scale))) /
                           (2.0 * h * scale))
            assert ok, (v, idx, gU[(v,) + idx], fd)


def test_stage_adjoints_compose_to_the_step_adjoint():
    """Four asterx_rk_stage_adjoint calls with the linear RK4 bookkeeping reproduce asterx_rk4_step_adjoint."""
    need_gpu()
    w = W.smooth_general(n=(10, 9, 8), seed=108, **CASES["minmod_copy_lorenz"])
    prob = Problem(w, seed=2205)
    case = GpuCase(w)
    s = case.solver
    dt = w.dt
    # forward stages (the checkpoints Y0..Y3)
    Y = [case.dev(prob.U)]
    acc = s.zeros_state()
    P = case.dev(prob.P)
    for st in range(3):
        nxt = Y[-1].clone()
        s.rk_stage(st, dt, Y[0], Y[st], nxt, acc, P)
        Y.append(nxt)
    lam = case.dev(np.where(prob.mask, prob.r_mu, 0.0))
    # reverse: k-bar weights through the stages, U_n collects every stage input's adjoint plus lam
    total = lam.clone()
    lam_s = s.zeros_state()
    s.rk_stage_adjoint(3, dt, Y[3], P, lam, None, lam_s)
    total += lam_s
    lam_acc = lam.clone()
    lam_next = lam_s
    for st in (2, 1, 0):
        out = s.zeros_state()
        s.rk_stage_adjoint(st, dt, Y[st], P, lam_next, lam_acc, out)
        total += out
        lam_next = out
    ref = case.dev(np.where(prob.mask, prob.r_mu, 0.0))
    s.rk4_step_adjoint(case.dev(prob.U), case.dev(prob.P), ref, dt)
    a, r = case.host(total), case.host(ref)
    for v in range(9):
        scale = np.abs(r[v]).max()
        assert np.abs(a[v] - r[v]).max() <= 1e-12 * scale, v


def test_autograd_functions_match_the_direct_calls():
    """The loss gradient through torch.autograd (InitialData, RK4Step) equals the direct adjoint calls."""
    need_gpu()
    from paper_2406_11669_gb300.autograd import InitialData, RK4Step
    w = W.smooth_general(n=(9, 8, 10), seed=109, **CASES["ppm_periodic_lorenz"])
    case = GpuCase(w)
    s = case.solver
    g, n = w.g, w.n
    inter = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    P0 = case.dev(O.prims_array(w))
    pot0 = s.zeros_state()
    pot0[5], pot0[6], pot0[7], pot0[8] = (case.dev(w.A["Ax"]), case.dev(w.A["Ay"]), case.dev(w.A["Az"]),
                                          case.dev(w.Psi))
    T = torch.ones_like(pot0[0])
    # autograd
    Pr = P0.clone().requires_grad_(True)
    pot = pot0.clone().requires_grad_(True)
    Pbuf = P0.clone()
    U = InitialData.apply(Pr, pot, s)
    for _ in range(2):
        U = RK4Step.apply(U, s, Pbuf, w.dt)
    loss = 0.5 * ((U[0][inter] - T[inter]) ** 2).sum()
    loss.backward()
    # direct calls
    U = pot0.clone()
    U[:5].zero_()
    s.fill_ghosts(U)
    Pd = P0.clone()
    s.prim2con(U, Pd)
    U0 = U.clone()
    ckpt = [s.zeros_state() for _ in range(2)]
    s.rk4_steps_checkpointed(U, Pd, w.dt, ckpt)
    lam = torch.zeros_like(U)
    lam[(0,) + inter] = U[(0,) + inter] - T[inter]
    s.rk4_adjoint_steps(ckpt, Pd, lam, w.dt)
    lamP = s.zeros_prims()
    s.prim2con_adjoint(U0, P0, lam, lamP)
    # per tensor scale: the Psi gradient is zero up to rounding (see the loss-gradient test)
    for a, r in ((Pr.grad, lamP), (pot.grad, lam)):
        a, r = case.host(a), case.host(r)
        scale = np.abs(r).max()
        for v in range(r.shape[0]):
            assert np.abs(a[v] - r[v]).max() <= 1e-12 * scale, v
