"""The gradient the benchmark times, checked on its own data: J = 1/2 sum_interior (D~_10 - T)^2 after ten RK4
steps of the 64^3 weak-field block (PPM, periodic, lapse 1 - 0.01 sin 2 pi x; seeded modes and target), with
respect to the initial primitives and potentials, against central differences of the forward steps at h = 1e-6
(other step sizes, or a one-sided quotient, where a limiter's switching surface lies within h of the state, or
where the forward map's own small jumps are not small against the quotient: the recovery stops its Newton
iteration at a tolerance of 1e-13, so its result jumps by about that much where the iteration count changes
between x - h and x + h, which puts jumps of order 1e-13 / h into the quotient, summed over the cells the probe
reaches in 40 stages; a larger h shrinks them).

64 seeded probes (16 on rho, 8 on each velocity component, 8 on each potential component) and 4 seeded random
directions over rho, v^i and A_i at once must agree to 1e-5 relative: each probe against the larger of its own
magnitude and 5% of its field's largest gradient entry (a probe whose gradient is tiny is judged on the field's
scale, which keeps limiter switching in the reach of the difference quotient from deciding it), and at least
95% of the probes also against their own magnitude alone.  The pressure is left out: it is uniform
in this workload (p = 1), so PPM's limiter sits exactly on its switching surface in p, where the derivative is
one-sided and no difference quotient is linear in h.  The forward steps run through the same library entry points
the gradient's forward pass uses (each verified against the oracle elsewhere); the loss difference is formed as
1/2 sum (D+ - D-)(D+ + D- - 2T), which avoids the cancellation of two nearly equal sums of squares."""
import numpy as np
import pytest

from gpu_helpers import independent
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS = 10
HS = (1e-6, 1e-5, 1e-4, 1e-3, 1e-7)
RTOL = 1e-5


def test_ten_step_gradient_matches_central_differences():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    w = W.weak_field_modes()
    dev = torch.device("cuda")
    M = torch.from_numpy(np.ascontiguousarray(np.stack([w.metric[k] for k in W.METRIC_NAMES]))).to(dev)
    P0 = torch.from_numpy(np.ascontiguousarray(np.stack([w.prims[k] for k in W.PRIM_NAMES]))).to(dev)
    base = torch.zeros((9,) + w.shape, dtype=torch.float64, device=dev)
    for v, name in ((5, "Ax"), (6, "Ay"), (7, "Az")):
        base[v] = torch.from_numpy(w.A[name]).to(dev)
    base[8] = torch.from_numpy(w.Psi).to(dev)
    T = torch.from_numpy(W.weak_field_target(w)).to(dev)
    g, n = w.g, w.n
    inter = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    s = A.Solver.for_workload(w, device=dev)
    s.prepare(M)

    def final_density(P, pot):
        U = pot.clone()
        s.fill_ghosts(U)
        Pw = P.clone()
        s.prim2con(U, Pw)
        for _ in range(NSTEPS):
            s.rk4_step(U, Pw, w.dt)
        return U[0][inter].clone()

    # the gradient, as the benchmark forms it
    U = base.clone()
    s.fill_ghosts(U)
    P = P0.clone()
    s.prim2con(U, P)
    U0 = U.clone()
    ckpt = [torch.empty_like(U) for _ in range(NSTEPS)]
    s.rk4_steps_checkpointed(U, P, w.dt, ckpt)
    lam = torch.zeros_like(U)
    lam[(0,) + inter] = U[(0,) + inter] - T[inter]
    s.rk4_adjoint_steps(ckpt, P, lam, w.dt)
    lamP = torch.zeros_like(P0)
    s.prim2con_adjoint(U0, P0, lam, lamP)
    torch.cuda.synchronize()
    gP, gU = lamP.cpu().numpy(), lam.cpu().numpy()
    # forward without checkpoints reproduces the checkpointed forward
    D_ref = final_density(P0, base)
    assert torch.equal(D_ref, U[0][inter])

    def dJ(dP, dpot):
        """(J(x + d) - J(x), J(x) - J(x - d)) for the direction d = (dP, dpot) (device arrays), each formed as
        1/2 sum (D1 - D0)(D1 + D0 - 2T)."""
        Dp = final_density(P0 + dP, base + dpot)
        Dm = final_density(P0 - dP, base - dpot)
        up = float(torch.sum(0.5 * (Dp - D_ref) * (Dp + D_ref - 2.0 * T[inter])))
        down = float(torch.sum(0.5 * (D_ref - Dm) * (D_ref + Dm - 2.0 * T[inter])))
        return up, down

    def closest(ad, quotient, floor):
        """(error against max(|fd|, floor), error against |fd| alone, h): the smallest relative differences of ad
        from the difference quotients over HS, stopping at the first step size that agrees.  PPM's limiters make
        the map piecewise smooth: where a switching surface lies within h of the state, the central quotient
        mixes two branches, and the adjoint (the derivative of the branch the state is on) equals one of the
        one-sided quotients instead; where the gradient entry is small, a larger h keeps the quotient's rounding
        below it.  An adjoint error shows in all three quotients at every h."""
        best, own = None, None
        for h in HS:
            up, down = quotient(h)
            for fd in (0.5 * (up + down), up, down):
                e = abs(ad - fd)
                b, o = e / max(abs(fd), floor), e / max(abs(fd), 1e-300)
                best = b if best is None else min(best, b)
                own = o if own is None else min(own, o)
            if own <= RTOL:
                break
        return best, own, h

    rng = W.Rng(4104)
    pick = lambda lo, hi: int(lo + min(int(rng.uniform(1)[0] * (hi - lo)), hi - lo - 1))
    probes = [(0, 16)] + [(v, 8) for v in (2, 3, 4)] + [(v, 8) for v in (5, 6, 7)]
    worst = 0.0
    smaller = 0
    tight = 0  # probes within RTOL of their own magnitude
    for v, count in probes:
        sl = inter if v < 5 else independent(w, v)
        arr, grad = (P0, gP[v]) if v < 5 else (base, gU[v])
        scale = max(float(arr[v][sl].abs().max()), 0.05 if v < 5 else 1e-3)
        gmax = np.abs(grad[sl]).max()
        for _ in range(count):
            idx = tuple(pick(x.start, x.stop) for x in sl)

            def quotient(h):
                d = torch.zeros_like(arr)
                d[(v,) + idx] = h * scale
                up, down = dJ(d, torch.zeros_like(base)) if v < 5 else dJ(torch.zeros_like(P0), d)
                return up / (h * scale), down / (h * scale)

            err, own, h = closest(grad[idx], quotient, 0.05 * gmax)
            worst = max(worst, err)
            smaller += h != HS[0]
            tight += own <= RTOL
            assert err <= RTOL, (v, idx, grad[idx], err)
    # random directions over rho, v^i and A_i together
    for q in range(4):
        dP = torch.zeros_like(P0)
        dA = torch.zeros_like(base)
        ad = 0.0
        for v in (0, 2, 3, 4, 5, 6, 7):
            sl = inter if v < 5 else independent(w, v)
            arr = P0 if v < 5 else base
            scale = max(float(arr[v][sl].abs().max()), 0.05 if v < 5 else 1e-3)
            shape = arr[v][sl].shape
            r = rng.uniform(int(np.prod(shape)), -1.0, 1.0).reshape(shape) * scale
            tgt = dP if v < 5 else dA
            tgt[v][sl] = torch.from_numpy(r).to(dev)
            ad += float(np.sum((gP[v] if v < 5 else gU[v])[sl] * r))
        err, _, h = closest(ad, lambda h: tuple(x / h for x in dJ(h * dP, h * dA)), 0.0)
        worst = max(worst, err)
        smaller += h != HS[0]
        assert err <= RTOL, (q, ad, err)
    assert tight >= 0.95 * 64, tight
    print(f"worst relative difference {worst:.2e} over 64 probes and 4 directions; {smaller} needed another h; "
          f"{tight} of 64 probes within {RTOL} of their own magnitude")
