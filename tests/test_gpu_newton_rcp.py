"""Error bound of the reciprocal the magnetosonic-speed Newton iteration (Sec. 3.3) uses for its corrections: a
hardware reciprocal estimate refined by one Newton-Raphson step, which squares the estimate's relative error.

A Newton correction stops the iteration once it falls below 3e-9 of the speed scale, so a relative error of the
correction far below 1e-6 leaves the converged root unchanged to rounding; the bound asserted here, 1e-11 over
the whole range the solver uses it in (1e-290 < |d| < 1e290, both signs, including powers of two and their
neighbours), is far inside that.  The reference values are numpy's correctly rounded 1/d.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_newton_reciprocal_relative_error():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    rng = np.random.default_rng(2406)
    mags = 10.0 ** rng.uniform(-289.5, 289.5, 1 << 20)
    d = mags * rng.choice([-1.0, 1.0], mags.size)
    p2 = 2.0 ** np.arange(-960, 961, 7, dtype=np.float64)
    special = np.concatenate([p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), -p2, 1.0 + 2.0 ** -np.arange(1, 53),
                              [1.0, -1.0, 3.0, 1.0 / 3.0, 0.1, 7.0e-289, 6.0e289]])
    d = np.concatenate([d, special])
    dd = torch.from_numpy(d).cuda()
    out = torch.empty_like(dd)
    A.newton_rcp(dd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = 1.0 / d
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"largest relative error {rel.max():.3e} over {d.size} values")
    assert np.all(np.isfinite(got))
    assert rel.max() <= 1e-11


def test_two_step_reciprocal_is_within_an_ulp_or_two():
    """The reciprocal used where a correctly rounded quotient is not needed (face solve, WENO-Z weights, Noble
    iteration): the estimate refined by two Newton-Raphson steps inside binary exponents +-960, 1/d outside.
    Against numpy's correctly rounded 1/d it must be within two units in the last place everywhere, and exact
    outside the refined range (the quotient itself)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    rng = np.random.default_rng(2407)
    mags = 10.0 ** rng.uniform(-300.0, 300.0, 1 << 20)
    d = mags * rng.choice([-1.0, 1.0], mags.size)
    p2 = 2.0 ** np.arange(-1000, 1001, 7, dtype=np.float64)
    special = np.concatenate([p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), -p2, 1.0 + 2.0 ** -np.arange(1, 53),
                              [1.0, -1.0, 3.0, 1.0 / 3.0, 0.1, 6.0, 7.0e-289, 6.0e289, 1e-305, 1e305]])
    d = np.concatenate([d, special])
    dd = torch.from_numpy(d).cuda()
    out = torch.empty_like(dd)
    A.recip(dd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = 1.0 / d
    ulps = np.abs(got - ref) / np.spacing(np.abs(ref))
    print(f"largest error {ulps.max():.2f} ulp over {d.size} values")
    assert np.all(np.isfinite(got))
    assert ulps.max() <= 2.0
    outside = np.abs(np.frexp(d)[1] - 1) >= 960
    assert np.array_equal(got[outside], ref[outside])


def test_corrected_quotient_is_the_correctly_rounded_quotient():
    """Division by sqrt(gamma) in the recovery and the centre field: the quotient formed from the correctly rounded
    1 / b and one fused correction must equal the correctly rounded a / b bit for bit (so those kernels divide
    exactly as the oracle does), on random pairs over many decades, on b near 1 (metric determinants) and on
    pairs whose quotients are near rounding ties."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11669_gb300 import asterx as A
    rng = np.random.default_rng(2408)
    n = 1 << 21
    a = 10.0 ** rng.uniform(-150.0, 150.0, n) * rng.choice([-1.0, 1.0], n)
    b = 10.0 ** rng.uniform(-100.0, 100.0, n) * rng.choice([-1.0, 1.0], n)
    b[: n // 4] = 1.0 + rng.uniform(-0.5, 2.0, n // 4)  # sqrt(gamma) of the workloads' metrics
    m = np.arange(1, 1 << 16, dtype=np.float64)
    a = np.concatenate([a, m * 2.0 ** -20, 1.0 + m * 2.0 ** -52])
    b = np.concatenate([b, np.full(m.size, 3.0), 1.0 + m[::-1] * 2.0 ** -40])
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty_like(ad)
    A.quotient(ad, bd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, a / b), int(np.sum(got != a / b))
