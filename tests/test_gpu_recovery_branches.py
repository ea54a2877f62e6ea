"""GPU parity of every branch of the primitive recovery (Sec. 3.5 Noble 2D, Sec. 3.5 Palenzuela 1D fallback,
Sec. 3.6 atmosphere), against the oracle, on 110,592 independent seeded states (one per cell of a 48^3 block:
rho in [1e-10, 1], p / rho in [1e-4, 10], W in [1, 10], b^2 / rho <= 100), 3% of them started from a poor guess.

Four settings drive the branches: the default recovery (Noble); one Noble iteration (c2p_maxiter = 1: Noble
cannot converge from a perturbed guess, so Palenzuela recovers the cells); and, on a state in which 2% of the
cells carry a negative tau~ (no physical solution for most: both solvers fail, flag -1, counted in n_failed; a
few are recovered by Palenzuela) and 1% a D~ below the atmosphere threshold (flag 2), the default recovery and
the recovery without fallback (Noble's failures go to the atmosphere with flag -1).  On these states no branch
decision changes when the inputs move by one ulp (checked with the oracle), so the two sides must take the same
branch in every cell.  Flags and branch counters must match the oracle's; the recovered
primitives agree to 1e-10 where both recovered the cell (the pressure relative to rho h, which the recovery
determines) and to rounding elsewhere (the atmosphere state);
conserved variables reset to the atmosphere agree to rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

from gpu_helpers import GpuCase, interior, stats_dict

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def states():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.recovery_states()
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    rng = np.random.default_rng(3)
    guess = P * (1.0 + 1e-3 * rng.standard_normal(P.shape))  # a previous-stage-like guess
    sel = W.Rng(1107).uniform(U[0].size).reshape(U[0].shape)
    Up = U.copy()
    neg = sel < 0.02
    Up[4][neg] = -np.abs(Up[4][neg])
    atm = (sel >= 0.02) & (sel < 0.03)
    Up[0][atm] = 1e-14
    bad = (sel >= 0.03) & (sel < 0.06)  # a poor guess: Noble needs many more iterations from it
    guess[0][bad] *= 1e4
    guess[1][bad] *= 1e-4
    return w, U, Up, guess


SETTINGS = {
    "default": (dict(), False),
    "one_noble_iteration": (dict(c2p_maxiter=1), False),
    "no_fallback": (dict(use_fallback=0), True),
    "both_fail_and_atmosphere": (dict(), True),
}


@pytest.mark.parametrize("setting", list(SETTINGS))
def test_recovery_branches_match_the_oracle(states, setting):
    w, U0, Upert, guess = states
    change, perturbed = SETTINGS[setting]
    params = dict(w.params, **change)
    Uin = Upert if perturbed else U0
    case = GpuCase(w, params=params)
    U = case.dev(Uin)
    P = case.dev(guess)
    fl = case.flags()
    st = case.stats()
    case.solver.con2prim(U, P, fl, st)
    Uo, Po = Uin.copy(), guess.copy()
    flags_o, st_o = O.con2prim(w, case.M, Uo, Po, params=params)
    sl = interior(w)
    fg, fo = case.host(fl)[sl], flags_o[sl]
    assert np.array_equal(fg, fo), (setting, int((fg != fo).sum()))
    sg = stats_dict(st)
    for k in ("n_noble", "n_fallback", "n_atm", "n_failed"):
        assert sg[k] == st_o[k], (setting, k, sg, st_o)
    assert abs(sg["iters"] - st_o["iters"]) <= 0.005 * max(st_o["iters"], 1) + 2, (sg, st_o)
    # which branches this setting reaches, on both sides
    if setting == "one_noble_iteration":
        assert st_o["n_fallback"] > 0.9 * fo.size and st_o["n_noble"] == 0
    if setting == "no_fallback":
        assert st_o["n_failed"] > 0 and st_o["n_fallback"] == 0
    if setting == "both_fail_and_atmosphere":
        assert st_o["n_fallback"] > 0 and st_o["n_failed"] > 0 and st_o["n_atm"] > 0
    # primitives where the cell was recovered (flags 0, 1); the atmosphere state elsewhere
    Pg = case.host(P)
    rec = (fo == 0) | (fo == 1)
    rel = np.abs(Pg[0][sl] - Po[0][sl]) / np.abs(Po[0][sl])
    assert rel[rec].max(initial=0.0) <= 1e-10, setting
    # the recovery fixes the enthalpy h = 1 + Gamma p / ((Gamma - 1) rho) and p follows from h - 1, so a cold
    # state (p / rho down to 1e-4) loses up to log10(h / (h - 1)) digits in p: p is compared against rho h
    rhoh = Po[0][sl] + Po[1][sl] * w.params["gamma"] / (w.params["gamma"] - 1.0)
    dp = np.abs(Pg[1][sl] - Po[1][sl]) / rhoh
    assert dp[rec].max(initial=0.0) <= 1e-10, setting
    for v in (2, 3, 4):
        assert np.abs(Pg[v][sl] - Po[v][sl])[rec].max(initial=0.0) <= 1e-10, (setting, v)
    for v in range(5):  # rho_atm, K rho_atm^Gamma_atm (the device's pow within an ulp), v = 0
        a, b = Pg[v][sl][~rec], Po[v][sl][~rec]
        assert np.all(np.abs(a - b) <= 4e-16 * np.abs(b)), (setting, v)
    # conserved variables: unchanged where recovered, reset to the atmosphere state (B kept) elsewhere
    Ug = case.host(U)
    for v in range(5):
        a, b = Ug[v][sl], Uo[v][sl]
        assert np.array_equal(a[rec], b[rec]), (setting, v)
        scale = np.abs(b[~rec]).max(initial=0.0)
        assert np.abs(a[~rec] - b[~rec]).max(initial=0.0) <= 1e-13 * max(scale, 1e-300), (setting, v)
