"""Degenerate cases of the method on the GPU against the oracle: no magnetic field (the quartic's slow roots
collapse onto the fluid speed), and a field along x whose Alfven speed equals the sound speed (the fast and
Alfven roots of the quartic coincide along x, a double root).  The states are uniform up to a 1e-3 velocity
ripple, so the hydro right-hand sides are small differences of O(1) fluxes: they are compared against the size
of the flux differences they are made of, |U| / dx, as well as their own size.
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase, owned, rel_field_err
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _uniform_with_ripple(bx, bc, n=(10, 9, 8), ripple=1e-3):
    """rho = 1, p = 1 (Gamma = 4/3), B = (bx, 0, 0) from A_z = bx y, a small velocity ripple; flat metric."""
    w = W.flat_modes(n=n)
    w.bc = (bc,) * 3
    X, Y, Z = W.positions(w.n, w.g, w.x0, w.dx, W.CELL)
    shape = w.shape
    w.prims = dict(rho=np.full(shape, 1.0), press=np.full(shape, 1.0),
                   velx=np.broadcast_to(ripple * np.sin(2 * math.pi * (X + 0.3 * Y)), shape).copy(),
                   vely=np.broadcast_to(ripple * np.cos(2 * math.pi * (Y - 0.2 * Z)), shape).copy(),
                   velz=np.broadcast_to(ripple * np.sin(2 * math.pi * (Z + 0.1 * X)), shape).copy())
    _, Yz, _ = W.positions(w.n, w.g, w.x0, w.dx, W.ZEDGE)
    w.A = dict(Ax=np.zeros(shape), Ay=np.zeros(shape), Az=np.broadcast_to(bx * Yz, shape).copy())
    return w


def _rhs_errors(w):
    case = GpuCase(w)
    U, P = O.initial_state(w)
    O.ghost_fill_state(w, U)
    O.con2prim(w, case.M, U, P)
    O.ghost_fill_prims(w, P)
    dU_o, _ = O.rhs(w, case.M, U, P)
    dU = case.solver.zeros_state()
    case.solver.rhs(case.dev(U), case.dev(P), dU, w.dt)
    dUg = case.host(dU)
    errs = []
    for v in range(9):
        e, scale = rel_field_err(dUg, dU_o, w, v)
        floor = np.abs(U[v][owned(w, v)]).max() / min(w.dx) if v < 5 else 0.0
        errs.append(e * scale / max(scale, floor, 1e-300))
    return errs


def test_no_magnetic_field():
    need_gpu()
    errs = _rhs_errors(_uniform_with_ripple(0.0, W.BC_COPY))
    assert max(errs) <= 1e-12, errs


def test_alfven_speed_equal_to_sound_speed_along_x():
    """c_A = c_s: with rho h = 5 and Gamma p / (rho h) = 4/15, b^2 = 20/11 gives c_A^2 = b^2 / (rho h + b^2) = 4/15."""
    need_gpu()
    errs = _rhs_errors(_uniform_with_ripple(math.sqrt(20.0 / 11.0), W.BC_COPY))
    print("relative field errors", errs)
    assert max(errs) <= 1e-12, errs
