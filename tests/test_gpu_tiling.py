"""Same-level ghost exchange (asterx_batch_prepare_tiled): blocks that tile one domain evolve as one block covering
the domain would.

The definition of the exchange is that a block's ghost value equals the domain's value at that position, so the
reference is the single block over the whole domain (itself parity-tested against the oracle).  With a flat
metric every stencil sees identical inputs on both sides, so the owned values of every tiled block equal the
single block's bit for bit, with periodic and with copy boundaries, through prim->cons and two RK4 steps.  With
a curved metric the 4th-order interpolation of the metric to a block's outermost ghost cells shifts its stencil
inward (the vertex array ends there), so values near block boundaries differ at the interpolation's truncation
level; that case is checked to shrink steeply with resolution.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import CELL_LIKE, GpuCase
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CUTS = ([0, 7, 15, 24], [0, 9, 20], [0, 5, 16])  # 3 x 2 x 2 uneven blocks of a 24 x 20 x 16 domain


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def owned(w, v):
    g, n = w.g, w.n
    return tuple(slice(g, g + n[a] + (0 if (CELL_LIKE[v][a] or w.bc[a] == W.BC_PERIODIC) else 1)) for a in (2, 1, 0))


def domain(kind):
    n = tuple(c[-1] for c in CUTS)
    if kind == "periodic_flat":
        return W.flat_modes(n=n)
    if kind == "copy_curved":  # every field and the whole metric vary smoothly
        return W.smooth_general(n=n, recon=W.RECON_WENOZ, bc=W.BC_COPY)
    w = W.balsara_schwarzschild(n=n)
    w.metric = W.flat_metric(w.shape)
    return w


def tiled_run(w, U, P, steps):
    """The domain's state cut into the tiling's blocks, stepped by the batched launch with ghost exchange."""
    from paper_2406_11669_gb300 import asterx as A
    M = O.metric_array(w)
    entries, subs = [], []
    nblk = [len(c) - 1 for c in CUTS]
    for bz in range(nblk[2]):
        for by in range(nblk[1]):
            for bx in range(nblk[0]):
                lo = (CUTS[0][bx], CUTS[1][by], CUTS[2][bz])
                n = tuple(CUTS[d][b + 1] - CUTS[d][b] for d, b in enumerate((bx, by, bz)))
                ws = W.sub_block(w, lo, n)
                sl = (slice(None),) + tuple(slice(lo[d], lo[d] + n[d] + 2 * w.g + 1) for d in (2, 1, 0))
                dev = lambda a: torch.from_numpy(np.ascontiguousarray(a[sl])).cuda()
                entries.append((ws.n, ws.g, ws.x0, ws.dx, ws.bc, dev(M), dev(U), dev(P)))
                subs.append((lo, ws))
    batch = A.Batch(w.params, entries, tiling=(nblk, CUTS))
    batch.prepare()
    return batch, entries, subs


def compare(w, big, entries, subs, field_range, tol):
    worst = 0.0
    for (lo, ws), e in zip(subs, entries):
        got = e[6].cpu().numpy()
        for v in field_range:
            sl = owned(ws, v)
            gsl = tuple(slice(s.start + lo[d], s.stop + lo[d]) for s, d in zip(sl, (2, 1, 0)))
            a, r = got[v][sl], big[v][gsl]
            if tol == 0.0:
                assert np.array_equal(a, r), (lo, v, np.abs(a - r).max())
            else:
                scale = max(np.abs(big[v]).max(), 1e-300)
                worst = max(worst, np.abs(a - r).max() / scale)
    return worst


@pytest.mark.parametrize("kind", ["periodic_flat", "copy_flat"])
def test_tiled_domain_steps_like_one_block(kind):
    need_gpu()
    w = domain(kind)
    U = np.zeros((9,) + w.shape)
    U[5], U[6], U[7], U[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
    P = O.prims_array(w)
    # the single block over the whole domain
    case = GpuCase(w)
    Ub, Pb = case.dev(U), case.dev(P)
    case.solver.fill_ghosts(Ub)
    case.solver.prim2con(Ub, Pb)
    # the tiled domain from the same generator arrays (its ghosts come from the neighbours)
    batch, entries, subs = tiled_run(w, U, P, 2)
    batch.prim2con()
    torch.cuda.synchronize()
    compare(w, case.host(Ub), entries, subs, range(5), 0.0)
    for _ in range(2):
        case.solver.rk4_step(Ub, Pb, w.dt)
    batch.step(w.dt, nsteps=2)
    torch.cuda.synchronize()
    compare(w, case.host(Ub), entries, subs, range(9), 0.0)
    batch.release()


def curved_difference(scale):
    global CUTS
    saved = CUTS
    CUTS = tuple([c * scale for c in cuts] for cuts in saved)
    try:
        w = domain("copy_curved")
        U = np.zeros((9,) + w.shape)
        U[5], U[6], U[7], U[8] = w.A["Ax"], w.A["Ay"], w.A["Az"], w.Psi
        P = O.prims_array(w)
        case = GpuCase(w)
        Ub, Pb = case.dev(U), case.dev(P)
        case.solver.fill_ghosts(Ub)
        case.solver.prim2con(Ub, Pb)
        case.solver.rk4_step(Ub, Pb, w.dt)
        batch, entries, subs = tiled_run(w, U, P, 1)
        batch.prim2con()
        batch.step(w.dt)
        torch.cuda.synchronize()
        worst = compare(w, case.host(Ub), entries, subs, range(9), 1.0)
        batch.release()
        return worst
    finally:
        CUTS = saved


def test_tiled_curved_domain_converges_to_one_block():
    """A general smooth metric: the tiled blocks differ from the single block only through the metric interpolated
    to each block's outermost ghost layer (its stencil shifted inward where the vertex array ends), a 4th-order
    truncation difference that falls steeply when the same domain is resolved twice as finely."""
    need_gpu()
    d1 = curved_difference(1)
    d2 = curved_difference(2)
    print(f"largest difference relative to the field's magnitude: {d1:.2e} (24 cells), {d2:.2e} (48 cells)")
    assert d1 <= 1e-4 and d2 <= d1 / 6.0
