"""Pins of the oracle's two-level refinement (prolongation to a nested fine block of half the spacing, restriction
back; the prolongation the paper describes for its AMR magnetic-rotor test: third-order conservative along
cell-centred directions with a linear fallback, polynomial along vertex-centred ones).

Closed forms: cell averages of a product of quadratics prolong to the exact fine cell averages; vertex values of
a product of cubics prolong to the exact fine vertex values; an edge field (cell-centred along its direction,
vertex-centred across) mixes both exactly.  Conservation: the eight fine children of a coarse cell average to it
for any data, limited or not, so restricting a prolonged field returns the coarse field.  The fallback keeps a
prolonged value inside the range of its three coarse neighbours where the parabola would leave it.  The two-level
step keeps a uniform state uniform.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_11669_gb300 import workloads as W

L = (3, 4, 3)
M = (4, 3, 5)  # coarse cells under the fine box


def levels(n=(12, 12, 12)):
    wc = W.smooth_general(n=n, bc=W.BC_COPY)
    wfd = W.smooth_general(n=tuple(2 * v for v in n), bc=W.BC_COPY)
    wf = W.sub_block(wfd, tuple(2 * v for v in L), tuple(2 * v for v in M))
    return wc, wf


def coords(w, stagger):
    """Cell-centre (stagger 1) or vertex (stagger 0) coordinates per axis (x, y, z), lower cell faces too."""
    out = []
    for a in range(3):
        i = np.arange(w.N[a] + 1)
        lo = w.x0[a] + (i - w.g) * w.dx[a]
        out.append(lo)
    return out


def avg_quad(c, x0, h):
    """Cell average of c0 + c1 x + c2 x^2 over [x0, x0 + h]."""
    x1 = x0 + h
    return c[0] + c[1] * (x0 + x1) / 2 + c[2] * (x1 ** 3 - x0 ** 3) / (3 * h)


def cubic(c, x):
    return c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3


QUAD = [(1.0, 0.7, 0.2), (0.5, -0.8, 0.2), (2.0, 0.6, -0.2)]  # monotone over the padded box
CUB = [(0.3, 0.2, -0.4, 0.5), (1.0, -0.3, 0.2, 0.1), (-0.2, 0.5, 0.1, -0.3)]


def field(w, cl):
    """Cell-like axes: exact cell averages of the quadratics; vertex-like axes: the cubics at the vertices."""
    x = coords(w, 0)
    f = []
    for a in range(3):
        f.append(avg_quad(QUAD[a], x[a], w.dx[a]) if cl[a] else cubic(CUB[a], x[a]))
    return np.einsum("k,j,i->kji", f[2], f[1], f[0])


CELL_LIKE = [(1, 1, 1)] * 5 + [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 0)]


def fine_valid(wf, cl):
    """Points of the fine padded array where the field is defined (cell-like axes end at N - 1)."""
    return tuple(slice(0, wf.N[a] + (0 if cl[a] else 1)) for a in (2, 1, 0))


def test_polynomials_are_prolonged_exactly():
    wc, wf = levels()
    Uc = np.zeros((9,) + wc.shape)
    Pc = np.zeros((5,) + wc.shape)
    for v in range(9):
        Uc[v] = field(wc, CELL_LIKE[v])
    for v in range(5):
        Pc[v] = field(wc, (1, 1, 1))
    Uf = np.zeros((9,) + wf.shape)
    Pf = np.zeros((5,) + wf.shape)
    O.prolong(wc, wf, L, Uc, Pc, Uf, Pf, all_points=True)
    for v in range(9):
        ref = field(wf, CELL_LIKE[v])
        sl = fine_valid(wf, CELL_LIKE[v])
        assert np.abs(Uf[v][sl] - ref[sl]).max() <= 1e-13 * np.abs(ref[sl]).max(), v
    ref = field(wf, (1, 1, 1))
    sl = fine_valid(wf, (1, 1, 1))
    assert np.abs(Pf[0][sl] - ref[sl]).max() <= 1e-13 * np.abs(ref[sl]).max()


def test_prolongation_conserves_and_restriction_inverts_it():
    wc, wf = levels()
    rng = np.random.default_rng(7)
    Uc = rng.uniform(0.5, 1.5, (9,) + wc.shape)  # rough data: the fallback acts often
    Pc = rng.uniform(0.5, 1.5, (5,) + wc.shape)
    Uf = np.zeros((9,) + wf.shape)
    Pf = np.zeros((5,) + wf.shape)
    O.prolong(wc, wf, L, Uc, Pc, Uf, Pf, all_points=True)
    g = wf.g
    # the 8 children of every coarse cell under the fine interior average to it
    for v in range(5):
        kids = Uf[v][g:g + 2 * M[2], g:g + 2 * M[1], g:g + 2 * M[0]]
        avg = kids.reshape(M[2], 2, M[1], 2, M[0], 2).mean(axis=(1, 3, 5))
        par = Uc[v][wc.g + L[2]:wc.g + L[2] + M[2], wc.g + L[1]:wc.g + L[1] + M[1], wc.g + L[0]:wc.g + L[0] + M[0]]
        assert np.abs(avg - par).max() <= 1e-14, v
    back = np.array(Uc)
    back[:, wc.g + L[2]:wc.g + L[2] + M[2], wc.g + L[1]:wc.g + L[1] + M[1], wc.g + L[0]:wc.g + L[0] + M[0]] = 0.0
    O.restrict(wc, wf, L, back, Uf)
    for v in range(9):
        assert np.abs(back[v] - Uc[v]).max() <= 1e-14, v


def test_linear_fallback_keeps_prolonged_values_in_range():
    """Coarse averages (0, 1, 0.5) along x: the parabola would put 1.0625 in the right half of the middle cell; the
    fallback (minmod slope 0 there) keeps both halves at 1."""
    wc, wf = levels()
    Uc = np.ones((9,) + wc.shape)
    Pc = np.ones((5,) + wc.shape)
    line = np.ones(wc.shape[2])
    I = wc.g + L[0] + 1
    line[I - 1], line[I], line[I + 1] = 0.0, 1.0, 0.5
    Uc[0] = np.broadcast_to(line, wc.shape)
    Uf = np.zeros((9,) + wf.shape)
    Pf = np.zeros((5,) + wf.shape)
    O.prolong(wc, wf, L, Uc, Pc, Uf, Pf, all_points=True)
    g = wf.g
    kids = Uf[0][g + 3, g + 3, g + 2:g + 4]  # the two fine halves of coarse cell L + 1 along x
    assert np.array_equal(kids, [1.0, 1.0])
    sl = fine_valid(wf, (1, 1, 1))
    assert Uf[0][sl].min() >= 0.0 and Uf[0][sl].max() <= 1.0


def test_two_level_step_keeps_a_uniform_state():
    from test_oracle_grid import _uniform_workload
    wc = _uniform_workload(W.RECON_PPM, "flat")
    Lr = (2, 2, 1)
    wf = W.Workload("fine", (8, 6, 8), wc.g, tuple(wc.x0[d] + Lr[d] * wc.dx[d] for d in range(3)),
                    tuple(h / 2 for h in wc.dx), wc.bc, wc.params, wc.dt / 2, {}, {}, None, {})
    Uc, Pc = O.initial_state(wc)
    O.ghost_fill_state(wc, Uc)
    Mc = O.metric_array(wc)
    Uf = np.zeros((9,) + wf.shape)
    Pf = np.zeros((5,) + wf.shape)
    O.prolong(wc, wf, Lr, Uc, Pc, Uf, Pf, all_points=True)
    Mf = np.stack([np.full(wf.shape, Mc[q].flat[0]) for q in range(16)])
    Uc1, Uf1 = O.refined_rk4_step(wc, Mc, Uc.copy(), Pc.copy(), wf, Mf, Uf.copy(), Pf.copy(), Lr, wf.dt)
    g = wf.g
    for v in range(5):
        sl = (slice(g, g + wf.n[2]), slice(g, g + wf.n[1]), slice(g, g + wf.n[0]))
        assert np.abs(Uf1[v][sl] - Uf[v][sl]).max() <= 1e-13 * max(np.abs(Uf[v][sl]).max(), 1.0), v
        slc = (slice(wc.g, wc.g + wc.n[2]), slice(wc.g, wc.g + wc.n[1]), slice(wc.g, wc.g + wc.n[0]))
        assert np.abs(Uc1[v][slc] - Uc[v][slc]).max() <= 1e-13 * max(np.abs(Uc[v][slc]).max(), 1.0), v
