"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the oracle on the same
seeded inputs, compare field by field on the owned ranges."""
import numpy as np

import oracle as O
from paper_2406_11669_gb300 import workloads as W

# owned index ranges per state field: cell-like axes g..g+n-1, vertex-like axes g..g+n
CELL_LIKE = [(1, 1, 1)] * 5 + [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 0)]


def owned(w, v):
    g, n = w.g, w.n
    sl = []
    for a in (2, 1, 0):
        hi = g + n[a] - 1 if CELL_LIKE[v][a] else g + n[a]
        sl.append(slice(g, hi + 1))
    return tuple(sl)


def independent(w, v):
    """Like owned(), without the vertex index g+n along periodic axes (the periodic image of index g)."""
    g, n = w.g, w.n
    sl = []
    for a in (2, 1, 0):
        hi = g + n[a] - 1 if (CELL_LIKE[v][a] or w.bc[a] == W.BC_PERIODIC) else g + n[a]
        sl.append(slice(g, hi + 1))
    return tuple(sl)


def interior(w):
    g, n = w.g, w.n
    return (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))


GROUPS = [(0,), (1, 2, 3), (1, 2, 3), (1, 2, 3), (4,), (5, 6, 7), (5, 6, 7), (5, 6, 7), (8,)]


def field_scale(ref, w, v):
    """Magnitude a field's error is measured against: the maximum over its group (D~ | S~_i | tau~ | A_i | Psi)
    on the owned range; Psi, often identically zero, is floored at 1e-3 of the potential's magnitude."""
    scale = max(np.abs(ref[u][owned(w, u)]).max() for u in GROUPS[v])
    if v == 8:
        scale = max(scale, 1e-3 * max(np.abs(ref[u][owned(w, u)]).max() for u in (5, 6, 7)))
    return scale


def rel_field_err(a, ref, w, v, abs_allow=0.0):
    sl = owned(w, v)
    scale = max(field_scale(ref, w, v), 1e-300)
    err = np.maximum(np.abs(a[v][sl] - ref[v][sl]) - abs_allow, 0.0)
    return err.max() / scale, scale


class GpuCase:
    """A workload on the GPU: solver with its workspace prepared from the workload's metric."""

    def __init__(self, w, params=None):
        import torch
        from paper_2406_11669_gb300 import asterx as A
        self.torch = torch
        self.w = w
        self.params = dict(params or w.params)
        self.solver = A.Solver(self.params, w.n, w.g, w.x0, w.dx, w.bc)
        self.M = O.metric_array(w)
        self.Md = self.dev(self.M)
        self.solver.prepare(self.Md)

    def dev(self, x):
        return self.torch.from_numpy(np.ascontiguousarray(x)).cuda()

    @staticmethod
    def host(t):
        return t.detach().cpu().numpy()

    def stats(self):
        return self.torch.zeros(5, dtype=self.torch.int64, device="cuda")

    def flags(self):
        return self.torch.zeros(self.w.shape, dtype=self.torch.int8, device="cuda")


def stats_dict(t):
    v = t.cpu().numpy().astype(np.int64)
    return dict(n_noble=int(v[0]), n_fallback=int(v[1]), n_atm=int(v[2]), n_failed=int(v[3]), iters=int(v[4]))


def small_workloads():
    """Small blocks of every workload kind, with ragged extents (not multiples of 8, 16 or 32)."""
    c3 = W.star_block((16, 20, 12), (0.3515625, -0.0390625, -0.0234375), name="star_block_surface")
    return {
        "flat_modes": W.flat_modes(n=(20, 13, 9)),
        "balsara_schwarzschild": W.balsara_schwarzschild(n=(26, 10, 9)),
        "star": c3,
        "weak_field_modes": W.weak_field_modes(n=(12, 10, 11)),
        "torus_jet": W.torus_jet(n=(22, 21, 18)),
        "alfven1d": W.alfven_wave(16, recon=W.RECON_PPM),
    }


def assert_stats_match(gpu, ref):
    """Branch counts identical; total Noble iterations within 0.5% (a cell may converge one step apart)."""
    for k in ("n_noble", "n_fallback", "n_atm", "n_failed"):
        assert gpu[k] == ref[k], (k, gpu, ref)
    assert abs(gpu["iters"] - ref["iters"]) <= 0.005 * max(ref["iters"], 1) + 2, (gpu, ref)
