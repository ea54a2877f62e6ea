"""The C ABI library without a GPU: it loads, exports every function include/asterx.h declares, sizes
workspaces, and rejects invalid arguments on the host before any CUDA call (ASTERX_EINVAL / ASTERX_ENOMEM)."""
import ctypes
import os
import re

import pytest

from paper_2406_11669_gb300 import asterx as A
from paper_2406_11669_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "asterx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asterx_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    L = A.lib()
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(L, name), name


def test_abi_version_and_status_strings():
    L = A.lib()
    assert L.asterx_abi_version() == A.ABI_VERSION
    assert L.asterx_status_str(A.ASTERX_EINVAL) == b"invalid argument"


def test_workspace_size_and_invalid_blocks():
    good = A.block_struct((32, 32, 32), 3, (0, 0, 0), (1 / 32,) * 3, (0, 0, 0))
    assert A.workspace_size(good) > 39 ** 3 * 8 * 150
    for bad in (A.block_struct((0, 32, 32), 3, (0, 0, 0), (1 / 32,) * 3, (0, 0, 0)),
                A.block_struct((32, 32, 32), 2, (0, 0, 0), (1 / 32,) * 3, (0, 0, 0)),
                A.block_struct((32, 32, 32), 3, (0, 0, 0), (0.0, 1.0, 1.0), (0, 0, 0)),
                A.block_struct((32, 32, 32), 3, (0, 0, 0), (1 / 32,) * 3, (0, 2, 0))):
        assert A.workspace_size(bad) == 0


def _params(**kw):
    return A.params_struct(W.default_params(**kw))


@pytest.mark.parametrize("change", [dict(gamma=1.0), dict(rho_atm=0.0), dict(recon=7), dict(gauge=3),
                                    dict(c2p_maxiter=0), dict(W_max=1.0), dict(use_fallback=2), dict(flux=2),
                                    dict(efield=-1)])
def test_invalid_params_rejected_on_host(change):
    L = A.lib()
    p = _params(**change)
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    ws_bytes = A.workspace_size(b)
    rc = L.asterx_con2prim(ctypes.byref(p), ctypes.byref(b), ctypes.byref(st), ctypes.byref(pr), None, None,
                           ctypes.c_void_p(256), ws_bytes, None)
    assert rc == A.ASTERX_EINVAL


def test_small_workspace_and_bad_pointers_rejected():
    L = A.lib()
    p = _params()
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    need = A.workspace_size(b)
    rc = L.asterx_rk4_step(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.01), ctypes.byref(st),
                           ctypes.byref(pr), None, None, ctypes.c_void_p(256), need - 8, None)
    assert rc == A.ASTERX_ENOMEM
    bad = A.State(*([8] * 8 + [0]))  # a null field pointer
    rc = L.asterx_rk4_step(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.01), ctypes.byref(bad),
                           ctypes.byref(pr), None, None, ctypes.c_void_p(256), need, None)
    assert rc == A.ASTERX_EINVAL
    rc = L.asterx_rk_stage(ctypes.byref(p), ctypes.byref(b), 4, ctypes.c_double(0.01), ctypes.byref(st),
                           ctypes.byref(st), ctypes.byref(st), ctypes.byref(st), ctypes.byref(pr), None, None,
                           ctypes.c_void_p(256), need, None)
    assert rc == A.ASTERX_EINVAL  # stage out of range
    rc = L.asterx_rk4_step(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(-1.0), ctypes.byref(st),
                           ctypes.byref(pr), None, None, ctypes.c_void_p(256), need, None)
    assert rc == A.ASTERX_EINVAL  # dt <= 0
    rc = L.asterx_rk4_step(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.01), ctypes.byref(st),
                           ctypes.byref(pr), None, None, ctypes.c_void_p(100), need, None)
    assert rc == A.ASTERX_EINVAL  # workspace not 256-byte aligned


def test_host_buffer_step_rejects_bad_arguments_on_host():
    """asterx_rk4_step_host checks dt, the host pointers, the device fields and the stats alignment before it
    creates its second stream or copies anything."""
    L = A.lib()
    p = _params()
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    need = A.workspace_size(b)
    hu = (ctypes.c_void_p * 9)(*([16] * 9))
    hp = (ctypes.c_void_p * 5)(*([16] * 5))

    def call(dt=0.01, hu=hu, hp=hp, st=st, stats=None):
        return L.asterx_rk4_step_host(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(dt), hu, hp, ctypes.byref(st),
                                      ctypes.byref(pr), stats, ctypes.c_void_p(256), need, None)
    for dt in (0.0, -1.0, float("nan"), float("inf")):
        assert call(dt=dt) == A.ASTERX_EINVAL, dt
    assert call(hu=(ctypes.c_void_p * 9)(*([16] * 8 + [0]))) == A.ASTERX_EINVAL
    assert call(hp=(ctypes.c_void_p * 5)(*([0] + [16] * 4))) == A.ASTERX_EINVAL
    assert call(st=A.State(*([8] * 8 + [0]))) == A.ASTERX_EINVAL
    assert call(stats=ctypes.c_void_p(12)) == A.ASTERX_EINVAL  # not 8-byte aligned


def test_batch_workspace_size_and_validation():
    L = A.lib()
    arr = (A.BatchBlock * 2)()
    for i, n in enumerate(((8, 12, 16), (16, 8, 8))):
        arr[i].blk = A.block_struct(n, 3, (0, 0, 0), (0.1,) * 3, (1, 1, 1))
        arr[i].metric = A.Metric(*([8] * 16))
        arr[i].U = A.State(*([8] * 9))
        arr[i].P = A.Prims(*([8] * 5))
    size = L.asterx_batch_workspace_size(arr, 2)
    single = sum(A.workspace_size(arr[i].blk) for i in range(2))
    assert size > single
    arr[1].blk = A.block_struct((0, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (1, 1, 1))
    assert L.asterx_batch_workspace_size(arr, 2) == 0
    p = _params()
    rc = L.asterx_batched_step(ctypes.byref(p), arr, 2, ctypes.c_double(0.01), 1, None, ctypes.c_void_p(256),
                               size, None)
    assert rc == A.ASTERX_EINVAL


def test_adjoint_workspace_size_and_validation():
    L = A.lib()
    p = _params()
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    V = 15 ** 3
    size = L.asterx_adjoint_workspace_size(ctypes.byref(b))
    assert size >= 161 * V * 8 + V  # stage states, adjoint accumulators, flags
    bad_b = A.block_struct((8, 8, 8), 2, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    assert L.asterx_adjoint_workspace_size(ctypes.byref(bad_b)) == 0
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    need = A.workspace_size(b)
    args = (ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.01), ctypes.byref(st), ctypes.byref(pr))
    rc = L.asterx_rhs_adjoint(*args, ctypes.byref(st), ctypes.byref(st), ctypes.c_void_p(256), need,
                              ctypes.c_void_p(512), size - 8, None)
    assert rc == A.ASTERX_ENOMEM
    rc = L.asterx_rhs_adjoint(*args, ctypes.byref(st), ctypes.byref(st), ctypes.c_void_p(256), need, None, size,
                              None)
    assert rc == A.ASTERX_EINVAL  # no adjoint workspace
    rc = L.asterx_rk4_step_adjoint(*args, ctypes.byref(st), ctypes.c_void_p(256), need, ctypes.c_void_p(300),
                                   size, None)
    assert rc == A.ASTERX_EINVAL  # adjoint workspace not 256-byte aligned
    bad = A.State(*([8] * 8 + [0]))
    rc = L.asterx_rk4_step_adjoint(*args, ctypes.byref(bad), ctypes.c_void_p(256), need, ctypes.c_void_p(512),
                                   size, None)
    assert rc == A.ASTERX_EINVAL  # null adjoint field
    rc = L.asterx_rk4_step_adjoint(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.0), ctypes.byref(st),
                                   ctypes.byref(pr), ctypes.byref(st), ctypes.c_void_p(256), need,
                                   ctypes.c_void_p(512), size, None)
    assert rc == A.ASTERX_EINVAL  # dt <= 0


def test_tmunu_and_metric_step_validation():
    L = A.lib()
    p = _params()
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    need = A.workspace_size(b)
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    m = A.Metric(*([8] * 16))
    T = A.TmunuFields(*([8] * 10))
    ws = ctypes.c_void_p(256)
    rc = L.asterx_tmunu(ctypes.byref(p), ctypes.byref(b), ctypes.byref(m), ctypes.byref(st), ctypes.byref(pr),
                        ctypes.byref(A.TmunuFields(*([8] * 9 + [0]))), ws, need, None)
    assert rc == A.ASTERX_EINVAL  # null output field
    rc = L.asterx_tmunu(ctypes.byref(p), ctypes.byref(b), ctypes.byref(A.Metric(*([8] * 15 + [12]))),
                        ctypes.byref(st), ctypes.byref(pr), ctypes.byref(T), ws, need, None)
    assert rc == A.ASTERX_EINVAL  # misaligned metric field
    rc = L.asterx_tmunu(ctypes.byref(p), ctypes.byref(b), ctypes.byref(m), ctypes.byref(st), ctypes.byref(pr),
                        ctypes.byref(T), ws, need - 8, None)
    assert rc == A.ASTERX_ENOMEM
    ms = (ctypes.POINTER(A.Metric) * 4)(*[ctypes.pointer(m)] * 3 + [ctypes.POINTER(A.Metric)()])
    rc = L.asterx_rk4_step_metrics(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.01), ms, ctypes.byref(st),
                                   ctypes.byref(pr), None, None, ws, need, None)
    assert rc == A.ASTERX_EINVAL  # missing stage metric
    ms = (ctypes.POINTER(A.Metric) * 4)(*[ctypes.pointer(m)] * 4)
    rc = L.asterx_rk4_step_metrics(ctypes.byref(p), ctypes.byref(b), ctypes.c_double(0.0), ms, ctypes.byref(st),
                                   ctypes.byref(pr), None, None, ws, need, None)
    assert rc == A.ASTERX_EINVAL  # dt <= 0


def test_tiled_batch_validation():
    """asterx_batch_prepare_tiled rejects blocks that do not tile the domain as the cuts describe."""
    L = A.lib()
    p = _params()
    cuts = ([0, 8, 20], [0, 12], [0, 6])
    nblk = (2, 1, 1)

    def arr_for(ns, x0s, dxs=None):
        arr = (A.BatchBlock * len(ns))()
        for i, (n, x0) in enumerate(zip(ns, x0s)):
            arr[i].blk = A.block_struct(n, 3, x0, dxs[i] if dxs else (0.1,) * 3, (1, 1, 1))
            arr[i].metric = A.Metric(*([8] * 16))
            arr[i].U = A.State(*([8] * 9))
            arr[i].P = A.Prims(*([8] * 5))
        return arr

    def tiling(nb=nblk, cc=cuts):
        t = A.Tiling()
        keep = [(ctypes.c_int * len(c))(*c) for c in cc]
        for d in range(3):
            t.nblk[d] = nb[d]
            t.cuts[d] = ctypes.cast(keep[d], ctypes.POINTER(ctypes.c_int))
        return t, keep

    good = arr_for([(8, 12, 6), (12, 12, 6)], [(0.0, 0.0, 0.0), (0.8, 0.0, 0.0)])
    size = L.asterx_batch_workspace_size(good, 2)
    assert size > 0
    cases = [
        (arr_for([(8, 12, 6), (11, 12, 6)], [(0.0, 0.0, 0.0), (0.8, 0.0, 0.0)]), tiling()),  # n off the cuts
        (arr_for([(8, 12, 6), (12, 12, 6)], [(0.0, 0.0, 0.0), (0.9, 0.0, 0.0)]), tiling()),  # origin off
        (arr_for([(8, 12, 6), (12, 12, 6)], [(0.0, 0.0, 0.0), (0.8, 0.0, 0.0)],
                 [(0.1,) * 3, (0.1, 0.1, 0.2)]), tiling()),                                  # spacing differs
        (good, tiling(nb=(1, 1, 1), cc=([0, 20], [0, 12], [0, 6]))),                          # block count
        (arr_for([(2, 12, 6), (18, 12, 6)], [(0.0, 0.0, 0.0), (0.2, 0.0, 0.0)]),
         tiling(cc=([0, 2, 20], [0, 12], [0, 6]))),                                           # a block under 3 cells
    ]
    for arr, (t, keep) in cases:
        sz = max(L.asterx_batch_workspace_size(arr, 2), size)
        rc = L.asterx_batch_prepare_tiled(ctypes.byref(p), arr, 2, ctypes.byref(t), ctypes.c_void_p(256), sz, None)
        assert rc == A.ASTERX_EINVAL


def test_refinement_nesting_validation():
    """asterx_prolong checks the nesting on the host: half the spacing, even fine extents, a fine corner on a
    coarse vertex, the box inside the coarse interior."""
    L = A.lib()
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    c = A.block_struct((16, 16, 16), 3, (0.0, 0.0, 0.0), (0.1,) * 3, (1, 1, 1))
    bad = [
        A.block_struct((8, 8, 8), 3, (0.3, 0.3, 0.3), (0.06, 0.05, 0.05), (1, 1, 1)),  # not half the spacing
        A.block_struct((7, 8, 8), 3, (0.3, 0.3, 0.3), (0.05,) * 3, (1, 1, 1)),         # odd fine extent
        A.block_struct((8, 8, 8), 3, (0.35, 0.3, 0.3), (0.05,) * 3, (1, 1, 1)),        # corner between coarse vertices
        A.block_struct((8, 8, 8), 3, (1.3, 0.3, 0.3), (0.05,) * 3, (1, 1, 1)),         # beyond the coarse interior
        A.block_struct((8, 8, 8), 3, (-0.1, 0.3, 0.3), (0.05,) * 3, (1, 1, 1)),        # before it
    ]
    for f in bad:
        rc = L.asterx_prolong(ctypes.byref(c), ctypes.byref(f), ctypes.byref(st), ctypes.byref(pr),
                              ctypes.byref(st), ctypes.byref(pr), 0, None)
        assert rc == A.ASTERX_EINVAL


def test_subcycled_step_workspace_and_validation():
    """asterx_rk4_step_subcycled: its scratch holds 50 coarse padded fields (U_n, Y_1..Y_3, the interpolated
    state, its primitives); a short, missing or misaligned scratch, a bad nesting or dt <= 0 are refused on the
    host before any launch."""
    L = A.lib()
    p = _params()
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    c = A.block_struct((16, 16, 16), 3, (0.0, 0.0, 0.0), (0.1,) * 3, (1, 1, 1))
    f = A.block_struct((8, 8, 8), 3, (0.3, 0.3, 0.3), (0.05,) * 3, (1, 1, 1))
    need = L.asterx_subcycle_workspace_size(ctypes.byref(c))
    assert need == (50 * 23 ** 3 * 8 + 255) // 256 * 256
    bad_blk = A.block_struct((16, 16, 16), 3, (0, 0, 0), (0.0, 0.1, 0.1), (1, 1, 1))
    assert L.asterx_subcycle_workspace_size(ctypes.byref(bad_blk)) == 0
    wc, wf = A.workspace_size(c), A.workspace_size(f)

    def call(fine=f, dt=0.01, wt=256, wt_bytes=need):
        return L.asterx_rk4_step_subcycled(ctypes.byref(p), ctypes.byref(c), ctypes.byref(fine), ctypes.c_double(dt),
                                           ctypes.byref(st), ctypes.byref(pr), ctypes.byref(st), ctypes.byref(pr),
                                           None, ctypes.c_void_p(256), wc, ctypes.c_void_p(256), wf,
                                           ctypes.c_void_p(wt) if wt is not None else None, wt_bytes, None)

    assert call(wt_bytes=need - 8) == A.ASTERX_ENOMEM
    assert call(wt=None) == A.ASTERX_EINVAL
    assert call(wt=128) == A.ASTERX_EINVAL
    assert call(dt=0.0) == A.ASTERX_EINVAL
    assert call(fine=A.block_struct((8, 8, 8), 3, (0.35, 0.3, 0.3), (0.05,) * 3, (1, 1, 1))) == A.ASTERX_EINVAL


@pytest.mark.parametrize("n", [(1, 1, 2 ** 31 - 7), (2 ** 21 - 7,) * 3, (2 ** 20 + 1, 1, 1), (40, 40, 40),
                               (0, 8, 8), (-5, 8, 8)])
def test_noalloc_rejects_blocks_it_cannot_hold_on_host(n):
    """The allocation-free recovery rejects, before any CUDA call, blocks whose padded volume exceeds its fixed
    scratch array, including sizes whose padded volume overflows a 32- or 64-bit product."""
    L = A.lib()
    p = _params()
    b = A.block_struct(n, 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    m = A.Metric(*([8] * 16))
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    rc = L.asterx_con2prim_noalloc(ctypes.byref(p), ctypes.byref(b), ctypes.byref(m), ctypes.byref(st),
                                   ctypes.byref(pr), None, None, None)
    assert rc == A.ASTERX_EINVAL


@pytest.mark.parametrize("change", [dict(K_atm=float("inf")), dict(gamma_atm=float("inf")),
                                    dict(W_max=float("inf")), dict(recon=7), dict(gauge=3), dict(flux=2),
                                    dict(efield=-1), dict(xi_lorenz=-1.0)])
def test_noalloc_applies_the_workspace_entry_points_parameter_rules(change):
    L = A.lib()
    p = _params(**change)
    b = A.block_struct((8, 8, 8), 3, (0, 0, 0), (0.1,) * 3, (0, 0, 0))
    m = A.Metric(*([8] * 16))
    st = A.State(*([8] * 9))
    pr = A.Prims(*([8] * 5))
    rc = L.asterx_con2prim_noalloc(ctypes.byref(p), ctypes.byref(b), ctypes.byref(m), ctypes.byref(st),
                                   ctypes.byref(pr), None, None, None)
    assert rc == A.ASTERX_EINVAL
    b.x0[0] = float("nan")
    rc = L.asterx_con2prim_noalloc(ctypes.byref(_params()), ctypes.byref(b), ctypes.byref(m), ctypes.byref(st),
                                   ctypes.byref(pr), None, None, None)
    assert rc == A.ASTERX_EINVAL
