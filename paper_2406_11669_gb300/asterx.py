"""Python binding of the C ABI in include/asterx.h (argument marshalling only).

Every step of the GRMHD stage runs in the CUDA library libasterx.so; this module only turns torch CUDA tensors
into the pointer structs of the ABI and forwards the current CUDA stream.  There is no fallback: if the library
is missing and cannot be built, importing raises.

Tensors: the state is a float64 CUDA tensor of shape (9, Nz+1, Ny+1, Nx+1) (D~, S~x, S~y, S~z, tau~, A_x, A_y,
A_z, Psi), the primitives (5, ...) (rho, p, v^x, v^y, v^z), the metric (16, ...) (alpha, beta^i, gamma_ij, K_ij);
all contiguous.  Function names follow the ABI.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

ASTERX_OK, ASTERX_EINVAL, ASTERX_ECUDA, ASTERX_ENOMEM, ASTERX_EC2P, ASTERX_ETIMEOUT = range(6)
ABI_VERSION = 2


class AsterxError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({_status_str(status)})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("rho_atm", ctypes.c_double), ("K_atm", ctypes.c_double),
                ("gamma_atm", ctypes.c_double), ("c2p_tol", ctypes.c_double), ("c2p_maxiter", ctypes.c_int),
                ("brent_maxiter", ctypes.c_int), ("W_max", ctypes.c_double), ("recon", ctypes.c_int),
                ("gauge", ctypes.c_int), ("xi_lorenz", ctypes.c_double), ("use_fallback", ctypes.c_int),
                ("flux", ctypes.c_int), ("efield", ctypes.c_int)]


class Block(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("g", ctypes.c_int), ("x0", ctypes.c_double * 3),
                ("dx", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


class State(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("D", "Sx", "Sy", "Sz", "tau", "Ax", "Ay", "Az", "Psi")]


class Prims(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("rho", "press", "velx", "vely", "velz")]


class Metric(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("alp", "betax", "betay", "betaz", "gxx", "gxy", "gxz", "gyy",
                                                "gyz", "gzz", "kxx", "kxy", "kxz", "kyy", "kyz", "kzz")]


class TmunuFields(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("tt", "tx", "ty", "tz", "xx", "xy", "xz", "yy", "yz", "zz")]


class BatchBlock(ctypes.Structure):
    _fields_ = [("blk", Block), ("metric", Metric), ("U", State), ("P", Prims)]


class Tiling(ctypes.Structure):
    _fields_ = [("nblk", ctypes.c_int * 3), ("cuts", ctypes.POINTER(ctypes.c_int) * 3)]


class C2PStats(ctypes.Structure):
    _fields_ = [("n_noble", ctypes.c_ulonglong), ("n_fallback", ctypes.c_ulonglong),
                ("n_atm", ctypes.c_ulonglong), ("n_failed", ctypes.c_ulonglong), ("iters", ctypes.c_ulonglong)]


_lib = None


def lib():
    """The loaded libasterx.so (built in-tree on first use if absent)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, sz, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
        P, B = ctypes.POINTER(Params), ctypes.POINTER(Block)
        S, Pr, M = ctypes.POINTER(State), ctypes.POINTER(Prims), ctypes.POINTER(Metric)
        L.asterx_abi_version.restype = ctypes.c_int
        L.asterx_status_str.restype = ctypes.c_char_p
        L.asterx_status_str.argtypes = [ctypes.c_int]
        L.asterx_workspace_size.restype = ctypes.c_size_t
        L.asterx_workspace_size.argtypes = [B]
        L.asterx_prepare.argtypes = [P, B, M, vp, sz, st]
        L.asterx_prim2con.argtypes = [P, B, S, Pr, vp, sz, st]
        L.asterx_con2prim.argtypes = [P, B, S, Pr, vp, vp, vp, sz, st]
        L.asterx_fill_ghosts.argtypes = [P, B, S, vp, sz, st]
        L.asterx_rhs.argtypes = [P, B, S, Pr, S, ctypes.c_double, vp, sz, st]
        L.asterx_rk_stage.argtypes = [P, B, ctypes.c_int, ctypes.c_double, S, S, S, S, Pr, vp, vp, vp, sz, st]
        L.asterx_rk4_step.argtypes = [P, B, ctypes.c_double, S, Pr, vp, vp, vp, sz, st]
        L.asterx_rk2_step.argtypes = [P, B, ctypes.c_double, S, Pr, vp, vp, vp, sz, st]
        L.asterx_rk4_step_host.argtypes = [P, B, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), S, Pr, vp, vp, sz, st]
        L.asterx_tmunu.argtypes = [P, B, M, S, Pr, ctypes.POINTER(TmunuFields), vp, sz, st]
        L.asterx_rk4_step_metrics.argtypes = [P, B, ctypes.c_double, ctypes.POINTER(M), S, Pr, vp, vp, vp, sz, st]
        L.asterx_prolong.argtypes = [B, B, S, Pr, S, Pr, ctypes.c_int, st]
        L.asterx_rk4_step_refined.argtypes = [P, B, B, ctypes.c_double, S, Pr, S, Pr, vp, vp, sz, vp, sz, st]
        L.asterx_subcycle_workspace_size.restype = ctypes.c_size_t
        L.asterx_subcycle_workspace_size.argtypes = [B]
        L.asterx_rk4_step_subcycled.argtypes = [P, B, B, ctypes.c_double, S, Pr, S, Pr, vp, vp, sz, vp, sz, vp, sz,
                                                st]
        BB = ctypes.POINTER(BatchBlock)
        L.asterx_batch_workspace_size.restype = ctypes.c_size_t
        L.asterx_batch_workspace_size.argtypes = [BB, ctypes.c_int]
        L.asterx_batch_prepare.argtypes = [P, BB, ctypes.c_int, vp, sz, st]
        L.asterx_batch_prim2con.argtypes = [P, BB, ctypes.c_int, vp, sz, st]
        L.asterx_batched_step.argtypes = [P, BB, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp, sz, st]
        L.asterx_batch_release.argtypes = [vp]
        L.asterx_batch_prepare_tiled.argtypes = [P, BB, ctypes.c_int, ctypes.POINTER(Tiling), vp, sz, st]
        for name in ("asterx_batch_prepare", "asterx_batch_prim2con", "asterx_batched_step", "asterx_batch_release",
                     "asterx_batch_prepare_tiled"):
            getattr(L, name).restype = ctypes.c_int
        L.asterx_adjoint_workspace_size.restype = ctypes.c_size_t
        L.asterx_adjoint_workspace_size.argtypes = [B]
        L.asterx_rhs_adjoint.argtypes = [P, B, ctypes.c_double, S, Pr, S, S, vp, sz, vp, sz, st]
        L.asterx_rk4_step_adjoint.argtypes = [P, B, ctypes.c_double, S, Pr, S, vp, sz, vp, sz, st]
        L.asterx_prim2con_adjoint.argtypes = [P, B, S, Pr, S, Pr, vp, sz, vp, sz, st]
        L.asterx_rk_stage_adjoint.argtypes = [P, B, ctypes.c_int, ctypes.c_double, S, Pr, S, S, S, vp, sz, vp, sz,
                                              st]
        L.asterx_rk4_steps_checkpointed.argtypes = [P, B, ctypes.c_double, ctypes.c_int, S, Pr, S, vp, vp, sz, st]
        L.asterx_rk4_adjoint_steps.argtypes = [P, B, ctypes.c_double, ctypes.c_int, S, Pr, S, vp, sz, vp, sz, st]
        for name in ("asterx_rhs_adjoint", "asterx_rk4_step_adjoint", "asterx_prim2con_adjoint", "asterx_rk_stage_adjoint",
                     "asterx_rk4_steps_checkpointed", "asterx_rk4_adjoint_steps"):
            getattr(L, name).restype = ctypes.c_int
        L.asterx_con2prim_noalloc.argtypes = [P, B, M, S, Pr, vp, vp, st]
        L.asterx_con2prim_noalloc.restype = ctypes.c_int
        L.asterx_profile_enable.argtypes = [ctypes.c_int]
        L.asterx_profile_read.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.asterx_profile_disable.restype = None
        L.asterx_dfma_probe.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_long, st]
        L.asterx_newton_rcp.argtypes = [vp, vp, ctypes.c_long, st]
        L.asterx_recip.argtypes = [vp, vp, ctypes.c_long, st]
        L.asterx_quotient.argtypes = [vp, vp, vp, ctypes.c_long, st]
        for name in ("asterx_prepare", "asterx_prim2con", "asterx_con2prim", "asterx_fill_ghosts", "asterx_rhs",
                     "asterx_rk_stage", "asterx_rk4_step", "asterx_rk2_step", "asterx_rk4_step_host", "asterx_tmunu",
                     "asterx_rk4_step_metrics", "asterx_prolong", "asterx_rk4_step_refined", "asterx_rk4_step_subcycled",
                     "asterx_profile_enable",
                     "asterx_profile_read", "asterx_dfma_probe", "asterx_newton_rcp", "asterx_recip",
                     "asterx_quotient"):
            getattr(L, name).restype = ctypes.c_int
        if L.asterx_abi_version() != ABI_VERSION:
            raise ImportError(f"libasterx ABI {L.asterx_abi_version()} != binding ABI {ABI_VERSION}")
        _lib = L
    return _lib


def _status_str(s: int) -> str:
    try:
        return lib().asterx_status_str(int(s)).decode()
    except Exception:  # pragma: no cover - only used for messages
        return "?"


def _check(status: int, what: str):
    if status != ASTERX_OK:
        raise AsterxError(status, what)


# -------------------------------------------------------------------------------------------------- structs


def params_struct(p: dict) -> Params:
    return Params(p["gamma"], p["rho_atm"], p["K_atm"], p["gamma_atm"], p["c2p_tol"], int(p["c2p_maxiter"]),
                  int(p["brent_maxiter"]), p["W_max"], int(p["recon"]), int(p["gauge"]), p["xi_lorenz"],
                  int(p["use_fallback"]), int(p.get("flux", 0)), int(p.get("efield", 0)))


def block_struct(n, g, x0, dx, bc) -> Block:
    b = Block()
    for d in range(3):
        b.n[d] = int(n[d])
        b.x0[d] = float(x0[d])
        b.dx[d] = float(dx[d])
        b.bc[d] = int(bc[d])
    b.g = int(g)
    return b


def _field_ptrs(t, count):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need a contiguous float64 CUDA tensor"
    assert t.shape[0] == count
    V = t[0].numel()
    base = t.data_ptr()
    return [base + 8 * V * v for v in range(count)]


def state_struct(U) -> State:
    return State(*_field_ptrs(U, 9))


def prims_struct(P) -> Prims:
    return Prims(*_field_ptrs(P, 5))


def metric_struct(M) -> Metric:
    return Metric(*_field_ptrs(M, 16))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_size(block: Block) -> int:
    return int(lib().asterx_workspace_size(ctypes.byref(block)))


class Solver:
    """One block plus its workspace.  The workspace is a caller-owned torch allocation (256-byte aligned);
    prepare() derives the frozen-metric geometry into it."""

    def __init__(self, params: dict, n, g, x0, dx, bc, device="cuda"):
        import torch
        self.params = dict(params)
        self.p = params_struct(self.params)
        self.b = block_struct(n, g, x0, dx, bc)
        self.n = tuple(int(v) for v in n)
        self.g = int(g)
        N = [self.n[d] + 2 * self.g for d in range(3)]
        self.shape = (N[2] + 1, N[1] + 1, N[0] + 1)
        self.ws_bytes = workspace_size(self.b)
        if self.ws_bytes == 0:
            raise AsterxError(ASTERX_EINVAL, "invalid block")
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = ctypes.c_void_p(self.ws.data_ptr() + off)
        self.stats = torch.zeros(5, dtype=torch.int64, device=device)

    @classmethod
    def for_workload(cls, w, device="cuda"):
        return cls(w.params, w.n, w.g, w.x0, w.dx, w.bc, device)

    def zeros_state(self):
        import torch
        return torch.zeros((9,) + self.shape, dtype=torch.float64, device=self.ws.device)

    def zeros_prims(self):
        import torch
        return torch.zeros((5,) + self.shape, dtype=torch.float64, device=self.ws.device)

    def _args(self):
        return ctypes.byref(self.p), ctypes.byref(self.b)

    def prepare(self, metric, stream=None):
        self._metric = metric  # keep the vertex metric alive while the workspace refers to it
        m = metric_struct(metric)
        _check(lib().asterx_prepare(*self._args(), ctypes.byref(m), self.ws_ptr, self.ws_bytes, _stream(stream)),
               "asterx_prepare")

    def prim2con(self, U, P, stream=None):
        u, p = state_struct(U), prims_struct(P)
        _check(lib().asterx_prim2con(*self._args(), ctypes.byref(u), ctypes.byref(p), self.ws_ptr, self.ws_bytes,
                                     _stream(stream)), "asterx_prim2con")

    def fill_ghosts(self, U, stream=None):
        u = state_struct(U)
        _check(lib().asterx_fill_ghosts(*self._args(), ctypes.byref(u), self.ws_ptr, self.ws_bytes,
                                        _stream(stream)), "asterx_fill_ghosts")

    def con2prim(self, U, P, flags=None, stats=None, stream=None):
        u, p = state_struct(U), prims_struct(P)
        fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_con2prim(*self._args(), ctypes.byref(u), ctypes.byref(p), fl, sp, self.ws_ptr,
                                     self.ws_bytes, _stream(stream)), "asterx_con2prim")

    def rhs(self, U, P, dU, dt, stream=None):
        u, p, d = state_struct(U), prims_struct(P), state_struct(dU)
        _check(lib().asterx_rhs(*self._args(), ctypes.byref(u), ctypes.byref(p), ctypes.byref(d), float(dt),
                                self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_rhs")

    def rk_stage(self, stage, dt, Un, Us, Unext, Uacc, P, flags=None, stats=None, stream=None):
        a = [state_struct(x) for x in (Un, Us, Unext, Uacc)]
        p = prims_struct(P)
        fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk_stage(*self._args(), int(stage), float(dt), *[ctypes.byref(x) for x in a],
                                     ctypes.byref(p), fl, sp, self.ws_ptr, self.ws_bytes, _stream(stream)),
               "asterx_rk_stage")

    def rk4_step(self, U, P, dt, flags=None, stats=None, stream=None):
        u, p = state_struct(U), prims_struct(P)
        fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk4_step(*self._args(), float(dt), ctypes.byref(u), ctypes.byref(p), fl, sp,
                                     self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_rk4_step")

    def rk2_step(self, U, P, dt, flags=None, stats=None, stream=None):
        u, p = state_struct(U), prims_struct(P)
        fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk2_step(*self._args(), float(dt), ctypes.byref(u), ctypes.byref(p), fl, sp,
                                     self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_rk2_step")

    def rk4_step_host(self, hU, hP, dU, dP, dt, stats=None, stream=None):
        """hU (9, ...) and hP (5, ...) are pinned host tensors; dU, dP device tensors of the same shapes."""
        hu = (ctypes.c_void_p * 9)(*[hU[v].data_ptr() for v in range(9)])
        hp = (ctypes.c_void_p * 5)(*[hP[v].data_ptr() for v in range(5)])
        u, p = state_struct(dU), prims_struct(dP)
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk4_step_host(*self._args(), float(dt), hu, hp, ctypes.byref(u), ctypes.byref(p), sp,
                                          self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_rk4_step_host")

    def tmunu(self, U, P, T, stream=None):
        """T (10, ...): T_{mu nu} (tt, tx, ty, tz, xx, xy, xz, yy, yz, zz) at the owned vertices from U's A and P
        (ghosts filled) with the metric this solver was prepared from."""
        m, u, p = metric_struct(self._metric), state_struct(U), prims_struct(P)
        t = TmunuFields(*_field_ptrs(T, 10))
        _check(lib().asterx_tmunu(*self._args(), ctypes.byref(m), ctypes.byref(u), ctypes.byref(p), ctypes.byref(t),
                                  self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_tmunu")

    def rk4_step_metrics(self, U, P, dt, metrics, flags=None, stats=None, stream=None):
        """One RK4 step whose stage s runs on metrics[s] (four (16, ...) tensors); the solver ends prepared from
        metrics[3]."""
        assert len(metrics) == 4
        ms = [metric_struct(M) for M in metrics]
        arr = (ctypes.POINTER(Metric) * 4)(*[ctypes.pointer(m) for m in ms])
        u, p = state_struct(U), prims_struct(P)
        fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk4_step_metrics(*self._args(), float(dt), arr, ctypes.byref(u), ctypes.byref(p), fl, sp,
                                             self.ws_ptr, self.ws_bytes, _stream(stream)),
               "asterx_rk4_step_metrics")
        self._metric = metrics[3]

    def _adjoint_ws(self):
        import torch
        if getattr(self, "aws", None) is None:
            self.aws_bytes = int(lib().asterx_adjoint_workspace_size(ctypes.byref(self.b)))
            self.aws = torch.empty(self.aws_bytes + 256, dtype=torch.uint8, device=self.ws.device)
            off = (-self.aws.data_ptr()) % 256
            self.aws_ptr = ctypes.c_void_p(self.aws.data_ptr() + off)
        return self.aws_ptr, self.aws_bytes

    def rhs_adjoint(self, U, P, mu, lam, dt, stream=None):
        """lam = (dL/dU)^T mu for the stage right-hand side L at U (adjoint workspace allocated on first use)."""
        ap, ab = self._adjoint_ws()
        u, p, m, l = state_struct(U), prims_struct(P), state_struct(mu), state_struct(lam)
        _check(lib().asterx_rhs_adjoint(*self._args(), float(dt), ctypes.byref(u), ctypes.byref(p), ctypes.byref(m),
                                        ctypes.byref(l), self.ws_ptr, self.ws_bytes, ap, ab, _stream(stream)),
               "asterx_rhs_adjoint")

    def rk_stage_adjoint(self, stage, dt, Us, P, lam_next, lam_acc, lam_s, stream=None):
        """lam_s = (dL/dUs)^T (c dt lam_next + b dt lam_acc) for stage 0..2, (dL/dUs)^T (dt/6 lam_next) for stage 3."""
        ap, ab = self._adjoint_ws()
        la = ctypes.byref(state_struct(lam_acc)) if lam_acc is not None else None
        _check(lib().asterx_rk_stage_adjoint(*self._args(), int(stage), float(dt), ctypes.byref(state_struct(Us)),
                                             ctypes.byref(prims_struct(P)), ctypes.byref(state_struct(lam_next)),
                                             la, ctypes.byref(state_struct(lam_s)), self.ws_ptr, self.ws_bytes, ap,
                                             ab, _stream(stream)), "asterx_rk_stage_adjoint")

    def rk4_step_adjoint(self, Un, P, lam, dt, stream=None):
        """In place: lam = dJ/dU_{n+1} on entry, dJ/dU_n on exit, for the RK4 step taken from state Un."""
        ap, ab = self._adjoint_ws()
        u, p, l = state_struct(Un), prims_struct(P), state_struct(lam)
        _check(lib().asterx_rk4_step_adjoint(*self._args(), float(dt), ctypes.byref(u), ctypes.byref(p),
                                             ctypes.byref(l), self.ws_ptr, self.ws_bytes, ap, ab, _stream(stream)),
               "asterx_rk4_step_adjoint")

    def prim2con_adjoint(self, U, P, lam, lamP, stream=None):
        """In place: lam = dJ/dU0 on entry; on exit fields A, Psi of lam hold dJ/dA, dJ/dPsi and lamP = dJ/dP."""
        ap, ab = self._adjoint_ws()
        u, p, l, lp = state_struct(U), prims_struct(P), state_struct(lam), prims_struct(lamP)
        _check(lib().asterx_prim2con_adjoint(*self._args(), ctypes.byref(u), ctypes.byref(p), ctypes.byref(l),
                                             ctypes.byref(lp), self.ws_ptr, self.ws_bytes, ap, ab, _stream(stream)),
               "asterx_prim2con_adjoint")

    def rk4_steps_checkpointed(self, U, P, dt, ckpt, stats=None, stream=None):
        """len(ckpt) RK4 steps in place; ckpt[k] (device tensor of U's shape) receives the state before step k."""
        arr = (State * len(ckpt))(*[state_struct(c) for c in ckpt])
        u, p = state_struct(U), prims_struct(P)
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_rk4_steps_checkpointed(*self._args(), float(dt), len(ckpt), ctypes.byref(u),
                                                   ctypes.byref(p), arr, sp, self.ws_ptr, self.ws_bytes,
                                                   _stream(stream)), "asterx_rk4_steps_checkpointed")

    def rk4_adjoint_steps(self, ckpt, P, lam, dt, stream=None):
        """In place: lam = dJ/dU_N on entry, dJ/dU_0 on exit, for the steps whose checkpoints are ckpt."""
        ap, ab = self._adjoint_ws()
        arr = (State * len(ckpt))(*[state_struct(c) for c in ckpt])
        p, l = prims_struct(P), state_struct(lam)
        _check(lib().asterx_rk4_adjoint_steps(*self._args(), float(dt), len(ckpt), arr, ctypes.byref(p),
                                              ctypes.byref(l), self.ws_ptr, self.ws_bytes, ap, ab,
                                              _stream(stream)), "asterx_rk4_adjoint_steps")


# ---------------------------------------------------------------------------------------- measurement helpers


def profile_enable(max_launches: int):
    _check(lib().asterx_profile_enable(int(max_launches)), "asterx_profile_enable")


def profile_read():
    n = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().asterx_profile_read(ctypes.byref(n), ctypes.byref(ms)), "asterx_profile_read")
    return n.value, ms.value


def profile_disable():
    lib().asterx_profile_disable()


def dfma_probe(out, blocks, threads, iters, stream=None):
    _check(lib().asterx_dfma_probe(ctypes.c_void_p(out.data_ptr()), int(blocks), int(threads), int(iters),
                                   _stream(stream)), "asterx_dfma_probe")


def quotient(a, b, out, stream=None):
    """The corrected quotient a / b (from 1 / b and one correction) of device doubles, into out."""
    _check(lib().asterx_quotient(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), int(a.numel()), _stream(stream)), "asterx_quotient")


def recip(d, out, stream=None):
    """The two-step reciprocal (face solve, WENO-Z weights, Noble iteration) of the device doubles d, into out."""
    _check(lib().asterx_recip(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(d.numel()),
                              _stream(stream)), "asterx_recip")


def newton_rcp(d, out, stream=None):
    """The speed solver's Newton-correction reciprocal of the device doubles d, written to out."""
    _check(lib().asterx_newton_rcp(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(d.numel()),
                                   _stream(stream)), "asterx_newton_rcp")


NOALLOC_MAX_ENTRIES = 65536


def con2prim_noalloc(params: dict, n, g, x0, dx, bc, metric, U, P, flags=None, stats=None, stream=None):
    """asterx_con2prim_noalloc: the recovery with its scratch in the library's fixed device array (no caller
    workspace); see include/asterx.h for the size limit and the sharing rules."""
    p, b = params_struct(params), block_struct(n, g, x0, dx, bc)
    m, u, pr = metric_struct(metric), state_struct(U), prims_struct(P)
    fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
    sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
    return lib().asterx_con2prim_noalloc(ctypes.byref(p), ctypes.byref(b), ctypes.byref(m), ctypes.byref(u),
                                         ctypes.byref(pr), fl, sp, _stream(stream))


def prolong(coarse, fine, Uc, Pc, Uf, Pf, all_points=False, stream=None):
    """Fine ghost points (every point with all_points) of Uf, Pf from the coarse level (two Solvers)."""
    _check(lib().asterx_prolong(ctypes.byref(coarse.b), ctypes.byref(fine.b), ctypes.byref(state_struct(Uc)),
                                ctypes.byref(prims_struct(Pc)), ctypes.byref(state_struct(Uf)),
                                ctypes.byref(prims_struct(Pf)), int(bool(all_points)), _stream(stream)),
           "asterx_prolong")


def rk4_step_refined(coarse, fine, Uc, Pc, Uf, Pf, dt, stats=None, stream=None):
    """One RK4 step of two refinement levels (coarse and fine Solvers, both prepared) with time step dt."""
    sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
    _check(lib().asterx_rk4_step_refined(ctypes.byref(coarse.p), ctypes.byref(coarse.b), ctypes.byref(fine.b),
                                         float(dt), ctypes.byref(state_struct(Uc)), ctypes.byref(prims_struct(Pc)),
                                         ctypes.byref(state_struct(Uf)), ctypes.byref(prims_struct(Pf)), sp,
                                         coarse.ws_ptr, coarse.ws_bytes, fine.ws_ptr, fine.ws_bytes,
                                         _stream(stream)), "asterx_rk4_step_refined")


def rk4_step_subcycled(coarse, fine, Uc, Pc, Uf, Pf, dt, stats=None, stream=None):
    """One coarse RK4 step of size dt with the fine level subcycled (two steps of dt / 2; coarse and fine
    Solvers, both prepared).  The scratch space is a torch allocation kept on the coarse Solver."""
    import torch
    need = int(lib().asterx_subcycle_workspace_size(ctypes.byref(coarse.b)))
    if need == 0:
        raise AsterxError("asterx_subcycle_workspace_size: invalid coarse block")
    buf = getattr(coarse, "_subcycle_ws", None)
    if buf is None or buf.numel() < need + 256:
        buf = torch.empty(need + 256, dtype=torch.uint8, device=coarse.ws.device)
        coarse._subcycle_ws = buf
    ptr = ctypes.c_void_p(buf.data_ptr() + (-buf.data_ptr()) % 256)
    sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
    _check(lib().asterx_rk4_step_subcycled(ctypes.byref(coarse.p), ctypes.byref(coarse.b), ctypes.byref(fine.b),
                                           float(dt), ctypes.byref(state_struct(Uc)), ctypes.byref(prims_struct(Pc)),
                                           ctypes.byref(state_struct(Uf)), ctypes.byref(prims_struct(Pf)), sp,
                                           coarse.ws_ptr, coarse.ws_bytes, fine.ws_ptr, fine.ws_bytes, ptr, need,
                                           _stream(stream)), "asterx_rk4_step_subcycled")


class Batch:
    """Many blocks advanced together by asterx_batched_step.  `blocks` is a list of (n, g, x0, dx, bc, metric,
    U, P) with device tensors; all share `params`.  The pooled workspace is one torch allocation.  With
    `tiling` = (nblk, cuts) — blocks per axis and per axis the nblk + 1 cell offsets of the block boundaries,
    blocks listed x fastest — the blocks tile one domain and exchange their shared ghost layers."""

    def __init__(self, params: dict, blocks, device="cuda", tiling=None):
        import torch
        self.tiling = None
        if tiling is not None:
            nblk, cuts = tiling
            self._cuts = [(ctypes.c_int * len(c))(*[int(x) for x in c]) for c in cuts]
            t = Tiling()
            for d in range(3):
                t.nblk[d] = int(nblk[d])
                t.cuts[d] = ctypes.cast(self._cuts[d], ctypes.POINTER(ctypes.c_int))
            self.tiling = t
        self.params = dict(params)
        self.p = params_struct(self.params)
        self.keep = blocks  # tensors stay alive while the tables refer to them
        arr = (BatchBlock * len(blocks))()
        for i, (n, g, x0, dx, bc, M, U, P) in enumerate(blocks):
            arr[i].blk = block_struct(n, g, x0, dx, bc)
            arr[i].metric = metric_struct(M)
            arr[i].U = state_struct(U)
            arr[i].P = prims_struct(P)
        self.arr = arr
        self.nb = len(blocks)
        self.ws_bytes = int(lib().asterx_batch_workspace_size(arr, self.nb))
        if self.ws_bytes == 0:
            raise AsterxError(ASTERX_EINVAL, "invalid batch")
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = ctypes.c_void_p(self.ws.data_ptr() + off)

    def prepare(self, stream=None):
        if self.tiling is not None:
            _check(lib().asterx_batch_prepare_tiled(ctypes.byref(self.p), self.arr, self.nb, ctypes.byref(self.tiling),
                                                    self.ws_ptr, self.ws_bytes, _stream(stream)),
                   "asterx_batch_prepare_tiled")
        else:
            _check(lib().asterx_batch_prepare(ctypes.byref(self.p), self.arr, self.nb, self.ws_ptr, self.ws_bytes,
                                              _stream(stream)), "asterx_batch_prepare")

    def prim2con(self, stream=None):
        _check(lib().asterx_batch_prim2con(ctypes.byref(self.p), self.arr, self.nb, self.ws_ptr, self.ws_bytes,
                                           _stream(stream)), "asterx_batch_prim2con")

    def step(self, dt, nsteps=1, stats=None, stream=None):
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _check(lib().asterx_batched_step(ctypes.byref(self.p), self.arr, self.nb, float(dt), int(nsteps), sp,
                                         self.ws_ptr, self.ws_bytes, _stream(stream)), "asterx_batched_step")

    def release(self):
        """Drops the step graphs the library cached for this batch's workspace (also done on deletion)."""
        if getattr(self, "ws_ptr", None) is not None:
            lib().asterx_batch_release(self.ws_ptr)

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass
