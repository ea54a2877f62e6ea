"""ctypes loader for the CPU oracle (oracle/asterx_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg are the only
users.  The product library never imports this package.  Arrays follow the layout of the workloads module:
float64, shape (Nz+1, Ny+1, Nx+1) per field, stacked as (9, ...) for the state (D, Sx, Sy, Sz, tau, Ax, Ay,
Az, Psi), (5, ...) for the primitives (rho, press, velx, vely, velz) and (16, ...) for the vertex metric.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asterx_oracle.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ (-O2, no floating-point contraction, OpenMP, portable flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("rho_atm", ctypes.c_double), ("K_atm", ctypes.c_double),
                ("gamma_atm", ctypes.c_double), ("c2p_tol", ctypes.c_double), ("c2p_maxiter", ctypes.c_int),
                ("brent_maxiter", ctypes.c_int), ("W_max", ctypes.c_double), ("recon", ctypes.c_int),
                ("gauge", ctypes.c_int), ("xi_lorenz", ctypes.c_double), ("use_fallback", ctypes.c_int),
                ("flux", ctypes.c_int), ("efield", ctypes.c_int)]


class OBlock(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("g", ctypes.c_int), ("x0", ctypes.c_double * 3),
                ("dx", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


class OStats(ctypes.Structure):
    _fields_ = [("n_noble", ctypes.c_ulonglong), ("n_fallback", ctypes.c_ulonglong),
                ("n_atm", ctypes.c_ulonglong), ("n_failed", ctypes.c_ulonglong), ("iters", ctypes.c_ulonglong)]

    def asdict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None
_P = ctypes.POINTER(ctypes.c_double)
_PP = ctypes.POINTER(_P)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_abi_version.restype = ctypes.c_int
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        # one thread unless asked otherwise: the test suite runs in parallel processes
        L.oracle_set_threads(int(os.environ.get("ORACLE_THREADS", "1")))
        for name in ("oracle_ghost_fill_state", "oracle_ghost_fill_prims"):
            getattr(L, name).argtypes = [ctypes.POINTER(OBlock), _PP]
        L.oracle_prim2con.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP]
        L.oracle_con2prim.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP,
                                      ctypes.c_void_p, ctypes.POINTER(OStats)]
        L.oracle_rhs.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP,
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_ulonglong)]
        L.oracle_face_B.argtypes = [ctypes.POINTER(OBlock), _PP, _PP]
        L.oracle_rk_stage.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, ctypes.c_int,
                                      ctypes.c_double, _PP, _PP, _PP, _PP, _PP, ctypes.c_void_p,
                                      ctypes.POINTER(OStats)]
        L.oracle_point_prim2con.argtypes = [ctypes.POINTER(OParams), _P, _P, _P, _P, _P]
        L.oracle_point_wave_speeds.argtypes = [ctypes.POINTER(OParams), _P, _P, _P, ctypes.c_int, _P]
        L.oracle_point_c2p.argtypes = [ctypes.POINTER(OParams), _P, _P, _P, _P, _P, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
        L.oracle_point_c2p.restype = ctypes.c_int
        L.oracle_batch_c2p.argtypes = [ctypes.POINTER(OParams), ctypes.c_long, _P, _P, _P, _P, _P, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_batch_prim2con.argtypes = [ctypes.POINTER(OParams), ctypes.c_long, _P, _P, _P, _P]
        L.oracle_point_recon.argtypes = [ctypes.c_int, _P, _P, _P]
        L.oracle_face_flops.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, ctypes.c_int,
                                        ctypes.c_int, _P]
        L.oracle_recon_flops.argtypes = [ctypes.c_int, _P, _P]
        L.oracle_stage_flops.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, ctypes.c_int,
                                         ctypes.c_double, _P]
        L.oracle_point_sources.argtypes = [ctypes.POINTER(OParams), _P, _P, _P, _P, _P, _P, _P]
        L.oracle_grid_sources.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP]
        L.oracle_rk_stage_given_ghosts.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, ctypes.c_int,
                                                   ctypes.c_double, _PP, _PP, _PP, _PP, _PP, ctypes.c_void_p,
                                                   ctypes.POINTER(OStats)]
        IP = ctypes.POINTER(ctypes.c_int)
        L.oracle_prolong.argtypes = [ctypes.POINTER(OBlock), ctypes.POINTER(OBlock), IP, _PP, _PP, _PP, _PP,
                                     ctypes.c_int]
        L.oracle_restrict.argtypes = [ctypes.POINTER(OBlock), ctypes.POINTER(OBlock), IP, _PP, _PP]
        L.oracle_point_face.argtypes = [ctypes.POINTER(OParams), _P, _P, _P, ctypes.c_double, ctypes.c_int, _P]
        L.oracle_centre_metric.argtypes = [ctypes.POINTER(OBlock), _PP, _PP]
        L.oracle_face_metric.argtypes = [ctypes.POINTER(OBlock), _PP, ctypes.c_int, _PP]
        L.oracle_tmunu.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP]
        L.oracle_stage_jvp.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP, _PP,
                                       _PP, ctypes.c_double]
        L.oracle_rk4_jvp.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP, _PP, _PP,
                                     ctypes.c_double]
        L.oracle_prim2con_jvp.argtypes = [ctypes.POINTER(OParams), ctypes.POINTER(OBlock), _PP, _PP, _PP, _PP,
                                          _PP, _PP]
    return _lib


# ------------------------------------------------------------------------------------------------------------


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's grid loops; returns the count in effect."""
    return int(lib().oracle_set_threads(int(n)))


def params_struct(p: dict) -> OParams:
    return OParams(p["gamma"], p["rho_atm"], p["K_atm"], p["gamma_atm"], p["c2p_tol"], int(p["c2p_maxiter"]),
                   int(p["brent_maxiter"]), p["W_max"], int(p["recon"]), int(p["gauge"]), p["xi_lorenz"],
                   int(p["use_fallback"]), int(p.get("flux", 0)), int(p.get("efield", 0)))


def block_struct(w) -> OBlock:
    b = OBlock()
    for d in range(3):
        b.n[d] = int(w.n[d])
        b.x0[d] = float(w.x0[d])
        b.dx[d] = float(w.dx[d])
        b.bc[d] = int(w.bc[d])
    b.g = int(w.g)
    return b


def _ptrs(arr: np.ndarray):
    assert arr.dtype == np.float64 and arr.flags.c_contiguous
    n = arr.shape[0]
    t = (_P * n)(*[arr[v].ctypes.data_as(_P) for v in range(n)])
    return t


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def metric_array(w) -> np.ndarray:
    from paper_2406_11669_gb300.workloads import METRIC_NAMES
    return np.ascontiguousarray(np.stack([w.metric[k] for k in METRIC_NAMES]))


def prims_array(w) -> np.ndarray:
    from paper_2406_11669_gb300.workloads import PRIM_NAMES
    return np.ascontiguousarray(np.stack([w.prims[k] for k in PRIM_NAMES]))


def initial_state(w):
    """(U, prims): the state with D, S, tau from the oracle's own prim->cons and A, Psi from the workload."""
    P = prims_array(w)
    U = np.zeros((9,) + w.shape)
    U[5] = w.A["Ax"]
    U[6] = w.A["Ay"]
    U[7] = w.A["Az"]
    U[8] = w.Psi
    M = metric_array(w)
    prim2con(w, M, U, P)
    return U, P


def ghost_fill_state(w, U):
    lib().oracle_ghost_fill_state(ctypes.byref(block_struct(w)), _ptrs(U))


def ghost_fill_prims(w, P):
    lib().oracle_ghost_fill_prims(ctypes.byref(block_struct(w)), _ptrs(P))


def prim2con(w, M, U, P, params=None):
    pp = params_struct(params or w.params)
    lib().oracle_prim2con(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), _ptrs(U), _ptrs(P))


def prim2con_jvp(w, M, U, dA, P, dP, params=None):
    """J dU0: the derivative of the conserved fields (D, S, tau) in the direction (dA (3 fields), dP (5
    fields)), by forward-mode dual numbers through B~ = curl A, the centre field and the pointwise map.  U's
    fields 0..4 receive the values (as prim2con writes them); A (fields 5..7) is read."""
    JU = np.zeros((5,) + w.shape)
    lib().oracle_prim2con_jvp(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)),
                              _ptrs(M), _ptrs(U), _ptrs(np.ascontiguousarray(dA)), _ptrs(P),
                              _ptrs(np.ascontiguousarray(dP)), _ptrs(JU))
    return JU


def con2prim(w, M, U, P, params=None):
    pp = params_struct(params or w.params)
    flags = np.zeros(w.shape, dtype=np.int8)
    st = OStats()
    lib().oracle_con2prim(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), _ptrs(U), _ptrs(P),
                          flags.ctypes.data, ctypes.byref(st))
    return flags, st.asdict()


def face_B(w, U):
    Bf = np.zeros((3,) + w.shape)
    lib().oracle_face_B(ctypes.byref(block_struct(w)), _ptrs(U), _ptrs(Bf))
    return Bf


def rhs(w, M, U, P, dt=None, params=None):
    """dU/dt of the 9 state fields (state and primitives must have their ghosts filled)."""
    pp = params_struct(params or w.params)
    dU = np.zeros((9,) + w.shape)
    it = (ctypes.c_ulonglong * 2)()
    lib().oracle_rhs(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), _ptrs(U), _ptrs(P), _ptrs(dU),
                     float(dt if dt is not None else w.dt), it)
    return dU, (int(it[0]), int(it[1]))


def rk_stage(w, M, stage, dt, Un, Us, Unext, Uacc, P, params=None):
    pp = params_struct(params or w.params)
    flags = np.zeros(w.shape, dtype=np.int8)
    st = OStats()
    lib().oracle_rk_stage(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), int(stage), float(dt),
                          _ptrs(Un), _ptrs(Us), _ptrs(Unext), _ptrs(Uacc), _ptrs(P), flags.ctypes.data,
                          ctypes.byref(st))
    return flags, st.asdict()


def rk4_step(w, M, U, P, dt=None, params=None):
    """One classical RK4 step; returns (U_next, stats summed over the four stages).  U is ghost-filled and
    may be reset to the atmosphere in place by the first stage's recovery; P is updated in place."""
    dt = float(dt if dt is not None else w.dt)
    Uacc = np.zeros_like(U)
    Us = U
    tot = None
    for s in range(4):
        Unext = Us.copy()  # entries outside the owned ranges stay defined; owned entries are overwritten
        _, st = rk_stage(w, M, s, dt, U, Us, Unext, Uacc, P, params)
        tot = st if tot is None else {k: tot[k] + st[k] for k in tot}
        Us = Unext
    return Us, tot


def centre_metric(w, M):
    """(53, ...) interpolated metric at every cell centre: alpha, beta^i, gamma_ij (6), gamma^ij (6), sqrt(gamma),
    K_ij (6), d_i alpha (3), d_i beta^j (9), d_i gamma_jk (18)."""
    out = np.zeros((53,) + w.shape)
    lib().oracle_centre_metric(ctypes.byref(block_struct(w)), _ptrs(M), _ptrs(out))
    return out


def face_metric(w, M, d):
    """(17, ...) interpolated metric at the faces normal to d: alpha, beta^i, gamma_ij, gamma^ij, sqrt(gamma)."""
    out = np.zeros((17,) + w.shape)
    lib().oracle_face_metric(ctypes.byref(block_struct(w)), _ptrs(M), int(d), _ptrs(out))
    return out


TMUNU_NAMES = ("tt", "tx", "ty", "tz", "xx", "xy", "xz", "yy", "yz", "zz")


def tmunu(w, M, U, P, params=None):
    """T_{mu nu} (10, ...) at the vertices g..g+n of every axis (zero elsewhere); U's A and P ghost-filled."""
    T = np.zeros((10,) + w.shape)
    lib().oracle_tmunu(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)), _ptrs(M),
                       _ptrs(U), _ptrs(P), _ptrs(T))
    return T


def stage_jvp(w, M, U, dU, P, dt=None, params=None):
    """(L, J dU): the stage operator L(U) = RHS(ghost fill U, recovery, ghost fill P) and its derivative in
    the direction dU, by forward-mode dual numbers (the recovery differentiated at its root).  U and dU are
    read only (ghost filled on copies); P holds the recovery's guess and receives the primitives."""
    L = np.zeros((9,) + w.shape)
    JL = np.zeros((9,) + w.shape)
    lib().oracle_stage_jvp(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)),
                           _ptrs(M), _ptrs(np.ascontiguousarray(U)), _ptrs(np.ascontiguousarray(dU)), _ptrs(P),
                           _ptrs(L), _ptrs(JL), float(dt if dt is not None else w.dt))
    return L, JL


def rk4_jvp(w, M, U, dU, P, dt=None, params=None):
    """(U_next, J dU): one RK4 step as rk4_step forms it and its derivative in the direction dU (owned
    ranges); U and dU are read only, P holds the guess and receives the last stage's primitives."""
    U1 = np.zeros((9,) + w.shape)
    JU1 = np.zeros((9,) + w.shape)
    lib().oracle_rk4_jvp(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)),
                         _ptrs(M), _ptrs(np.ascontiguousarray(U)), _ptrs(np.ascontiguousarray(dU)), _ptrs(P),
                         _ptrs(U1), _ptrs(JU1), float(dt if dt is not None else w.dt))
    return U1, JU1


def _ivec(L):
    return (ctypes.c_int * 3)(*[int(x) for x in L])


def prolong(wc, wf, L, Uc, Pc, Uf, Pf, all_points=False):
    """Fills the fine block's ghost points (every point with all_points) of Uf (9) and Pf (5) from the coarse
    level; the fine interior covers the coarse interior cells L .. L + n_fine / 2 - 1."""
    lib().oracle_prolong(ctypes.byref(block_struct(wc)), ctypes.byref(block_struct(wf)), _ivec(L), _ptrs(Uc),
                         _ptrs(Pc), _ptrs(Uf), _ptrs(Pf), int(bool(all_points)))


def restrict(wc, wf, L, Uc, Uf):
    """The coarse points under the fine interior from the fine state (9 fields)."""
    lib().oracle_restrict(ctypes.byref(block_struct(wc)), ctypes.byref(block_struct(wf)), _ivec(L), _ptrs(Uc),
                          _ptrs(Uf))


def rk_stage_given_ghosts(w, M, stage, dt, Un, Us, Unext, Uacc, P, params=None):
    pp = params_struct(params or w.params)
    flags = np.zeros(w.shape, dtype=np.int8)
    st = OStats()
    lib().oracle_rk_stage_given_ghosts(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), int(stage),
                                       float(dt), _ptrs(Un), _ptrs(Us), _ptrs(Unext), _ptrs(Uacc), _ptrs(P),
                                       flags.ctypes.data, ctypes.byref(st))
    return flags, st.asdict()


def refined_rk4_step(wc, Mc, Uc, Pc, wf, Mf, Uf, Pf, L, dt, params=None):
    """One RK4 step of two refinement levels with one time step (no subcycling): each stage runs the coarse
    stage, prolongs the coarse stage state and primitives to the fine ghost points, and runs the fine stage on
    them; then the coarse points under the fine interior are restricted.  Returns (Uc_next, Uf_next)."""
    Ua_c, Ua_f = np.zeros_like(Uc), np.zeros_like(Uf)
    Us_c, Us_f = Uc, Uf
    for s in range(4):
        Un_c = Us_c.copy()
        rk_stage(wc, Mc, s, dt, Uc, Us_c, Un_c, Ua_c, Pc, params)
        prolong(wc, wf, L, Us_c, Pc, Us_f, Pf)
        Un_f = Us_f.copy()
        rk_stage_given_ghosts(wf, Mf, s, dt, Uf, Us_f, Un_f, Ua_f, Pf, params)
        Us_c, Us_f = Un_c, Un_f
    restrict(wc, wf, L, Us_c, Us_f)
    return Us_c, Us_f


def rk4_dense_weights(theta):
    """The continuous extension of classical RK4: u(t_n + theta h) ~ u_n + h sum_i b_i(theta) k_i with
    b_1 = theta - 3 theta^2 / 2 + 2 theta^3 / 3, b_2 = b_3 = theta^2 - 2 theta^3 / 3, b_4 = -theta^2 / 2 +
    2 theta^3 / 3 (b(1) = the RK4 weights).  Returns the four b_i and their first three theta-derivatives as a
    (4, 4) array [derivative order, i]."""
    t = float(theta)
    return np.array([
        [t - 1.5 * t * t + 2.0 * t ** 3 / 3.0, t * t - 2.0 * t ** 3 / 3.0, t * t - 2.0 * t ** 3 / 3.0,
         -0.5 * t * t + 2.0 * t ** 3 / 3.0],
        [1.0 - 3.0 * t + 2.0 * t * t, 2.0 * t - 2.0 * t * t, 2.0 * t - 2.0 * t * t, -t + 2.0 * t * t],
        [-3.0 + 4.0 * t, 2.0 - 4.0 * t, 2.0 - 4.0 * t, -1.0 + 4.0 * t],
        [4.0, -4.0, -4.0, 4.0]])


def subcycle_stage_weights(m):
    """Weights beta[s, i] of the coarse slopes h k_i in the fine ghost values of stage s of fine substep m (0 or
    1; each of half the coarse step h, starting at theta0 = m / 2).  The fine RK4 stage states of a linear
    problem are Taylor sums about the substep start: u, u + (h_f/2) u', u + (h_f/2) u' + (h_f^2/4) u'', and
    u + h_f u' + (h_f^2/2) u'' + (h_f^3/4) u'''; u and its time derivatives come from the coarse step's dense
    output (the time interpolation that replaces buffer zones in the paper's subcycling, Sec. 3.10; the
    stage-consistent form of Mongwane 2015).  With h_f = h / 2 the powers of h_f become 1/4, 1/16, 1/2, 1/8 and
    1/32 times the dense output's theta-derivatives."""
    B = rk4_dense_weights(0.5 * m)
    return np.array([B[0],
                     B[0] + 0.25 * B[1],
                     B[0] + 0.25 * B[1] + (1.0 / 16.0) * B[2],
                     B[0] + 0.5 * B[1] + 0.125 * B[2] + (1.0 / 32.0) * B[3]])


def subcycle_ghost_state(Un, Y1, Y2, Y3, U1, m, s):
    """The coarse state that feeds the fine ghost points at stage s of fine substep m: U_n + sum_i beta[s, i]
    h k_i, the slopes taken from the coarse step's base U_n, stage states Y_1..Y_3 and result U_1 = U_{n+1}."""
    g0 = 2.0 * (Y1 - Un)
    g1 = 2.0 * (Y2 - Un)
    g2 = Y3 - Un
    g3 = 6.0 * (U1 - Un) - g0 - 2.0 * g1 - 2.0 * g2
    beta = subcycle_stage_weights(m)
    return Un + (beta[s, 0] * g0 + beta[s, 1] * g1 + beta[s, 2] * g2 + beta[s, 3] * g3)


def subcycled_rk4_step(wc, Mc, Uc, Pc, wf, Mf, Uf, Pf, L, dt, params=None):
    """One coarse RK4 step of size dt with the fine level subcycled (two RK4 steps of dt / 2).  The coarse step
    runs first and keeps its stage states Y_1..Y_3 and its base U_n (as the first stage's recovery leaves it);
    its slopes h k_i follow from them (h k_1 = 2 (Y_1 - U_n), h k_2 = 2 (Y_2 - U_n), h k_3 = Y_3 - U_n,
    h k_4 = 6 (U_{n+1} - U_n) - h k_1 - 2 h k_2 - 2 h k_3).  Before each fine stage the coarse state
    U_n + sum_i beta[s, i] h k_i (subcycle_stage_weights) is ghost-filled, recovered (seeded by the previous
    recovery, starting from the primitives the coarse step leaves) and prolonged to the fine ghost points.  After
    both substeps the coarse points under the fine interior are restricted.  Returns (Uc_next, Uf_next)."""
    h = float(dt)
    Ua = np.zeros_like(Uc)
    Y = [Uc, np.array(Uc), np.array(Uc), np.array(Uc)]
    Un = None
    for s in range(4):
        nxt = Y[s + 1] if s < 3 else Uc
        rk_stage(wc, Mc, s, h, Uc, Y[s], nxt, Ua, Pc, params)
        if s == 0:
            Un = Uc.copy()
    Pt = Pc.copy()
    for m in range(2):
        Ua_f = np.zeros_like(Uf)
        Us_f = Uf
        for s in range(4):
            Yt = subcycle_ghost_state(Un, Y[1], Y[2], Y[3], Uc, m, s)
            ghost_fill_state(wc, Yt)
            con2prim(wc, Mc, Yt, Pt, params)
            ghost_fill_prims(wc, Pt)
            prolong(wc, wf, L, Yt, Pt, Us_f, Pf)
            Un_f = Us_f.copy()
            rk_stage_given_ghosts(wf, Mf, s, 0.5 * h, Uf, Us_f, Un_f, Ua_f, Pf, params)
            Us_f = Un_f
        Uf = Us_f
    restrict(wc, wf, L, Uc, Uf)
    return Uc, Uf


def rk2_step(w, M, U, P, dt=None, params=None):
    """One RK2 step (explicit midpoint: U_1 = U_n + dt/2 L(U_n), U_{n+1} = U_n + dt L(U_1)); as rk4_step."""
    dt = float(dt if dt is not None else w.dt)
    Uacc = np.zeros_like(U)
    U1 = U.copy()
    _, s0 = rk_stage(w, M, 4, dt, U, U, U1, Uacc, P, params)
    U2 = U1.copy()
    _, s1 = rk_stage(w, M, 5, dt, U, U1, U2, Uacc, P, params)
    return U2, {k: s0[k] + s1[k] for k in s0}


def rk4_step_metrics(w, Ms, U, P, dt=None, params=None):
    """One RK4 step whose stage s runs on the metric Ms[s] (a time-dependent spacetime sampled at the stage
    times); otherwise as rk4_step."""
    dt = float(dt if dt is not None else w.dt)
    Uacc = np.zeros_like(U)
    Us = U
    tot = None
    for s in range(4):
        Unext = Us.copy()
        _, st = rk_stage(w, Ms[s], s, dt, U, Us, Unext, Uacc, P, params)
        tot = st if tot is None else {k: tot[k] + st[k] for k in tot}
        Us = Unext
    return Us, tot


def point_face(params, m16, L8, R8, Bn, d):
    """One face solve: dict with F (5), Fb (3: induction fluxes along d of B~^x,y,z), cmax, cmin, vbar (3).
    L8, R8: rho, p, u^x, u^y, u^z (u = W v), B^x, B^y, B^z (undensitised; the normal entry unused)."""
    out = np.zeros(13)
    lib().oracle_point_face(ctypes.byref(params_struct(params)), _p(np.ascontiguousarray(m16, float)),
                            _p(np.ascontiguousarray(L8, float)), _p(np.ascontiguousarray(R8, float)), float(Bn),
                            int(d), _p(out))
    return dict(F=out[:5], Fb=out[5:8], cmax=out[8], cmin=out[9], vbar=out[10:13])


def point_prim2con(params, m16, prim5, B3):
    cons = np.zeros(5)
    fl = np.zeros(15)
    lib().oracle_point_prim2con(ctypes.byref(params_struct(params)), _p(np.ascontiguousarray(m16, float)),
                                _p(np.ascontiguousarray(prim5, float)), _p(np.ascontiguousarray(B3, float)),
                                _p(cons), _p(fl))
    return cons, fl.reshape(3, 5)


def point_wave_speeds(params, m16, prim5, B3, d):
    lam = np.zeros(2)
    lib().oracle_point_wave_speeds(ctypes.byref(params_struct(params)), _p(np.ascontiguousarray(m16, float)),
                                   _p(np.ascontiguousarray(prim5, float)), _p(np.ascontiguousarray(B3, float)),
                                   int(d), _p(lam))
    return lam[0], lam[1]


def point_c2p(params, m16, cons5, B3, guess5, which=0):
    out = np.zeros(5)
    it = ctypes.c_int(0)
    flag = lib().oracle_point_c2p(ctypes.byref(params_struct(params)), _p(np.ascontiguousarray(m16, float)),
                                  _p(np.ascontiguousarray(cons5, float)), _p(np.ascontiguousarray(B3, float)),
                                  _p(np.ascontiguousarray(guess5, float)), _p(out), int(which), ctypes.byref(it))
    return flag, out, it.value


def batch_c2p(params, m16, cons5, B3, guess5, which=0):
    """Recovery of n undensitised states: arrays (n,16), (n,5), (n,3), (n,5) -> (flags, prims, iters)."""
    n = cons5.shape[0]
    out = np.zeros((n, 5))
    flags = np.zeros(n, dtype=np.int32)
    iters = np.zeros(n, dtype=np.int32)
    lib().oracle_batch_c2p(ctypes.byref(params_struct(params)), n, _p(np.ascontiguousarray(m16, float)),
                           _p(np.ascontiguousarray(cons5, float)), _p(np.ascontiguousarray(B3, float)),
                           _p(np.ascontiguousarray(guess5, float)), _p(out), int(which), flags.ctypes.data,
                           iters.ctypes.data)
    return flags, out, iters


def batch_prim2con(params, m16, prim5, B3):
    n = prim5.shape[0]
    out = np.zeros((n, 5))
    lib().oracle_batch_prim2con(ctypes.byref(params_struct(params)), n, _p(np.ascontiguousarray(m16, float)),
                                _p(np.ascontiguousarray(prim5, float)), _p(np.ascontiguousarray(B3, float)),
                                _p(out))
    return out


def point_recon(scheme, a5):
    aL = np.zeros(1)
    aR = np.zeros(1)
    lib().oracle_point_recon(int(scheme), _p(np.ascontiguousarray(a5, float)), _p(aL), _p(aR))
    return aL[0], aR[0]


def point_sources(params, m16, dalp, dbeta, dg, prim5, B3):
    src = np.zeros(5)
    lib().oracle_point_sources(ctypes.byref(params_struct(params)), _p(np.ascontiguousarray(m16, float)),
                               _p(np.ascontiguousarray(dalp, float)), _p(np.ascontiguousarray(dbeta, float)),
                               _p(np.ascontiguousarray(dg, float)), _p(np.ascontiguousarray(prim5, float)),
                               _p(np.ascontiguousarray(B3, float)), _p(src))
    return src


def grid_sources(w, M, U, P, params=None):
    pp = params_struct(params or w.params)
    src = np.zeros((5,) + w.shape)
    lib().oracle_grid_sources(ctypes.byref(pp), ctypes.byref(block_struct(w)), _ptrs(M), _ptrs(U), _ptrs(P),
                              _ptrs(src))
    return src


def face_flops(w, M, U, P, d, stride=1, params=None):
    """Flop counts of the face solve along d: dict(faces, add, mul, div, sqrt, speed_iters)."""
    out = np.zeros(6)
    lib().oracle_face_flops(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)),
                            _ptrs(M), _ptrs(U), _ptrs(P), int(d), int(stride), _p(out))
    return dict(zip(("faces", "add", "mul", "div", "sqrt", "speed_iters"), out.tolist()))


def recon_flops(scheme, a5):
    out = np.zeros(4)
    lib().oracle_recon_flops(int(scheme), _p(np.ascontiguousarray(a5, float)), _p(out))
    return dict(zip(("add", "mul", "div", "sqrt"), out.tolist()))


STAGE_FLOP_PARTS = ("ghost_state", "recovery", "ghost_prims", "faces", "hydro_cells", "potentials", "edges", "psi",
                    "combine")


def stage_flops(w, M, U, P, stage=1, dt=None, params=None):
    """Algorithmic flop counts of one RK stage on state U (ghosts filled on a copy) with the recovery's guess P,
    part by part (each a dict add, mul, div, sqrt), plus the interior cell count (n_cells), the speed iterations and faces of the
    face solves, the flops spent inside the speed Newton loops, the Noble iterations and the recovery's branch
    counts.  The right-hand side's recomputation of the face and centre field is reported apart ('rhs_field')."""
    out = np.zeros(60)
    lib().oracle_stage_flops(ctypes.byref(params_struct(params or w.params)), ctypes.byref(block_struct(w)),
                             _ptrs(M), _ptrs(np.ascontiguousarray(U)), _ptrs(np.ascontiguousarray(P)), int(stage),
                             float(dt if dt is not None else w.dt), _p(out))
    keys = ("add", "mul", "div", "sqrt")
    res = {"n_cells": out[0]}
    for q, name in enumerate(STAGE_FLOP_PARTS):
        res[name] = dict(zip(keys, out[1 + 4 * q:5 + 4 * q].tolist()))
    res["rhs_field"] = dict(zip(keys, out[45:49].tolist()))
    res.update(speed_iters=out[37], faces_solved=out[38], speed_loop_flops=out[39], noble_iters=out[40],
               n_noble=out[41], n_fallback=out[42], n_atm=out[43], n_failed=out[44], cellvar_flops=out[49],
               recon_flops=out[50], facesolve_flops=out[51], edge_ppm_flops=out[52], recovery_field_flops=out[53])
    return res
