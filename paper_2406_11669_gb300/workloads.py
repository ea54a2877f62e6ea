"""Seeded synthetic inputs for the GRMHD RK stage (shared by the CUDA path's tests, the oracle's tests and bench).

This module only *generates inputs*: primitive variables at cell centres, the vector potential at edges, the
scalar potential at vertices and a frozen 3+1 metric (alpha, beta^i, gamma_ij, K_ij) at vertices.  It holds none
of the method's arithmetic: no conserved variables, no discrete curl, no reconstruction.  Each side (the CUDA
library and the CPU oracle) turns these arrays into conserved variables with its own prim->cons.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), written here as a counter-based hash:
the k-th draw of a stream with seed s is mix(s + (k+1)*0x9E3779B97F4A7C15).

Data layout (also the layout of the C ABI): every field is a float64 array of shape (Nz+1, Ny+1, Nx+1), x fastest,
with N = n + 2g per axis.  Index (i, j, k) names the object whose lower corner is vertex (i, j, k):
cell centre (i+1/2, j+1/2, k+1/2), x-face (i, j+1/2, k+1/2), x-edge (i+1/2, j, k), vertex (i, j, k).
Vertex i sits at x0 + (i - g) dx.

The five workloads follow the paper's tests and benchmarks (Sec. 4, Table 1, Sec. 5 "Setup A"):
  flat_modes             32^3 periodic, flat metric, minmod, smooth Fourier-mode data
  balsara_schwarzschild  128^3, Schwarzschild (isotropic), WENO-Z, Balsara-1 states split along x (Table 1)
  star_layout/star_block 512 uneven blocks, Schwarzschild M=0.2, PPM, magnetised-star profile (Eq. magtovAvec,
                         n_s = 1)
  weak_field_modes       64^3 periodic, weak-field lapse, PPM, smooth data (adjoint workload, seeded target)
  torus_jet              256^3, Schwarzschild, WENO-Z, rotating torus plus an axial jet with W up to 7
Constants the paper leaves open are fixed here and listed in the design notes of the repository.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RECON_MINMOD, RECON_PPM, RECON_WENOZ, RECON_MP5 = 0, 1, 2, 3
BC_PERIODIC, BC_COPY = 0, 1
GAUGE_LORENZ, GAUGE_ALGEBRAIC = 0, 1
FLUX_HLLE, FLUX_LXF = 0, 1          # Riemann solver (Eq. HLLEfluxes, Eq. LxFfluxes)
EFIELD_UCT, EFIELD_FCT = 0, 1       # edge electric field (upwind or flux constrained transport)

PRIM_NAMES = ("rho", "press", "velx", "vely", "velz")
CONS_NAMES = ("D", "Sx", "Sy", "Sz", "tau")
STATE_NAMES = ("D", "Sx", "Sy", "Sz", "tau", "Ax", "Ay", "Az", "Psi")
METRIC_NAMES = ("alp", "betax", "betay", "betaz", "gxx", "gxy", "gxz", "gyy", "gyz", "gzz",
                "kxx", "kxy", "kxz", "kyy", "kyz", "kzz")

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start..start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Sequential uniform doubles in [0, 1) from one SplitMix64 stream (53-bit mantissa)."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, count: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (splitmix64(self.seed, self.pos, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        self.pos += count
        return lo + (hi - lo) * u

    def choice(self, options, count: int = 1) -> np.ndarray:
        u = self.uniform(count)
        idx = np.minimum((u * len(options)).astype(np.int64), len(options) - 1)
        return np.asarray(options)[idx]


@dataclasses.dataclass
class Workload:
    """One block of synthetic input: geometry, parameters, primitives, potentials and the frozen metric."""
    name: str
    n: tuple            # interior cells (nx, ny, nz)
    g: int              # ghost layers
    x0: tuple           # position of the first interior vertex
    dx: tuple
    bc: tuple           # per axis: BC_PERIODIC or BC_COPY
    params: dict
    dt: float
    prims: dict         # rho, press, velx, vely, velz at cell centres
    A: dict             # Ax, Ay, Az at edges
    Psi: np.ndarray     # densitised scalar potential at vertices
    metric: dict        # 16 fields at vertices

    @property
    def N(self):
        return tuple(int(m) + 2 * self.g for m in self.n)

    @property
    def shape(self):
        """numpy shape of every field array: (Nz+1, Ny+1, Nx+1)."""
        N = self.N
        return (N[2] + 1, N[1] + 1, N[0] + 1)

    @property
    def interior_cells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def default_params(**kw) -> dict:
    p = dict(gamma=5.0 / 3.0, rho_atm=1e-7, K_atm=1.0, gamma_atm=5.0 / 3.0, c2p_tol=1e-13, c2p_maxiter=100,
             brent_maxiter=300, W_max=50.0, recon=RECON_PPM, gauge=GAUGE_LORENZ, xi_lorenz=0.0, use_fallback=1,
             flux=FLUX_HLLE, efield=EFIELD_UCT)
    p.update(kw)
    return p


# ----------------------------------------------------------------------------------------------------------
# positions of the staggered objects


def _axis(x0, dx, g, Np1, half):
    return x0 + (np.arange(Np1, dtype=np.float64) - g + (0.5 if half else 0.0)) * dx


def positions(n, g, x0, dx, stagger):
    """Broadcastable (z, y, x) coordinate arrays for a staggering given as three half-offset flags (x, y, z)."""
    N = [int(m) + 2 * g for m in n]
    ax = [_axis(x0[d], dx[d], g, N[d] + 1, stagger[d]) for d in range(3)]
    X = ax[0][None, None, :]
    Y = ax[1][None, :, None]
    Z = ax[2][:, None, None]
    return X, Y, Z


CELL = (True, True, True)
VERTEX = (False, False, False)
XEDGE = (True, False, False)
YEDGE = (False, True, False)
ZEDGE = (False, False, True)


def _full(shape, v):
    return np.full(shape, v, dtype=np.float64)


def flat_metric(shape) -> dict:
    m = {k: _full(shape, 0.0) for k in METRIC_NAMES}
    m["alp"][...] = 1.0
    m["gxx"][...] = 1.0
    m["gyy"][...] = 1.0
    m["gzz"][...] = 1.0
    return m


def schwarzschild_isotropic(X, Y, Z, M, centre, shape) -> dict:
    """Isotropic Schwarzschild slice: psi = 1 + M/2r, alpha = (1 - M/2r)/(1 + M/2r), gamma_ij = psi^4 delta_ij,
    beta = K = 0 (a static slice).  The metric is an input of the path; this is how the input is drawn."""
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    r = np.broadcast_to(r, shape)
    h = M / (2.0 * r)
    psi = 1.0 + h
    m = {k: _full(shape, 0.0) for k in METRIC_NAMES}
    m["alp"][...] = (1.0 - h) / (1.0 + h)
    p4 = psi ** 4
    m["gxx"][...] = p4
    m["gyy"][...] = p4
    m["gzz"][...] = p4
    return m


def _fourier_vector_modes(rng: Rng, nmodes: int, kmax: int = 2, transverse: bool = True):
    modes = []
    while len(modes) < nmodes:
        k = rng.choice(np.arange(-kmax, kmax + 1), 3).astype(np.float64)
        if not np.any(k):
            continue
        a = rng.uniform(3, -1.0, 1.0)
        if transverse:
            a = a - (a @ k) / (k @ k) * k
        phi = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
        modes.append((k, a, phi))
    return modes


def _eval_vector_sin(modes, X, Y, Z, shape):
    out = [np.zeros(shape) for _ in range(3)]
    for k, a, phi in modes:
        s = np.sin(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + phi)
        for d in range(3):
            out[d] += a[d] * s
    return out


def _fourier_potential(rng: Rng, nmodes: int, n, g, x0, dx, shape, Bmax, with_b2=False):
    """A = sum_m c_m cos(2 pi k_m . x + phi_m) sampled at the three edge families; amplitudes rescaled so that
    the analytic |curl A| peaks at Bmax over the cell centres (the discrete field is then close to Bmax).  With
    with_b2, also returns |curl A|^2 at the cell centres."""
    modes = _fourier_vector_modes(rng, nmodes, transverse=False)
    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    Bc = [np.zeros(shape) for _ in range(3)]
    for k, c, phi in modes:
        s = -2.0 * math.pi * np.sin(2.0 * math.pi * (k[0] * Xc + k[1] * Yc + k[2] * Zc) + phi)
        kc = np.cross(k, c)
        for d in range(3):
            Bc[d] += kc[d] * s
    bmag = np.sqrt(Bc[0] ** 2 + Bc[1] ** 2 + Bc[2] ** 2).max()
    scale = Bmax / bmag if bmag > 0 else 0.0
    A = {}
    for d, (name, st) in enumerate((("Ax", XEDGE), ("Ay", YEDGE), ("Az", ZEDGE))):
        X, Y, Z = positions(n, g, x0, dx, st)
        acc = np.zeros(shape)
        for k, c, phi in modes:
            acc += scale * c[d] * np.cos(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + phi)
        A[name] = acc
    if with_b2:
        return A, scale ** 2 * (Bc[0] ** 2 + Bc[1] ** 2 + Bc[2] ** 2)
    return A


def _smooth_periodic(name, n, seed, gamma, recon, alp_amp, vmax, Bmax, rho_amp, rho_modes):
    g = 3
    x0 = (0.0, 0.0, 0.0)
    dx = tuple(1.0 / m for m in n)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rng = Rng(seed)
    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    rho = np.broadcast_to(1.0 + 0.0 * Xc, shape).copy()
    if rho_modes == 0:
        rho += rho_amp * np.sin(2.0 * math.pi * Xc)
    else:
        for _ in range(rho_modes):
            k = rng.choice(np.arange(-2, 3), 3).astype(np.float64)
            if not np.any(k):
                k[0] = 1.0
            amp = float(rng.uniform(1, -1.0, 1.0)[0])
            phi = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
            rho += rho_amp * amp * np.sin(2.0 * math.pi * (k[0] * Xc + k[1] * Yc + k[2] * Zc) + phi)
    press = _full(shape, 1.0)
    vm = _fourier_vector_modes(rng, 4)
    v = _eval_vector_sin(vm, Xc, Yc, Zc, shape)
    vmag = np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2).max()
    v = [c * (vmax / vmag) for c in v]
    A = _fourier_potential(rng, 4, n, g, x0, dx, shape, Bmax)
    if alp_amp == 0.0:
        metric = flat_metric(shape)
    else:
        metric = flat_metric(shape)
        Xv, _, _ = positions(n, g, x0, dx, VERTEX)
        metric["alp"][...] = np.broadcast_to(1.0 - alp_amp * np.sin(2.0 * math.pi * Xv), shape)
    params = default_params(gamma=gamma, gamma_atm=gamma, rho_atm=1e-7, K_atm=1.0, recon=recon)
    prims = dict(rho=rho, press=press, velx=v[0], vely=v[1], velz=v[2])
    return Workload(name, tuple(n), g, x0, dx, (BC_PERIODIC,) * 3, params, 0.25 * min(dx), prims, A,
                    _full(shape, 0.0), metric)


def flat_modes(n=(32, 32, 32), seed=101) -> Workload:
    """32^3 periodic on [0,1]^3, flat metric, Gamma=4/3, minmod; rho = 1 + 0.1 sin 2 pi x, p = 1;
    |v| <= 0.1 from 4 transverse Fourier modes, |B| ~ 0.1 from 4 potential modes; dt = dx/4."""
    return _smooth_periodic("flat_modes_32cube_periodic_minmod", n, seed, 4.0 / 3.0, RECON_MINMOD,
                            0.0, 0.1, 0.1, 0.1, 0)


def weak_field_modes(n=(64, 64, 64), seed=104) -> Workload:
    """64^3 periodic, lapse 1 - 0.01 sin 2 pi x, gamma = I, Gamma = 4/3, PPM; rho = 1 + 0.05 * 3 modes, p = 1,
    |v| <= 0.2, |B| ~ 0.2; dt = dx/4 (the adjoint workload: 10 RK4 steps)."""
    return _smooth_periodic("weak_field_modes_64cube_periodic_ppm", n, seed, 4.0 / 3.0, RECON_PPM,
                            0.01, 0.2, 0.2, 0.05, 3)


def weak_field_target(w: Workload, seed=1104) -> np.ndarray:
    """Seeded target density field T = 1 + 0.05 * 3 modes at cell centres for the adjoint loss."""
    rng = Rng(seed)
    Xc, Yc, Zc = positions(w.n, w.g, w.x0, w.dx, CELL)
    T = np.ones(w.shape)
    for _ in range(3):
        k = rng.choice(np.arange(-2, 3), 3).astype(np.float64)
        if not np.any(k):
            k[1] = 1.0
        amp = float(rng.uniform(1, -1.0, 1.0)[0])
        phi = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
        T = T + 0.05 * amp * np.sin(2.0 * math.pi * (k[0] * Xc + k[1] * Yc + k[2] * Zc) + phi)
    return T


GRADIENT_DIRECTIONS = ("all_fields_a", "all_fields_b", "rho", "potentials")


def gradient_directions(w: Workload, seed=4201):
    """Seeded directions in the initial data for checking a gradient with respect to it: a list of (name, dP, dA)
    with dP (5, ...) over the primitives and dA (3, ...) over A_x, A_y, A_z, nonzero on the independent entries
    only (cells g..g+n-1; an edge's vertex-like axes g..g+n, or g..g+n-1 where periodic).  Entries are uniform in
    [-1, 1] times the field's scale (its largest magnitude there, at least 0.05 for a primitive and 1e-3 for a
    potential).  The pressure is never perturbed.  Directions, in GRADIENT_DIRECTIONS order: rho, v^i and A_i
    together (two draws), rho alone, A_i alone."""
    rng = Rng(seed)
    g, n = w.g, w.n
    cells = tuple(slice(g, g + n[a]) for a in (2, 1, 0))

    def edge(v):
        return tuple(slice(g, g + n[a] + (0 if (a == v or w.bc[a] == BC_PERIODIC) else 1)) for a in (2, 1, 0))

    def draw(arr, sl, floor):
        shape = arr[sl].shape
        scale = max(float(np.abs(arr[sl]).max()), floor)
        return rng.uniform(int(np.prod(shape)), -1.0, 1.0).reshape(shape) * scale

    out = []
    for name in GRADIENT_DIRECTIONS:
        dP = np.zeros((5,) + w.shape)
        dA = np.zeros((3,) + w.shape)
        if name != "potentials":
            for v in ((0, 2, 3, 4) if name != "rho" else (0,)):
                dP[v][cells] = draw(w.prims[PRIM_NAMES[v]], cells, 0.05)
        if name != "rho":
            for v, key in enumerate(("Ax", "Ay", "Az")):
                dA[v][edge(v)] = draw(w.A[key], edge(v), 1e-3)
        out.append((name, dP, dA))
    return out


def _smooth_scalar(rng: Rng, nmodes: int, X, Y, Z, shape, amp):
    """amp * sum of `nmodes` unit-amplitude-weighted sines with seeded wave vectors (|k_i| <= 2) and phases."""
    out = np.zeros(shape)
    for _ in range(nmodes):
        k = rng.choice(np.arange(-2, 3), 3).astype(np.float64)
        if not np.any(k):
            k[2] = 1.0
        a = float(rng.uniform(1, -1.0, 1.0)[0])
        phi = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
        out += amp * a * np.sin(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + phi)
    return np.broadcast_to(out, shape).copy()


def smooth_general(n=(12, 10, 11), seed=106, recon=RECON_PPM, bc=BC_PERIODIC, gauge=GAUGE_LORENZ) -> Workload:
    """Periodic-in-form smooth data on [0,1]^3 in which every field varies in all three directions: rho, p from
    3 modes each (5%), compressive velocity (|v| <= 0.2), |B| ~ 0.2, Psi ~ 0.02, and a general frozen metric
    (lapse, shift, spatial metric and extrinsic curvature all perturbed by 2-3% with their own modes).  No
    reconstruction limiter sits exactly at a branch point here, which makes it the workload for checking
    derivatives against finite differences."""
    g = 3
    x0 = (0.0, 0.0, 0.0)
    dx = tuple(1.0 / m for m in n)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rng = Rng(seed)
    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    rho = 1.0 + _smooth_scalar(rng, 3, Xc, Yc, Zc, shape, 0.05)
    press = 0.8 + _smooth_scalar(rng, 3, Xc, Yc, Zc, shape, 0.05)
    vm = _fourier_vector_modes(rng, 4, transverse=False)
    v = _eval_vector_sin(vm, Xc, Yc, Zc, shape)
    vmag = np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2).max()
    v = [c * (0.2 / vmag) for c in v]
    A = _fourier_potential(rng, 4, n, g, x0, dx, shape, 0.2)
    Xv, Yv, Zv = positions(n, g, x0, dx, VERTEX)
    psi = _smooth_scalar(rng, 2, Xv, Yv, Zv, shape, 0.02)
    metric = flat_metric(shape)
    metric["alp"] = 1.0 + _smooth_scalar(rng, 2, Xv, Yv, Zv, shape, 0.02)
    for name in ("betax", "betay", "betaz"):
        metric[name] = _smooth_scalar(rng, 2, Xv, Yv, Zv, shape, 0.03)
    for name in ("gxx", "gxy", "gxz", "gyy", "gyz", "gzz"):
        diag = name in ("gxx", "gyy", "gzz")
        metric[name] = (1.0 if diag else 0.0) + _smooth_scalar(rng, 2, Xv, Yv, Zv, shape, 0.03 if diag else 0.015)
    for name in METRIC_NAMES[10:]:
        metric[name] = _smooth_scalar(rng, 2, Xv, Yv, Zv, shape, 0.02)
    params = default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-7, K_atm=1.0, recon=recon, gauge=gauge)
    prims = dict(rho=rho, press=press, velx=v[0], vely=v[1], velz=v[2])
    rname = {RECON_MINMOD: "minmod", RECON_PPM: "ppm", RECON_WENOZ: "wenoz", RECON_MP5: "mp5"}[recon]
    bname = "periodic" if bc == BC_PERIODIC else "copy"
    return Workload(f"smooth_general_{rname}_{bname}", tuple(n), g, x0, dx, (bc,) * 3, params, 0.25 * min(dx), prims,
                    A, psi, metric)


def loop_advection(n=24, seed=0) -> Workload:
    """Magnetic loop advection (Sec. 4, loop-advection test): periodic [-1/2, 1/2]^2 (one cell in z), rho = 1,
    p = 3, v = (1/12, 1/24, 1/24), A_z = max(0, A_loop (R_loop - r)) with A_loop = 1e-3, R_loop = 0.3, Gamma = 5/3,
    minmod, dt = dx/4.  (The seed is unused: the set-up is deterministic.)"""
    g = 3
    nn = (n, n, 1)
    dx = (1.0 / n, 1.0 / n, 1.0 / n)
    x0 = (-0.5, -0.5, 0.0)
    N = [m + 2 * g for m in nn]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rho = _full(shape, 1.0)
    press = _full(shape, 3.0)
    v = [_full(shape, 1.0 / 12.0), _full(shape, 1.0 / 24.0), _full(shape, 1.0 / 24.0)]
    X, Y, _ = positions(nn, g, x0, dx, ZEDGE)
    r = np.sqrt(X ** 2 + Y ** 2)
    Az = np.broadcast_to(np.maximum(0.0, 1e-3 * (0.3 - r)), shape).copy()
    A = dict(Ax=_full(shape, 0.0), Ay=_full(shape, 0.0), Az=Az)
    params = default_params(gamma=5.0 / 3.0, gamma_atm=5.0 / 3.0, rho_atm=1e-7, K_atm=1.0, recon=RECON_MINMOD)
    prims = dict(rho=rho, press=press, velx=v[0], vely=v[1], velz=v[2])
    return Workload("loop_advection_2d", nn, g, x0, dx, (BC_PERIODIC,) * 3, params, 0.25 * dx[0], prims, A,
                    _full(shape, 0.0), flat_metric(shape))


def smooth_periodic_1d(n, seed=110, recon=RECON_PPM) -> Workload:
    """Smooth periodic data on [0,1] along x (one cell in y and z, every field a function of x only), shaped like
    the adjoint workload: rho = 1 + 0.05 * 3 modes, p = 1 + 0.05 * 2 modes, all three velocity components from
    4 modes (|v| <= 0.2), transverse B ~ 0.2 from A_y(x), A_z(x), lapse 1 - 0.01 sin 2 pi x; Gamma = 4/3,
    dt = dx/4.  The modes do not depend on n, so blocks of several n sample the same continuum data (a
    self-convergence study)."""
    g = 3
    nn = (n, 1, 1)
    dx = (1.0 / n, 1.0 / n, 1.0 / n)
    x0 = (0.0, 0.0, 0.0)
    N = [m + 2 * g for m in nn]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rng = Rng(seed)

    def modes(count):
        out = []
        for _ in range(count):
            k = float(rng.choice(np.arange(1, 3), 1)[0])
            a = rng.uniform(3, -1.0, 1.0)
            phi = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
            out.append((k, a, phi))
        return out

    def field(md, X, amp, comp=0, fn=np.sin):
        acc = np.zeros(shape)
        for k, a, phi in md:
            acc = acc + amp * a[comp] * fn(2.0 * math.pi * k * X + phi)
        return np.broadcast_to(acc, shape).copy()

    Xc, _, _ = positions(nn, g, x0, dx, CELL)
    rho = 1.0 + field(modes(3), Xc, 0.05)
    press = 1.0 + field(modes(2), Xc, 0.05)
    vm = modes(4)
    v = [field(vm, Xc, 1.0, d) for d in range(3)]
    vmag = max(np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2).max(), 1e-300)
    v = [c * (0.2 / vmag) for c in v]
    am = modes(4)
    Xy, _, _ = positions(nn, g, x0, dx, YEDGE)
    Xz, _, _ = positions(nn, g, x0, dx, ZEDGE)
    A = dict(Ax=_full(shape, 0.0), Ay=field(am, Xy, 0.2 / (2.0 * math.pi), 1, np.cos),
             Az=field(am, Xz, 0.2 / (2.0 * math.pi), 2, np.cos))
    metric = flat_metric(shape)
    Xv, _, _ = positions(nn, g, x0, dx, VERTEX)
    metric["alp"] = np.broadcast_to(1.0 - 0.01 * np.sin(2.0 * math.pi * Xv), shape).copy()
    params = default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-7, K_atm=1.0, recon=recon)
    prims = dict(rho=rho, press=press, velx=v[0], vely=v[1], velz=v[2])
    return Workload(f"smooth_periodic_1d_{n}", nn, g, x0, dx, (BC_PERIODIC,) * 3, params, 0.25 * dx[0], prims, A,
                    _full(shape, 0.0), metric)


def balsara_schwarzschild(n=(128, 128, 128), seed=102) -> Workload:
    """128^3 on [-1/2,1/2]^3, copy BCs, Gamma = 5/3, WENO-Z.  Table 1 test-1 states split at x = 0:
    left rho=1, p=1, right rho=0.125, p=0.1, v=0; densitised field B~x = 0.5, B~y = +1 (left) / -1 (right)
    from A_z = |x| + y/2.  Frozen isotropic Schwarzschild metric, M = 0.1, centred at (-1, 0, 0)."""
    del seed  # the data is deterministic; the seed is kept for a uniform signature
    g = 3
    x0 = (-0.5, -0.5, -0.5)
    dx = tuple(1.0 / m for m in n)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    Xc, _, _ = positions(n, g, x0, dx, CELL)
    left = np.broadcast_to(Xc < 0.0, shape)
    rho = np.where(left, 1.0, 0.125)
    press = np.where(left, 1.0, 0.1)
    zero = _full(shape, 0.0)
    X, Y, Z = positions(n, g, x0, dx, ZEDGE)
    Az = np.broadcast_to(np.abs(X) + 0.5 * Y, shape).copy()
    Xv, Yv, Zv = positions(n, g, x0, dx, VERTEX)
    metric = schwarzschild_isotropic(Xv, Yv, Zv, 0.1, (-1.0, 0.0, 0.0), shape)
    params = default_params(gamma=5.0 / 3.0, gamma_atm=5.0 / 3.0, rho_atm=1e-7, K_atm=1.0, recon=RECON_WENOZ)
    prims = dict(rho=rho, press=press, velx=zero.copy(), vely=zero.copy(), velz=zero.copy())
    A = dict(Ax=zero.copy(), Ay=zero.copy(), Az=Az)
    return Workload("balsara_schwarzschild_128cube_wenoz", tuple(n), g, x0, dx, (BC_COPY,) * 3, params,
                    0.25 * min(dx), prims, A, zero.copy(), metric)


def _poloidal_potential(n, g, x0, dx, shape, press_fn, grad_press_fn, p_cut, target):
    """A_phi = A_b varpi^2 max(p - p_cut, 0) (Eq. magtovAvec with n_s = 1) as Cartesian edge components
    A_x = -y A_b f, A_y = x A_b f.  A_b is set from the analytic flat-space curl so that max B^2/(2p) = target."""
    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    p = np.broadcast_to(press_fn(Xc, Yc, Zc), shape)
    f = np.maximum(p - p_cut, 0.0)
    gx, gy, gz = (np.broadcast_to(c, shape) for c in grad_press_fn(Xc, Yc, Zc))
    on = f > 0.0
    X = np.broadcast_to(Xc, shape)
    Y = np.broadcast_to(Yc, shape)
    Bx = np.where(on, -X * gz, 0.0)
    By = np.where(on, -Y * gz, 0.0)
    Bz = np.where(on, 2.0 * f + X * gx + Y * gy, 0.0)
    ratio = np.where(on, (Bx ** 2 + By ** 2 + Bz ** 2) / (2.0 * np.maximum(p, 1e-300)), 0.0)
    Ab = math.sqrt(target / ratio.max()) if ratio.max() > 0 else 0.0
    A = {}
    for name, st in (("Ax", XEDGE), ("Ay", YEDGE), ("Az", ZEDGE)):
        Xe, Ye, Ze = positions(n, g, x0, dx, st)
        fe = np.broadcast_to(np.maximum(press_fn(Xe, Ye, Ze) - p_cut, 0.0), shape)
        if name == "Ax":
            A[name] = -np.broadcast_to(Ye, shape) * Ab * fe
        elif name == "Ay":
            A[name] = np.broadcast_to(Xe, shape) * Ab * fe
        else:
            A[name] = _full(shape, 0.0)
    return A, Ab


def _star(R=0.4, rho_c=1e-3, rho_floor=1e-10, K=100.0):
    def rho(X, Y, Z):
        return np.maximum(rho_c * (1.0 - (X * X + Y * Y + Z * Z) / (R * R)), rho_floor)

    def press(X, Y, Z):
        return K * rho(X, Y, Z) ** 2

    def grad_press(X, Y, Z):
        r = rho(X, Y, Z)
        inside = r > rho_floor
        c = np.where(inside, 2.0 * K * r * (-2.0 * rho_c / (R * R)), 0.0)
        return c * X, c * Y, c * Z

    return rho, press, grad_press


def star_block(n, origin, dx=1.0 / 256.0, name="star_block") -> Workload:
    """One block of the uneven batch: magnetised star rho = max(1e-3 (1 - r^2/0.4^2), 1e-10), p = 100 rho^2,
    v = 0, poloidal A_phi with p_cut = 0.04 p_max and max b^2/2p ~ 1e-2; Schwarzschild M = 0.2 at (-1,0,0);
    Gamma = 2, atmosphere K = 100, Gamma_atm = 2, rho_atm = 1e-10; copy BCs, PPM."""
    g = 3
    x0 = tuple(float(o) for o in origin)
    dxs = (dx, dx, dx)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rho_fn, press_fn, _ = _star()
    Xc, Yc, Zc = positions(n, g, x0, dxs, CELL)
    rho = np.broadcast_to(rho_fn(Xc, Yc, Zc), shape).copy()
    press = np.broadcast_to(press_fn(Xc, Yc, Zc), shape).copy()
    p_max = 100.0 * 1e-3 ** 2
    # A_b must not depend on the block: it is fixed once on a reference grid through the star's centre.
    A, _ = _poloidal_potential_fixed(n, g, x0, dxs, shape, press_fn, 0.04 * p_max, _star_Ab())
    Xv, Yv, Zv = positions(n, g, x0, dxs, VERTEX)
    metric = schwarzschild_isotropic(Xv, Yv, Zv, 0.2, (-1.0, 0.0, 0.0), shape)
    zero = _full(shape, 0.0)
    params = default_params(gamma=2.0, gamma_atm=2.0, rho_atm=1e-10, K_atm=100.0, recon=RECON_PPM)
    prims = dict(rho=rho, press=press, velx=zero.copy(), vely=zero.copy(), velz=zero.copy())
    return Workload(name, tuple(int(m) for m in n), g, x0, dxs, (BC_COPY,) * 3, params, 0.25 * dx, prims, A,
                    zero.copy(), metric)


_AB_CACHE = {}


def _star_Ab():
    if "c3" not in _AB_CACHE:
        n = (64, 64, 64)
        g = 3
        dx = 1.0 / 64.0
        shape = (n[2] + 2 * g + 1,) * 3
        _, press_fn, gp = _star()
        _, Ab = _poloidal_potential(n, g, (-0.5, -0.5, -0.5), (dx, dx, dx), shape, press_fn, gp,
                                    0.04 * 100.0 * 1e-3 ** 2, 1e-2)
        _AB_CACHE["c3"] = Ab
    return _AB_CACHE["c3"]


def _poloidal_potential_fixed(n, g, x0, dx, shape, press_fn, p_cut, Ab):
    A = {}
    for name, st in (("Ax", XEDGE), ("Ay", YEDGE), ("Az", ZEDGE)):
        Xe, Ye, Ze = positions(n, g, x0, dx, st)
        fe = np.broadcast_to(np.maximum(press_fn(Xe, Ye, Ze) - p_cut, 0.0), shape)
        if name == "Ax":
            A[name] = -np.broadcast_to(Ye, shape) * Ab * fe
        elif name == "Ay":
            A[name] = np.broadcast_to(Xe, shape) * Ab * fe
        else:
            A[name] = _full(shape, 0.0)
    return A, Ab


def star_layout(nblocks=512, seed=103, sizes=(16, 24, 32, 48, 64), dx=1.0 / 256.0):
    """Seeded block table of the uneven batch: per axis n from `sizes`, origins uniform on the dx lattice such
    that each block lies inside [-1/2, 1/2]^3.  Returns a list of (n, origin)."""
    rng = Rng(seed)
    out = []
    for _ in range(nblocks):
        n = tuple(int(v) for v in rng.choice(np.asarray(sizes), 3))
        origin = []
        for d in range(3):
            cells = int(round(1.0 / dx)) - n[d]
            c = int(min(int(rng.uniform(1)[0] * (cells + 1)), cells))
            origin.append(-0.5 + c * dx)
        out.append((n, tuple(origin)))
    return out


def torus_jet(n=(256, 256, 256), seed=105) -> Workload:
    """256^3 on [-1/2,1/2]^3, copy BCs, Gamma = 4/3, WENO-Z.  Torus rho = max(1e-2 exp(-(varpi-0.3)^2/0.01
    - z^2/0.01), 1e-10), p = 0.1 rho^(4/3), rigid rotation Omega = 0.5, plus an axial jet (varpi < 0.1) whose
    Lorentz factor W = 1 + 6 exp(-(varpi/0.04)^2)(0.75 + 0.25 cos(2 pi z + phi_seed)) reaches 7.  Poloidal
    A_phi on the torus with max b^2/2p ~ 1e-2.  Schwarzschild M = 0.1 at (-1, 0, 0); atmosphere K = 0.1,
    Gamma_atm = 4/3, rho_atm = 1e-10."""
    g = 3
    x0 = (-0.5, -0.5, -0.5)
    dx = tuple(1.0 / m for m in n)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    rng = Rng(seed)
    phi_seed = float(rng.uniform(1, 0.0, 2.0 * math.pi)[0])
    Omega = 0.5
    M = 0.1
    centre = (-1.0, 0.0, 0.0)

    def rho_fn(X, Y, Z):
        w = np.sqrt(X * X + Y * Y)
        return np.maximum(1e-2 * np.exp(-(w - 0.3) ** 2 / 0.01 - Z * Z / 0.01), 1e-10)

    def press_fn(X, Y, Z):
        return 0.1 * rho_fn(X, Y, Z) ** (4.0 / 3.0)

    def grad_press_fn(X, Y, Z):
        w = np.sqrt(X * X + Y * Y) + 1e-300
        r = rho_fn(X, Y, Z)
        inside = r > 1e-10
        dr_dw = r * (-2.0 * (w - 0.3) / 0.01)
        dr_dz = r * (-2.0 * Z / 0.01)
        c = np.where(inside, 0.1 * (4.0 / 3.0) * r ** (1.0 / 3.0), 0.0)
        return c * dr_dw * X / w, c * dr_dw * Y / w, c * dr_dz

    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    rho = np.broadcast_to(rho_fn(Xc, Yc, Zc), shape).copy()
    press = np.broadcast_to(press_fn(Xc, Yc, Zc), shape).copy()
    # conformal factor of the input metric at the cell centres, used only to keep the drawn speeds subluminal
    rr = np.sqrt((Xc - centre[0]) ** 2 + Yc ** 2 + Zc ** 2)
    psi2 = (1.0 + M / (2.0 * rr)) ** 2
    w = np.sqrt(Xc * Xc + Yc * Yc)
    vhat_phi = Omega * w * psi2
    Wjet = 1.0 + 6.0 * np.exp(-(w / 0.04) ** 2) * (0.75 + 0.25 * np.cos(2.0 * math.pi * Zc + phi_seed))
    vhat_z = np.where(w < 0.1, np.sign(Zc) * np.sqrt(np.maximum(1.0 - 1.0 / Wjet ** 2, 0.0)), 0.0)
    vhat_z = vhat_z * np.sqrt(np.maximum(1.0 - vhat_phi ** 2, 0.0))
    velx = np.broadcast_to(-Omega * Yc, shape).copy()
    vely = np.broadcast_to(Omega * Xc, shape).copy()
    velz = np.broadcast_to(vhat_z / psi2, shape).copy()
    p_max = 0.1 * 1e-2 ** (4.0 / 3.0)
    A, _ = _poloidal_potential(n, g, x0, dx, shape, press_fn, grad_press_fn, 0.04 * p_max, 1e-2)
    Xv, Yv, Zv = positions(n, g, x0, dx, VERTEX)
    metric = schwarzschild_isotropic(Xv, Yv, Zv, M, centre, shape)
    params = default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-10, K_atm=0.1, recon=RECON_WENOZ)
    prims = dict(rho=rho, press=press, velx=velx, vely=vely, velz=velz)
    return Workload("torus_jet_256cube_schwarzschild_wenoz", tuple(n), g, x0, dx, (BC_COPY,) * 3, params,
                    0.25 * min(dx), prims, A, _full(shape, 0.0), metric)


def recovery_states(n=(48, 48, 48), seed=107, Bmax=0.03) -> Workload:
    """A block whose cells hold independent seeded states for the primitive recovery, over the ranges of the
    recovery's round-trip check: rho log-uniform in [1e-10, 1], p / rho log-uniform in [1e-4, 10], Lorentz factor
    uniform in [1, 10] in a random direction; the field comes from a smooth seeded potential (|B| up to about
    Bmax), and rho is raised where needed to keep b^2 / rho <= 100 (b^2 <= B^2 at rest, taken from the
    potential's analytic curl).  Isotropic Schwarzschild M = 0.1 at (-1, 0, 0) on [-1/2, 1/2]^3; Gamma = 4/3,
    atmosphere floor 1e-12 (below every drawn density)."""
    g = 3
    x0 = (-0.5, -0.5, -0.5)
    dx = tuple(1.0 / m for m in n)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    size = shape[0] * shape[1] * shape[2]
    rng = Rng(seed)
    rho = 10.0 ** rng.uniform(size, -10.0, 0.0).reshape(shape)
    press = rho * 10.0 ** rng.uniform(size, -4.0, 1.0).reshape(shape)
    Wl = rng.uniform(size, 1.0, 10.0).reshape(shape)
    # random directions: normalised Gaussian-free draw (uniform in a cube, rejected outside the unit ball)
    dirs = rng.uniform(3 * size, -1.0, 1.0).reshape((3,) + shape)
    norm = np.sqrt(dirs[0] ** 2 + dirs[1] ** 2 + dirs[2] ** 2)
    norm = np.where(norm > 1e-3, norm, 1.0)
    M, centre = 0.1, (-1.0, 0.0, 0.0)
    Xc, Yc, Zc = positions(n, g, x0, dx, CELL)
    rr = np.sqrt((Xc - centre[0]) ** 2 + (Yc - centre[1]) ** 2 + (Zc - centre[2]) ** 2)
    psi2 = (1.0 + M / (2.0 * rr)) ** 2
    speed = np.sqrt(1.0 - 1.0 / Wl ** 2) / psi2  # gamma_ij v^i v^j = psi^4 |v|^2 = 1 - 1/W^2
    vel = [dirs[d] / norm * speed for d in range(3)]
    A, B2 = _fourier_potential(rng, 4, n, g, x0, dx, shape, Bmax, with_b2=True)
    scale = np.maximum(1.0, 1.2 * B2 * psi2 ** 2 / (100.0 * rho))  # gamma_ij B^i B^j = psi^4 |B|^2
    rho = rho * scale
    press = press * scale
    Xv, Yv, Zv = positions(n, g, x0, dx, VERTEX)
    metric = schwarzschild_isotropic(Xv, Yv, Zv, M, centre, shape)
    params = default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-12, K_atm=0.1, recon=RECON_PPM)
    prims = dict(rho=rho, press=press, velx=vel[0], vely=vel[1], velz=vel[2])
    return Workload("recovery_states", tuple(n), g, x0, dx, (BC_COPY,) * 3, params, 0.25 * min(dx), prims, A,
                    _full(shape, 0.0), metric)


def weak_field_wave(nx, recon=RECON_PPM, amp=1e-3, cfl=0.25) -> Workload:
    """A smooth small-amplitude wave on the adjoint workload's weak-field lapse alpha = 1 - 0.01 sin 2 pi x
    (gamma = I, beta = K = 0), periodic on [0, 1] along x, one cell across y and z: rho = 1 + amp sin 2 pi x,
    p = 1 + amp cos 2 pi x, v^x = amp sin 2 pi x, B = 0, Gamma = 4/3; dt = cfl dx (for self-convergence)."""
    n = (int(nx), 1, 1)
    g = 3
    x0 = (0.0, 0.0, 0.0)
    h = 1.0 / nx
    dx = (h, h, h)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    Xc, _, _ = positions(n, g, x0, dx, CELL)
    Xv, _, _ = positions(n, g, x0, dx, VERTEX)
    s = np.broadcast_to(np.sin(2.0 * math.pi * Xc), shape)
    c = np.broadcast_to(np.cos(2.0 * math.pi * Xc), shape)
    prims = dict(rho=1.0 + amp * s, press=1.0 + amp * c, velx=amp * s, vely=_full(shape, 0.0),
                 velz=_full(shape, 0.0))
    metric = flat_metric(shape)
    metric["alp"][...] = np.broadcast_to(1.0 - 0.01 * np.sin(2.0 * math.pi * Xv), shape)
    zero = _full(shape, 0.0)
    params = default_params(gamma=4.0 / 3.0, gamma_atm=4.0 / 3.0, rho_atm=1e-7, K_atm=1.0, recon=recon)
    return Workload(f"weak_field_wave_{nx}", n, g, x0, dx, (BC_PERIODIC,) * 3, params, cfl * h, prims,
                    dict(Ax=zero, Ay=zero.copy(), Az=zero.copy()), zero.copy(), metric)


def alfven_wave(nx, recon=RECON_MINMOD, ny=1, nz=1, cfl=0.2):
    """Circularly polarised Alfven wave of Sec. 4.2: rho = 1, p = 0.5, A0 = 1, v_A = 0.5, B^x = 1,
    v^y = -v_A A0 cos kx, v^z = -v_A A0 sin kx, B^y = A0 B^x cos kx, B^z = A0 B^x sin kx, Gamma = 5/3, on
    [-1/2, 1/2] along x (periodic).  The potential A_y = -(A0 B^x/k) cos kx, A_z = -(A0 B^x/k) sin kx + B^x y
    has exactly this curl in the continuum.  Its B^x y part is not periodic in y, so y and z use copy BCs
    (linear extrapolation of A, which is exact for it); the data do not depend on y or z."""
    g = 3
    n = (nx, ny, nz)
    L = 1.0
    x0 = (-0.5, -0.5 * ny / nx, -0.5 * nz / nx)
    h = L / nx
    dx = (h, h, h)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    k = 2.0 * math.pi / L
    vA, A0, Bx = 0.5, 1.0, 1.0
    Xc, _, _ = positions(n, g, x0, dx, CELL)
    rho = _full(shape, 1.0)
    press = _full(shape, 0.5)
    velx = _full(shape, 0.0)
    vely = np.broadcast_to(-vA * A0 * np.cos(k * Xc), shape).copy()
    velz = np.broadcast_to(-vA * A0 * np.sin(k * Xc), shape).copy()
    # B = curl A with A_x = 0, A_y = (A0 Bx/k) sin(kx)... : B^y = -dA_z/dx, B^z = dA_y/dx
    Xy, _, _ = positions(n, g, x0, dx, YEDGE)
    Xz, Yz, _ = positions(n, g, x0, dx, ZEDGE)
    Ay = np.broadcast_to(-(A0 * Bx / k) * np.cos(k * Xy), shape).copy()
    # A_z = -(A0 Bx / k) sin(kx) gives B^y = -dA_z/dx = A0 Bx cos kx; plus Bx*y for the uniform B^x
    Az = np.broadcast_to(-(A0 * Bx / k) * np.sin(k * Xz) + Bx * Yz, shape).copy()
    zero = _full(shape, 0.0)
    params = default_params(gamma=5.0 / 3.0, gamma_atm=5.0 / 3.0, rho_atm=1e-9, K_atm=1.0, recon=recon)
    metric = flat_metric(shape)
    bc = (BC_PERIODIC, BC_COPY, BC_COPY)
    return Workload("alfven_wave", n, g, x0, dx, bc, params, cfl * h, dict(rho=rho, press=press, velx=velx,
                    vely=vely, velz=velz), dict(Ax=zero.copy(), Ay=Ay, Az=Az), zero.copy(), metric)


def shock_tube(states: dict, nx: int, gamma: float, recon=RECON_PPM):
    """1D Riemann problem along x split at x = 0 on [-1/2, 1/2] (copy BCs), from a dict with keys rho, p, vx,
    vy, vz, Bx, By, Bz each holding (left, right) -- e.g. the Balsara states of Table 1.  The potential is
    piecewise linear: A_z = B^x y - B^y x, A_y = B^z x (per side), continuous at x = 0."""
    g = 3
    n = (nx, 1, 1)
    h = 1.0 / nx
    x0 = (-0.5, -0.5 * h, -0.5 * h)
    dx = (h, h, h)
    N = [m + 2 * g for m in n]
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    Xc, _, _ = positions(n, g, x0, dx, CELL)
    left = np.broadcast_to(Xc < 0.0, shape)
    side = lambda key: np.where(left, states[key][0], states[key][1]).astype(np.float64)
    prims = dict(rho=side("rho"), press=side("p"), velx=side("vx"), vely=side("vy"), velz=side("vz"))
    Bx = float(states["Bx"][0])
    Xz, Yz, _ = positions(n, g, x0, dx, ZEDGE)
    Xy, _, _ = positions(n, g, x0, dx, YEDGE)
    By = np.where(Xz < 0.0, states["By"][0], states["By"][1])
    Bz = np.where(Xy < 0.0, states["Bz"][0], states["Bz"][1])
    Az = np.broadcast_to(Bx * Yz - By * Xz, shape).copy()
    Ay = np.broadcast_to(Bz * Xy, shape).copy()
    zero = _full(shape, 0.0)
    params = default_params(gamma=gamma, gamma_atm=gamma, rho_atm=1e-9, K_atm=1.0, recon=recon)
    return Workload("shock_tube", n, g, x0, dx, (BC_COPY,) * 3, params, 0.25 * h, prims,
                    dict(Ax=zero.copy(), Ay=Ay, Az=Az), zero.copy(), flat_metric(shape))


def sub_block(w: Workload, lo, n, name=None) -> Workload:
    """The block of `n` interior cells starting at interior cell `lo` of `w` (same spacing, same data): every
    array is sliced in padded index space, ghosts included, and the BCs are kept."""
    g = w.g
    sl = tuple(slice(lo[d], lo[d] + n[d] + 2 * g + 1) for d in (2, 1, 0))
    cut = lambda a: np.ascontiguousarray(a[sl])
    x0 = tuple(w.x0[d] + lo[d] * w.dx[d] for d in range(3))
    return Workload(name or w.name + "_sub", tuple(int(v) for v in n), g, x0, w.dx, w.bc, dict(w.params), w.dt,
                    {k: cut(v) for k, v in w.prims.items()}, {k: cut(v) for k, v in w.A.items()}, cut(w.Psi),
                    {k: cut(v) for k, v in w.metric.items()})
