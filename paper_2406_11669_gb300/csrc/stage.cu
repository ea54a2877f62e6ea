// Kernels of one RK stage of the Valencia GRMHD right-hand side (AsterX, arXiv:2406.11669).
//
// Stage order (Sec. 3.9 workflow): ghost fill of U_s, B~ = curl A, recovery on the interior (Sec. 3.5),
// ghost fill of the primitives, then per direction: reconstruction of each cell once (Sec. 3.3) and the face
// solve (prim->cons, fluxes, magnetosonic speeds, HLLE, upwind transverse velocities of Eq. uct1); vertex
// potentials G_A and F_Psi (Sec. 3.4); edges: UCT electric field (Eq. eq3.20) and dA/dt = -E - grad G_A;
// vertices: dPsi/dt (Eq. recastedScalarPot); cells: flux divergence plus source terms (Eq. grmhdsrc, 3+1 form).
// Each of the last three writes either dU/dt or the RK4 stage update.
//
// Every intermediate lives in the workspace: the path is bound by FP64 arithmetic, not by HBM, so each
// quantity is computed once and re-read rather than recomputed.
#include <cstdio>

#include "kernels.h"
#include "physics.cuh"

namespace asterx {

static __host__ int grid_for(long count, int threads) {
  long blocks = (count + threads - 1) / threads;
  const long cap = 152L * 64;
  return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

#define GRID_LOOP(t, count) \
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (count); t += (long)gridDim.x * blockDim.x)

struct Box {
  int lo[3];
  int e[3];
  __host__ __device__ long count() const { return (long)e[0] * e[1] * e[2]; }
  __device__ __forceinline__ void at(long t, int& i, int& j, int& k) const {
    i = lo[0] + (int)(t % e[0]);
    const long r = t / e[0];
    j = lo[1] + (int)(r % e[1]);
    k = lo[2] + (int)(r / e[1]);
  }
};

__host__ __device__ inline Box make_box(int l0, int h0, int l1, int h1, int l2, int h2) {
  Box x;
  x.lo[0] = l0; x.lo[1] = l1; x.lo[2] = l2;
  x.e[0] = h0 - l0 + 1; x.e[1] = h1 - l1 + 1; x.e[2] = h2 - l2 + 1;
  return x;
}

__device__ __forceinline__ long lin(const Blk& b, int i, int j, int k) { return i + b.sy * j + b.sz * k; }
__device__ __forceinline__ long stride(const Blk& b, int d) { return d == 0 ? 1 : (d == 1 ? b.sy : b.sz); }

// ----------------------------------------------------------------------------------------------------------
// Ghost zones (Sec. 3.8): periodic wrap, or copy of the nearest owned value; the edge potential A is
// extrapolated linearly along the normal under copy BCs (when at least two owned layers exist).
// A field's owned index range along an axis is [g, g+n-1] if it is cell-like there (or periodic), [g, g+n]
// if it is vertex-like with copy BCs.  Sweeps run x, then y, then z, each over the full range of the others.

struct GhostSet {
  double* f[9];
  int cell_like[9];  // bit a set: cell-like along axis a
  int linear[9];
  int nf;
};

template <int AX>
__global__ void k_ghost(Blk b, GhostSet s) {
  constexpr int A1 = (AX + 1) % 3, A2 = (AX + 2) % 3;
  const int g = b.g, n = b.n[AX], Nn = b.N[AX];
  const long m1 = b.N[A1] + 1, m2 = b.N[A2] + 1;
  const int slots = 2 * g + 1;
  const long count = slots * m1 * m2;
  const long st = stride(b, AX);
  GRID_LOOP(t, count) {
    const int q = (int)(t % slots);
    const long r = t / slots;
    const int q1 = (int)(r % m1);
    const int q2 = (int)(r / m1);
    const int i = (q < g) ? q : Nn - 2 * g + q;
    int p[3];
    p[AX] = 0;
    p[A1] = q1;
    p[A2] = q2;
    const long base = lin(b, p[0], p[1], p[2]);
    for (int f = 0; f < s.nf; f++) {
      const bool cl = (s.cell_like[f] >> AX) & 1;
      const int lo = g;
      const int hi = (cl || b.bc[AX] == 0) ? g + n - 1 : g + n;
      if (i >= lo && i <= hi) continue;
      double* __restrict__ a = s.f[f] + base;
      double v;
      if (b.bc[AX] == 0) {
        const int src = lo + (((i - lo) % n) + n) % n;
        v = a[src * st];
      } else {
        const int e0 = (i < lo) ? lo : hi;
        const double f0 = a[e0 * st];
        if (s.linear[f] && hi > lo) {
          const int e1 = (i < lo) ? lo + 1 : hi - 1;
          const double f1 = a[e1 * st];
          v = __dadd_rn(f0, __dmul_rn((double)(i < lo ? lo - i : i - hi), __dsub_rn(f0, f1)));
        } else {
          v = f0;
        }
      }
      a[i * st] = v;
    }
  }
}

static const int STATE_CELL_LIKE[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};

cudaError_t launch_ghost_state(const Blk& b, const F9& U, cudaStream_t s) {
  GhostSet gs;
  for (int f = 0; f < 9; f++) {
    gs.f[f] = U.f[f];
    gs.cell_like[f] = STATE_CELL_LIKE[f];
    gs.linear[f] = (f >= 5 && f <= 7);
  }
  gs.nf = 9;
  const int T = 256;
  const int slots = 2 * b.g + 1;
  k_ghost<0><<<grid_for((long)slots * (b.N[1] + 1) * (b.N[2] + 1), T), T, 0, s>>>(b, gs);
  k_ghost<1><<<grid_for((long)slots * (b.N[2] + 1) * (b.N[0] + 1), T), T, 0, s>>>(b, gs);
  k_ghost<2><<<grid_for((long)slots * (b.N[0] + 1) * (b.N[1] + 1), T), T, 0, s>>>(b, gs);
  return cudaGetLastError();
}

cudaError_t launch_ghost_prims(const Blk& b, const F5& P, cudaStream_t s) {
  GhostSet gs;
  for (int f = 0; f < 5; f++) {
    gs.f[f] = P.f[f];
    gs.cell_like[f] = 7;
    gs.linear[f] = 0;
  }
  gs.nf = 5;
  const int T = 256;
  const int slots = 2 * b.g + 1;
  k_ghost<0><<<grid_for((long)slots * (b.N[1] + 1) * (b.N[2] + 1), T), T, 0, s>>>(b, gs);
  k_ghost<1><<<grid_for((long)slots * (b.N[2] + 1) * (b.N[0] + 1), T), T, 0, s>>>(b, gs);
  k_ghost<2><<<grid_for((long)slots * (b.N[0] + 1) * (b.N[1] + 1), T), T, 0, s>>>(b, gs);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------------------------
// B~^i = [ijk] d_j A_k on faces (Eq. BEulerian, second-order differences of the edge values), then the
// undensitised centre field B^i = (B~^i_- + B~^i_+) / (2 sqrt(gamma_c)) (Sec. 3.1).

__global__ void k_bface(Blk b, const double* __restrict__ Ax, const double* __restrict__ Ay,
                        const double* __restrict__ Az, double* __restrict__ bf) {
  Box box = make_box(0, b.N[0], 0, b.N[1], 0, b.N[2]);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    // rounded operations without contraction: the face field is reproduced exactly by other implementations
    // of the same differences, so decisions taken downstream see identical inputs
    if (j < b.N[1] && k < b.N[2])
      bf[c] = __dsub_rn(__dmul_rn(__dsub_rn(Az[c + b.sy], Az[c]), b.idx[1]),
                        __dmul_rn(__dsub_rn(Ay[c + b.sz], Ay[c]), b.idx[2]));
    if (i < b.N[0] && k < b.N[2])
      bf[b.V + c] = __dsub_rn(__dmul_rn(__dsub_rn(Ax[c + b.sz], Ax[c]), b.idx[2]),
                              __dmul_rn(__dsub_rn(Az[c + 1], Az[c]), b.idx[0]));
    if (i < b.N[0] && j < b.N[1])
      bf[2 * b.V + c] = __dsub_rn(__dmul_rn(__dsub_rn(Ay[c + 1], Ay[c]), b.idx[0]),
                                  __dmul_rn(__dsub_rn(Ax[c + b.sy], Ax[c]), b.idx[1]));
  }
}

__global__ void k_bcentre(Blk b, const double* __restrict__ bf, const double* __restrict__ cg,
                          double* __restrict__ bc) {
  Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    const double sqg = cg[CG_SQG * b.V + c];
    bc[c] = 0.5 * (bf[c] + bf[c + 1]) / sqg;
    bc[b.V + c] = 0.5 * (bf[b.V + c] + bf[b.V + c + b.sy]) / sqg;
    bc[2 * b.V + c] = 0.5 * (bf[2 * b.V + c] + bf[2 * b.V + c + b.sz]) / sqg;
  }
}

cudaError_t launch_bfield(const Blk& b, const Ws& w, const F9& U, cudaStream_t s) {
  const int T = 256;
  k_bface<<<grid_for(b.V, T), T, 0, s>>>(b, U.f[5], U.f[6], U.f[7], w.bf);
  k_bcentre<<<grid_for((long)b.N[0] * b.N[1] * b.N[2], T), T, 0, s>>>(b, w.bf, w.cg, w.bc);
  return cudaGetLastError();
}

__device__ __forceinline__ void load_geo_centre(const Blk& b, const double* __restrict__ cg, long c, Geo& m) {
  m.alp = cg[CG_ALP * b.V + c];
  for (int a = 0; a < 3; a++) m.beta[a] = cg[(CG_BETA + a) * b.V + c];
  for (int a = 0; a < 6; a++) {
    m.g[a] = cg[(CG_G + a) * b.V + c];
    m.gu[a] = cg[(CG_GU + a) * b.V + c];
  }
  m.sqg = cg[CG_SQG * b.V + c];
}

// ----------------------------------------------------------------------------------------------------------
// Conserved variables from primitives at every cell (initial data, Eq. cons).

__global__ void k_prim2con(Blk b, Ws w, F9 U, F5 P, double gamma, double gfac) {
  Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    Geo m;
    load_geo_centre(b, w.cg, c, m);
    const double v[3] = {P.f[2][c], P.f[3][c], P.f[4][c]};
    const double W = 1.0 / sqrt(1.0 - contract_sym(m.g, v, v));
    const double u[3] = {W * v[0], W * v[1], W * v[2]};
    const double B[3] = {w.bc[c], w.bc[b.V + c], w.bc[2 * b.V + c]};
    SideOut o;
    face_side(m, 1.0 / m.alp, 0, P.f[0][c], P.f[1][c], u, B, gamma, gfac, o);
    for (int a = 0; a < 5; a++) U.f[a][c] = o.U[a];
  }
}

cudaError_t launch_prim2con(const StageArgs& a, const F9& U, const F5& P, cudaStream_t s) {
  const int T = 128;
  k_prim2con<<<grid_for((long)a.b.N[0] * a.b.N[1] * a.b.N[2], T), T, 0, s>>>(a.b, a.w, U, P, a.gamma,
                                                                               a.gfac);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------------------------
// Primitive recovery on interior cells (Sec. 3.5, 3.6): atmosphere if D~ < sqrt(gamma) rho_atm, else Noble 2D
// seeded by the previous primitives, Palenzuela 1D fallback, atmosphere with flag -1 if both fail.

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_c2p(Blk b, Ws w, F9 U, F5 P, C2PParams cp, signed char* __restrict__ flags,
                      unsigned long long* __restrict__ stats) {
  Box box = make_box(b.g, b.g + b.n[0] - 1, b.g, b.g + b.n[1] - 1, b.g, b.g + b.n[2] - 1);
  const long count = box.count();
  // the grid-stride loop is padded to whole warps so that the counter reduction sees full warps
  const long padded = (count + 31) / 32 * 32;
  GRID_LOOP(t, padded) {
    unsigned long long c_noble = 0, c_fb = 0, c_atm = 0, c_fail = 0, c_it = 0;
    if (t < count) {
      int i, j, k;
      box.at(t, i, j, k);
      const long c = lin(b, i, j, k);
      Geo m;
      load_geo_centre(b, w.cg, c, m);
      const double Dt = U.f[0][c];
      const double B[3] = {w.bc[c], w.bc[b.V + c], w.bc[2 * b.V + c]};
      C2PResult r;
      r.iters = 0;
      bool ok = false;
      bool atm = !(Dt >= m.sqg * cp.rho_atm);
      int flag = 2;
      if (!atm) {
        const double D = Dt / m.sqg;
        const double S[3] = {U.f[1][c] / m.sqg, U.f[2][c] / m.sqg, U.f[3][c] / m.sqg};
        const double tau = U.f[4][c] / m.sqg;
        double Bl[3];
        lower(m.g, B, Bl);
        const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
        const double S2 = contract_sym(m.gu, S, S);
        const double BS = B[0] * S[0] + B[1] * S[1] + B[2] * S[2];
        // initial guess from the previous primitives
        const double grho = P.f[0][c], gp = P.f[1][c];
        const double gv[3] = {P.f[2][c], P.f[3][c], P.f[4][c]};
        const double v2max = 1.0 - 1.0 / (cp.W_max * cp.W_max);
        double gv2 = contract_sym(m.g, gv, gv);
        if (!(gv2 >= 0.0)) gv2 = 0.0;
        if (gv2 > v2max) gv2 = v2max;
        const double gW = 1.0 / sqrt(1.0 - gv2);
        const double geps = gp / ((cp.gamma - 1.0) * grho);
        const double gh = 1.0 + geps + gp / grho;
        const double z0 = grho * gh * gW * gW;
        if (z0 > 0.0 && isfinite(z0)) ok = c2p_noble(m, D, S, tau, B, S2, B2, BS, z0, gv2, cp, r);
        flag = 0;
        if (!ok && cp.use_fallback) {
          ok = c2p_palenzuela(m, D, S, tau, B, S2, B2, BS, cp, r);
          flag = 1;
        }
        if (!ok) {
          flag = -1;
          atm = true;
        }
      }
      if (atm) {
        r.rho = cp.rho_atm;
        r.press = cp.K_atm * pow(cp.rho_atm, cp.gamma_atm);
        r.v[0] = r.v[1] = r.v[2] = 0.0;
        // conserved variables of the atmosphere state (v = 0, W = 1, b^2 = B^2), field kept (Sec. 3.6)
        double Bl[3];
        lower(m.g, B, Bl);
        const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
        U.f[0][c] = m.sqg * r.rho;
        U.f[1][c] = 0.0;
        U.f[2][c] = 0.0;
        U.f[3][c] = 0.0;
        U.f[4][c] = m.sqg * (r.press / (cp.gamma_atm - 1.0) + 0.5 * B2);
      }
      P.f[0][c] = r.rho;
      P.f[1][c] = r.press;
      P.f[2][c] = r.v[0];
      P.f[3][c] = r.v[1];
      P.f[4][c] = r.v[2];
      if (flags) flags[c] = (signed char)flag;
      c_it = r.iters;
      if (flag == 0) c_noble = 1;
      else if (flag == 1) c_fb = 1;
      else if (flag == 2) c_atm = 1;
      else c_fail = 1;
    }
    if (stats) {
      c_noble = warp_sum(c_noble);
      c_fb = warp_sum(c_fb);
      c_atm = warp_sum(c_atm);
      c_fail = warp_sum(c_fail);
      c_it = warp_sum(c_it);
      if ((threadIdx.x & 31) == 0) {
        if (c_noble) atomicAdd(stats + 0, c_noble);
        if (c_fb) atomicAdd(stats + 1, c_fb);
        if (c_atm) atomicAdd(stats + 2, c_atm);
        if (c_fail) atomicAdd(stats + 3, c_fail);
        if (c_it) atomicAdd(stats + 4, c_it);
      }
    }
  }
}

cudaError_t launch_c2p(const StageArgs& a, const F9& U, const F5& P, signed char* flags,
                       unsigned long long* stats, cudaStream_t s) {
  C2PParams cp;
  cp.gamma = a.gamma;
  cp.rho_atm = a.rho_atm;
  cp.K_atm = a.K_atm;
  cp.gamma_atm = a.gamma_atm;
  cp.tol = a.c2p_tol;
  cp.W_max = a.W_max;
  cp.maxiter = a.c2p_maxiter;
  cp.brent_maxiter = a.brent_maxiter;
  cp.use_fallback = a.use_fallback;
  const int T = 128;  // a multiple of 32: whole warps take part in the counter reduction
  const long count = (long)a.b.n[0] * a.b.n[1] * a.b.n[2];
  k_c2p<<<grid_for(count, T), T, 0, s>>>(a.b, a.w, U, P, cp, flags, stats);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------------------------
// u^i = W v^i at every cell (the reconstructed velocity variable).

__global__ void k_uvel(Blk b, Ws w, F5 P) {
  Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    double g6[6];
    for (int a = 0; a < 6; a++) g6[a] = w.cg[(CG_G + a) * b.V + c];
    const double v[3] = {P.f[2][c], P.f[3][c], P.f[4][c]};
    const double W = 1.0 / sqrt(1.0 - contract_sym(g6, v, v));
    w.uvel[c] = W * v[0];
    w.uvel[b.V + c] = W * v[1];
    w.uvel[2 * b.V + c] = W * v[2];
  }
}

// ----------------------------------------------------------------------------------------------------------
// Reconstruction along D of each cell once (cells g-1 .. g+n along D, all transverse cells): the values at the
// cell's lower and upper D-faces of rho, p, u^x, u^y, u^z and the two transverse centre B components.

template <int D, int SCHEME>
__global__ void k_recon(Blk b, Ws w, F5 P) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  int lo[3] = {0, 0, 0}, hi[3] = {b.N[0] - 1, b.N[1] - 1, b.N[2] - 1};
  lo[D] = b.g - 1;
  hi[D] = b.g + b.n[D];
  Box box = make_box(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
  const long st = stride(b, D);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    const double* src[NREC] = {P.f[0], P.f[1], w.uvel, w.uvel + b.V, w.uvel + 2 * b.V, w.bc + T1 * b.V,
                               w.bc + T2 * b.V};
#pragma unroll
    for (int v = 0; v < NREC; v++) {
      double a[5];
#pragma unroll
      for (int s = 0; s < 5; s++) a[s] = src[v][c + (s - 2) * st];
      double l, h;
      recon5<SCHEME>(a, l, h);
      w.rec[v * b.V + c] = l;
      w.rec[(NREC + v) * b.V + c] = h;
    }
  }
}

// Face solve along D for faces g..g+n along D and all transverse indices: left state = upper value of cell
// f-1, right state = lower value of cell f; HLLE (Eq. HLLEfluxes) and the upwind velocities of Eq. uct1.
template <int D>
__global__ void __launch_bounds__(128) k_faces(Blk b, Ws w, double gamma, double gfac) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  int lo[3] = {0, 0, 0}, hi[3] = {b.N[0] - 1, b.N[1] - 1, b.N[2] - 1};
  lo[D] = b.g;
  hi[D] = b.g + b.n[D];
  Box box = make_box(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
  const long st = stride(b, D);
  const double* __restrict__ fg = w.fg + (long)D * NFG * b.V;
  double* __restrict__ fd = w.face + (long)D * NFD * b.V;
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    Geo m;
    m.alp = fg[FG_ALP * b.V + c];
    for (int a = 0; a < 3; a++) m.beta[a] = fg[(FG_BETA + a) * b.V + c];
    for (int a = 0; a < 6; a++) {
      m.g[a] = fg[(FG_G + a) * b.V + c];
      m.gu[a] = fg[(FG_GU + a) * b.V + c];
    }
    m.sqg = fg[FG_SQG * b.V + c];
    const double ia = fg[FG_IALP * b.V + c];
    const double Bn = w.bf[D * b.V + c] / m.sqg;
    SideOut s[2];
#pragma unroll
    for (int side = 0; side < 2; side++) {
      const long cc = side == 0 ? c - st : c;
      const double* __restrict__ r = w.rec + (side == 0 ? NREC : 0) * b.V + cc;
      const double u[3] = {r[2 * b.V], r[3 * b.V], r[4 * b.V]};
      double B[3];
      B[D] = Bn;
      B[T1] = r[5 * b.V];
      B[T2] = r[6 * b.V];
      face_side(m, ia, D, r[0], r[b.V], u, B, gamma, gfac, s[side]);
    }
    const double cmax = fmax(0.0, fmax(s[0].lp, s[1].lp));
    const double cmin = -fmin(0.0, fmin(s[0].lm, s[1].lm));
    const double den = cmax + cmin;
    if (den > 0.0) {
      const double iden = 1.0 / den;
      for (int v = 0; v < 5; v++)
        fd[(FD_F + v) * b.V + c] =
            (cmin * s[1].F[v] + cmax * s[0].F[v] - cmax * cmin * (s[1].U[v] - s[0].U[v])) * iden;
      fd[FD_VB1 * b.V + c] = (cmax * s[0].vt[T1] + cmin * s[1].vt[T1]) * iden;
      fd[FD_VB2 * b.V + c] = (cmax * s[0].vt[T2] + cmin * s[1].vt[T2]) * iden;
    } else {
      for (int v = 0; v < 5; v++) fd[(FD_F + v) * b.V + c] = 0.5 * (s[0].F[v] + s[1].F[v]);
      fd[FD_VB1 * b.V + c] = 0.5 * (s[0].vt[T1] + s[1].vt[T1]);
      fd[FD_VB2 * b.V + c] = 0.5 * (s[0].vt[T2] + s[1].vt[T2]);
    }
    fd[FD_CMAX * b.V + c] = cmax;
    fd[FD_CMIN * b.V + c] = cmin;
  }
}

// ----------------------------------------------------------------------------------------------------------
// RK4 combine (classical): stage < 0 writes dU/dt.

__device__ __forceinline__ void combine(int stage, double dt, long c, int v, double k, const F9& Un,
                                        const F9& Unext, const F9& Uacc, const F9& dU) {
  if (stage < 0) {
    dU.f[v][c] = k;
  } else if (stage == 0) {
    Uacc.f[v][c] = (1.0 / 6.0) * dt * k;
    Unext.f[v][c] = Un.f[v][c] + 0.5 * dt * k;
  } else if (stage == 1) {
    Uacc.f[v][c] = Uacc.f[v][c] + (1.0 / 3.0) * dt * k;
    Unext.f[v][c] = Un.f[v][c] + 0.5 * dt * k;
  } else if (stage == 2) {
    Uacc.f[v][c] = Uacc.f[v][c] + (1.0 / 3.0) * dt * k;
    Unext.f[v][c] = Un.f[v][c] + 1.0 * dt * k;
  } else {
    Unext.f[v][c] = Un.f[v][c] + Uacc.f[v][c] + (1.0 / 6.0) * dt * k;
  }
}

// G_A = alpha Psi / sqrt(gamma) - beta^j A_j and F_Psi^j = alpha sqrt(gamma) gamma^jk A_k - beta^j Psi at
// vertices, with A_j averaged from the two adjacent j-edges (Sec. 3.4).
__global__ void k_vertex(Blk b, Ws w, F9 U, int lorenz) {
  Box box = make_box(b.g - 1, b.g + b.n[0] + 1, b.g - 1, b.g + b.n[1] + 1, b.g - 1, b.g + b.n[2] + 1);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    const double Av[3] = {0.5 * (U.f[5][c - 1] + U.f[5][c]), 0.5 * (U.f[6][c - b.sy] + U.f[6][c]),
                          0.5 * (U.f[7][c - b.sz] + U.f[7][c])};
    const double alp = w.vg[VG_ALP * b.V + c];
    const double bx = w.vg[(VG_BETA + 0) * b.V + c], by = w.vg[(VG_BETA + 1) * b.V + c],
                 bz = w.vg[(VG_BETA + 2) * b.V + c];
    const double sqg = w.vg[VG_SQG * b.V + c];
    double gu[6];
    for (int a = 0; a < 6; a++) gu[a] = w.vg[(VG_GU + a) * b.V + c];
    const double psi = U.f[8][c];
    const double bA = bx * Av[0] + by * Av[1] + bz * Av[2];
    w.ga[c] = lorenz ? (alp * psi / sqg - bA) : 0.0;
    const double as = alp * sqg;
    w.fpsi[c] = as * (gu[0] * Av[0] + gu[1] * Av[1] + gu[2] * Av[2]) - bx * psi;
    w.fpsi[b.V + c] = as * (gu[1] * Av[0] + gu[3] * Av[1] + gu[4] * Av[2]) - by * psi;
    w.fpsi[2 * b.V + c] = as * (gu[2] * Av[0] + gu[4] * Av[1] + gu[5] * Av[2]) - bz * psi;
  }
}

// PPM value at the interface between stencil positions 2 and 3 of f[0..5]
__device__ __forceinline__ void ppm_interface(const double f[6], double& L, double& R) {
  double l, h;
  recon5<1>(f, l, h);
  L = h;
  recon5<1>(f + 1, l, h);
  R = l;
}

// Edges along E (owned range): UCT electric field (Sec. 3.4, Eqs. uct1, uct2, eq3.20) with (E, d1, d2) cyclic,
//   E_E = -HLL_d1(v~^d1 B~^d2) + HLL_d2(v~^d2 B~^d1),
// products reconstructed with PPM to the edge from the faces normal to d2 (resp. d1), speeds a_+- at the edge
// the maximum over the two faces sharing it; then dA_E/dt = -E_E - d_E G_A.
template <int E>
__global__ void __launch_bounds__(128) k_edges(Blk b, Ws w, int stage, double dt, F9 Un, F9 Unext, F9 Uacc,
                                                 F9 dU) {
  constexpr int D1 = (E + 1) % 3, D2 = (E + 2) % 3;
  int lo[3] = {b.g, b.g, b.g}, hi[3] = {b.g + b.n[0], b.g + b.n[1], b.g + b.n[2]};
  hi[E] -= 1;
  Box box = make_box(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    double term[2];
#pragma unroll
    for (int tt = 0; tt < 2; tt++) {
      const int dr = tt == 0 ? D1 : D2;  // reconstruction / upwind direction
      const int df = tt == 0 ? D2 : D1;  // normal of the faces carrying v~^dr and B~^df
      const long sr = stride(b, dr);
      const long sf = stride(b, df);
      // component dr on df-faces: slot VB1 holds component (df+1)%3, VB2 holds (df+2)%3
      const int slot = (((df + 1) % 3) == dr) ? FD_VB1 : FD_VB2;
      const double* __restrict__ vb = w.face + ((long)df * NFD + slot) * b.V;
      const double* __restrict__ bn = w.bf + (long)df * b.V;
      double vs[6], bs[6];
#pragma unroll
      for (int s = 0; s < 6; s++) {
        const long q = c + (s - 3) * sr;
        vs[s] = vb[q];
        bs[s] = bn[q];
      }
      double vL, vR, BL, BR;
      ppm_interface(vs, vL, vR);
      ppm_interface(bs, BL, BR);
      const double* __restrict__ fdr = w.face + (long)dr * NFD * b.V;
      const long c0 = c - sf;
      const double ap = fmax(fdr[FD_CMAX * b.V + c0], fdr[FD_CMAX * b.V + c]);
      const double am = fmax(fdr[FD_CMIN * b.V + c0], fdr[FD_CMIN * b.V + c]);
      const double den = ap + am;
      term[tt] = (den > 0.0) ? (ap * vL * BL + am * vR * BR - ap * am * (BR - BL)) / den : 0.5 * (vL * BL + vR * BR);
    }
    const double Ee = -term[0] + term[1];
    const double dG = (w.ga[c + stride(b, E)] - w.ga[c]) / b.dx[E];
    combine(stage, dt, c, 5 + E, -Ee - dG, Un, Unext, Uacc, dU);
  }
}

// dPsi/dt = -d_j F_Psi^j - xi alpha Psi at vertices g..g+n (Eq. recastedScalarPot).
__global__ void k_psi(Blk b, Ws w, F9 Us, int lorenz, double xi, int stage, double dt, F9 Un, F9 Unext, F9 Uacc,
                      F9 dU) {
  Box box = make_box(b.g, b.g + b.n[0], b.g, b.g + b.n[1], b.g, b.g + b.n[2]);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    double r = 0.0;
    if (lorenz) {
      const double div = (w.fpsi[c + 1] - w.fpsi[c - 1]) / (2.0 * b.dx[0]) +
                         (w.fpsi[b.V + c + b.sy] - w.fpsi[b.V + c - b.sy]) / (2.0 * b.dx[1]) +
                         (w.fpsi[2 * b.V + c + b.sz] - w.fpsi[2 * b.V + c - b.sz]) / (2.0 * b.dx[2]);
      r = -div - xi * w.vg[VG_ALP * b.V + c] * Us.f[8][c];
    }
    combine(stage, dt, c, 8, r, Un, Unext, Uacc, dU);
  }
}

// Source terms (Eq. grmhdsrc in 3+1 form with the input K_ij, K = -1/2 L_n gamma of Sec. 2.1):
//   tau~: alpha sqrt(g) [T^00 (b^i b^j K_ij - b^i d_i alpha) + T^0i (2 b^j K_ij - d_i alpha) + T^ij K_ij]
//   S~_i: alpha sqrt(g) [-T^00 alpha d_i alpha + T^0_k d_i b^k + 1/2 (T^00 b^j b^k + 2 T^0j b^k + T^jk) d_i g_jk]
// (b = beta) with T^{mu nu} = (rho h + b^2) u u + (p + b^2/2) g^{mu nu} - b b (Eq. tmunu).
__device__ __forceinline__ void sources(const Geo& m, const double* __restrict__ cg, long V, long c, double rho,
                                        double press, const double v[3], const double B[3], double gfac,
                                        double src[5]) {
  double vl[3], Bl[3];
  lower(m.g, v, vl);
  lower(m.g, B, Bl);
  const double W = 1.0 / sqrt(1.0 - (v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2]));
  const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const double Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const double ia = 1.0 / m.alp;
  const double iW = 1.0 / W;
  const double b2 = B2 * iW * iW + Bv * Bv;
  const double rhoh = rho + gfac * press;
  const double e = rhoh + b2;
  const double pt = press + 0.5 * b2;
  double u[4], bb[4];
  u[0] = W * ia;
  bb[0] = W * Bv * ia;
  for (int a = 0; a < 3; a++) {
    u[1 + a] = W * (v[a] - m.beta[a] * ia);
    bb[1 + a] = (B[a] + m.alp * bb[0] * u[1 + a]) * iW;
  }
  const double ia2 = ia * ia;
  const double T00 = e * u[0] * u[0] - pt * ia2 - bb[0] * bb[0];
  double T0[3], T[6];
  for (int a = 0; a < 3; a++) T0[a] = e * u[0] * u[1 + a] + pt * m.beta[a] * ia2 - bb[0] * bb[1 + a];
  for (int a = 0; a < 3; a++)
    for (int q = a; q < 3; q++)
      T[sym(a, q)] = e * u[1 + a] * u[1 + q] + pt * (m.gu[sym(a, q)] - m.beta[a] * m.beta[q] * ia2) -
                     bb[1 + a] * bb[1 + q];
  double K[6], dalp[3];
  for (int a = 0; a < 6; a++) K[a] = cg[(CG_K + a) * V + c];
  for (int a = 0; a < 3; a++) dalp[a] = cg[(CG_DALP + a) * V + c];
  double betal[3];
  lower(m.g, m.beta, betal);
  const double asg = m.alp * m.sqg;
  // energy
  double Kb[3];  // K_ij beta^j
  for (int a = 0; a < 3; a++) Kb[a] = K[sym(a, 0)] * m.beta[0] + K[sym(a, 1)] * m.beta[1] + K[sym(a, 2)] * m.beta[2];
  double st = T00 * (m.beta[0] * Kb[0] + m.beta[1] * Kb[1] + m.beta[2] * Kb[2]);
  for (int a = 0; a < 3; a++) st += -T00 * m.beta[a] * dalp[a] + T0[a] * (2.0 * Kb[a] - dalp[a]);
  st += T[0] * K[0] + T[3] * K[3] + T[5] * K[5] + 2.0 * (T[1] * K[1] + T[2] * K[2] + T[4] * K[4]);
  src[0] = 0.0;
  src[4] = asg * st;
  // momentum
  double T0l[3];
  for (int q = 0; q < 3; q++)
    T0l[q] = betal[q] * T00 + m.g[sym(q, 0)] * T0[0] + m.g[sym(q, 1)] * T0[1] + m.g[sym(q, 2)] * T0[2];
  double M[6];  // T^00 b^j b^k + T^0j b^k + T^0k b^j + T^jk (symmetrised)
  for (int a = 0; a < 3; a++)
    for (int q = a; q < 3; q++)
      M[sym(a, q)] = T00 * m.beta[a] * m.beta[q] + T0[a] * m.beta[q] + T0[q] * m.beta[a] + T[sym(a, q)];
  for (int i = 0; i < 3; i++) {
    double s = -T00 * m.alp * dalp[i];
    for (int q = 0; q < 3; q++) s += T0l[q] * cg[(CG_DBETA + i * 3 + q) * V + c];
    const double* dg = cg + (CG_DG + i * 6) * V + c;
    s += 0.5 * (M[0] * dg[0] + M[3] * dg[3 * V] + M[5] * dg[5 * V]) + M[1] * dg[V] + M[2] * dg[2 * V] +
         M[4] * dg[4 * V];
    src[1 + i] = asg * s;
  }
}

// Interior cells: dU/dt = -sum_d (F_d(+) - F_d(-)) / dx_d + S (Eq. fluxconseqs, densitised).
__global__ void __launch_bounds__(128) k_cells(Blk b, Ws w, F5 P, double gfac, int stage, double dt, F9 Un,
                                                 F9 Unext, F9 Uacc, F9 dU) {
  Box box = make_box(b.g, b.g + b.n[0] - 1, b.g, b.g + b.n[1] - 1, b.g, b.g + b.n[2] - 1);
  GRID_LOOP(t, box.count()) {
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    double r[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double* __restrict__ fd = w.face + (long)d * NFD * b.V;
      const long c1 = c + stride(b, d);
#pragma unroll
      for (int v = 0; v < 5; v++) r[v] -= (fd[(FD_F + v) * b.V + c1] - fd[(FD_F + v) * b.V + c]) / b.dx[d];
    }
    Geo m;
    load_geo_centre(b, w.cg, c, m);
    const double v[3] = {P.f[2][c], P.f[3][c], P.f[4][c]};
    const double B[3] = {w.bc[c], w.bc[b.V + c], w.bc[2 * b.V + c]};
    double src[5];
    sources(m, w.cg, b.V, c, P.f[0][c], P.f[1][c], v, B, gfac, src);
#pragma unroll
    for (int q = 0; q < 5; q++) combine(stage, dt, c, q, r[q] + src[q], Un, Unext, Uacc, dU);
  }
}

// Measurement hook: when enabled, an event pair brackets every face-kernel launch on its own stream.
namespace {
struct FaceProfile {
  bool on = false;
  int cap = 0;
  int n = 0;
  cudaEvent_t* ev = nullptr;  // 2 * cap events
};
FaceProfile g_prof;
}  // namespace

cudaError_t profile_enable(int cap) {
  profile_disable();
  g_prof.ev = new cudaEvent_t[2 * (size_t)cap];
  for (int i = 0; i < 2 * cap; i++) {
    cudaError_t e = cudaEventCreate(&g_prof.ev[i]);
    if (e != cudaSuccess) {
      for (int q = 0; q < i; q++) cudaEventDestroy(g_prof.ev[q]);
      delete[] g_prof.ev;
      g_prof.ev = nullptr;
      return e;
    }
  }
  g_prof.cap = cap;
  g_prof.n = 0;
  g_prof.on = true;
  return cudaSuccess;
}

void profile_disable() {
  if (g_prof.ev) {
    for (int i = 0; i < 2 * g_prof.cap; i++) cudaEventDestroy(g_prof.ev[i]);
    delete[] g_prof.ev;
  }
  g_prof = FaceProfile();
}

cudaError_t profile_read(int* launches, double* total_ms) {
  double tot = 0.0;
  for (int i = 0; i < g_prof.n; i++) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(g_prof.ev[2 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    tot += ms;
  }
  *launches = g_prof.n;
  *total_ms = tot;
  return cudaSuccess;
}

template <int D>
static void launch_dir(const StageArgs& a, const F5& P, cudaStream_t s) {
  const Blk& b = a.b;
  long rc = (long)b.N[0] * b.N[1] * b.N[2] / b.N[D] * (b.n[D] + 2);
  const int T = 128;
  if (a.recon == 0) k_recon<D, 0><<<grid_for(rc, T), T, 0, s>>>(b, a.w, P);
  else if (a.recon == 1) k_recon<D, 1><<<grid_for(rc, T), T, 0, s>>>(b, a.w, P);
  else k_recon<D, 2><<<grid_for(rc, T), T, 0, s>>>(b, a.w, P);
  long fc = (long)b.N[0] * b.N[1] * b.N[2] / b.N[D] * (b.n[D] + 1);
  const bool mark = g_prof.on && g_prof.n < g_prof.cap;
  if (mark) cudaEventRecord(g_prof.ev[2 * g_prof.n], s);
  k_faces<D><<<grid_for(fc, T), T, 0, s>>>(b, a.w, a.gamma, a.gfac);
  if (mark) cudaEventRecord(g_prof.ev[2 * g_prof.n++ + 1], s);
}

cudaError_t launch_rhs(const StageArgs& a, const F9& Us, const F5& P, int stage, double dt, const F9& Un,
                       const F9& Unext, const F9& Uacc, const F9& dU, cudaStream_t s) {
  const Blk& b = a.b;
  const int T = 128;
  k_uvel<<<grid_for((long)b.N[0] * b.N[1] * b.N[2], T), T, 0, s>>>(b, a.w, P);
  launch_dir<0>(a, P, s);
  launch_dir<1>(a, P, s);
  launch_dir<2>(a, P, s);
  const int lorenz = (a.gauge == 0);
  k_vertex<<<grid_for((long)(b.n[0] + 3) * (b.n[1] + 3) * (b.n[2] + 3), T), T, 0, s>>>(b, a.w, Us, lorenz);
  const long ec = (long)(b.n[0] + 1) * (b.n[1] + 1) * (b.n[2] + 1);
  k_edges<0><<<grid_for(ec, T), T, 0, s>>>(b, a.w, stage, dt, Un, Unext, Uacc, dU);
  k_edges<1><<<grid_for(ec, T), T, 0, s>>>(b, a.w, stage, dt, Un, Unext, Uacc, dU);
  k_edges<2><<<grid_for(ec, T), T, 0, s>>>(b, a.w, stage, dt, Un, Unext, Uacc, dU);
  const double xi = a.xi > 0.0 ? a.xi : 1.5 / dt;
  k_psi<<<grid_for(ec, T), T, 0, s>>>(b, a.w, Us, lorenz, xi, stage, dt, Un, Unext, Uacc, dU);
  k_cells<<<grid_for((long)b.n[0] * b.n[1] * b.n[2], T), T, 0, s>>>(b, a.w, P, a.gfac, stage, dt, Un, Unext,
                                                                     Uacc, dU);
  return cudaGetLastError();
}

}  // namespace asterx
