// Kernels of one RK stage of the Valencia GRMHD right-hand side (AsterX, arXiv:2406.11669).
//
// Stage order (Sec. 3.12 workflow): ghost fill of U_s, B~ = curl A, recovery on the interior (Sec. 3.5),
// ghost fill of the primitives, then per direction: reconstruction of each cell once (Sec. 3.3) and the face
// solve (prim->cons, fluxes, magnetosonic speeds, HLLE, upwind transverse velocities of Eq. uct1); vertex
// potentials G_A and F_Psi (Sec. 3.4); edges: UCT electric field (Eq. eq3.20) and dA/dt = -E - grad G_A;
// vertices: dPsi/dt (Eq. recastedScalarPot); cells: flux divergence plus source terms (Eq. grmhdsrc, 3+1 form).
// Each of the last three writes either dU/dt or the RK4 stage update.
//
// Every intermediate lives in the workspace: the path is bound by FP64 arithmetic, not by HBM, so each
// quantity is computed once and re-read rather than recomputed.
//
// Each kernel body is a functor run(record, consts, t) over the block's own item space (t = 0 .. count-1).
// A single-block launch loops over one record's items; a batched launch loops over the items of every block
// of a device table (block found by binary search over the per-kind prefix offsets), so both run the same code.
#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "physics.cuh"

#include <cstdlib>
#include <mutex>
#include <vector>

namespace asterx {

static __host__ int grid_for(long count, int threads) {
  long blocks = (count + threads - 1) / threads;
  const long cap = 64L * device_sm_count();
  return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

#define GRID_LOOP(t, count) \
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (count); t += (long)gridDim.x * blockDim.x)

struct Box {
  int lo[3];
  int e[3];
  __host__ __device__ long count() const { return (long)e[0] * e[1] * e[2]; }
  __device__ __forceinline__ void at(long t, int& i, int& j, int& k) const {
    unflatten3(t, (unsigned)e[0], (unsigned)e[1], i, j, k);
    i += lo[0];
    j += lo[1];
    k += lo[2];
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

// Constants shared by every block of one launch.
struct StageConsts {
  double gamma, gfac, dt, xi;
  int stage, lorenz;
  int lxf, fct;  // Lax-Friedrichs fluxes; flux constrained transport
  C2PParams cp;
  unsigned long long* stats;
  const BlockRec* tab;  // tiled batch: this stage's block records (device), else null
  const Tiling* til;    // tiled batch: the tiling (device), else null
  int chunk;            // cells per item of the chunked kernels (set per launch)
};

// ----------------------------------------------------------------------------------------------------------
// Launch machinery: one record by value, or a device table of records with per-kind prefix offsets.

template <class Body>
__global__ void __launch_bounds__(128) k_single(BlockRec r, StageConsts k, long count) {
  GRID_LOOP(t, count) Body::run(r, k, t);
}

__device__ __forceinline__ int find_block(const long* __restrict__ off, int nb, long T) {
  int lo = 0, hi = nb;  // largest lo with off[lo] <= T
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= T) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <class Body>
__global__ void __launch_bounds__(128) k_batch(const BlockRec* __restrict__ tab, const long* __restrict__ off,
                                                 int nb, StageConsts k) {
  const long total = off[nb];
  GRID_LOOP(T, total) {
    const int blk = find_block(off, nb, T);
    Body::run(tab[blk], k, T - off[blk]);
  }
}

struct Single {
  BlockRec r;
  long count(int kind) const { return kind_count(kind, r.b); }
};

struct Batch {
  const BlockRec* tab;     // device, nb records of this stage
  const long* off;         // device, NKIND * (nb + 1) offsets
  const long* host_total;  // host, NKIND totals
  int nb;
  long count(int kind) const { return host_total[kind]; }
};

// ----------------------------------------------------------------------------------------------------------
// Launch-configuration autotuner.  Every work item is independent of the launch shape (grid-stride loops; the
// only warp-level code, the recovery's counter reduction, needs whole warps), so a launch may use any block size
// and grid, and the chunked kernels (sliding-stencil reconstruction and edge inputs) may walk their lines in
// pencils of RCHUNK or RCHUNK_LONG cells (separate item spaces, the same compiled kernel, so the same results).
// The candidates are 64 or 128 threads per block (the kernels are compiled for at most 128, which keeps single
// and batched launches of a body the same compiled code) with an oversubscribed grid (one thread per item up to
// 64 blocks per SM) or a persistent grid (as many blocks as are resident on the SMs at once, each looping over
// the items), times the pencil lengths.  For the kernel bodies whose outputs are a pure function of their inputs
// (reconstruction, face solve, edge inputs, u, face and centre field, vertex potentials), the first launch of a
// kernel at a given item count on a device, outside stream capture, times every candidate on the live data (each
// writes the same outputs) with CUDA events, and the fastest is cached for later launches of that kernel and item
// count; the other bodies, and launches during stream capture before tuning, take 128 threads, the
// oversubscribed grid and pencils of RCHUNK cells.  Tuning synchronises the host with the stream once per kernel
// and item count.  ASTERX_AUTOTUNE=0 in the environment turns it off.

struct LaunchCfg {
  int threads;
  int persistent;
  int variant;  // pencil length index of the chunked kernels (0: RCHUNK, 1: RCHUNK_LONG)
};
constexpr LaunchCfg kDefaultCfg = {128, 0, 0};
constexpr LaunchCfg kShapes[] = {{128, 0, 0}, {64, 0, 0}, {128, 1, 0}, {64, 1, 0}};

template <class Body> struct Tunable { static constexpr bool value = false; };
template <int D, int S> struct Recon;
template <int D> struct ReconPPM;
template <int D> struct ReconWENO;
template <int D> struct Faces;
template <int D> struct FacesAlt;
template <int DF, int K> struct EdgeRecon;
struct UVel;
struct BFace;
struct BCentre;
struct Vertex;
template <int D, int S> struct Tunable<Recon<D, S>> { static constexpr bool value = true; };
template <int D> struct Tunable<ReconPPM<D>> { static constexpr bool value = true; };
template <int D> struct Tunable<ReconWENO<D>> { static constexpr bool value = true; };
template <int D> struct Tunable<Faces<D>> { static constexpr bool value = true; };
template <int D> struct Tunable<FacesAlt<D>> { static constexpr bool value = true; };
template <int DF, int K> struct Tunable<EdgeRecon<DF, K>> { static constexpr bool value = true; };
template <> struct Tunable<UVel> { static constexpr bool value = true; };
template <> struct Tunable<BFace> { static constexpr bool value = true; };
template <> struct Tunable<BCentre> { static constexpr bool value = true; };
template <> struct Tunable<Vertex> { static constexpr bool value = true; };

namespace {
struct TuneEntry {
  int dev;
  const void* fn;
  long n;
  LaunchCfg cfg;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tuned;

bool autotune_on() {
  static const bool on = [] {
    const char* e = std::getenv("ASTERX_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

// With the autotuner off, ASTERX_PENCIL=16 runs the sliding-stencil kernels on the long pencils instead of the
// default ones (the results are the same bit for bit; the tests check that).
bool long_pencils() {
  static const bool on = [] {
    const char* e = std::getenv("ASTERX_PENCIL");
    return e && std::strcmp(e, "16") == 0;
  }();
  return on;
}

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}
}  // namespace

template <class Kern>
int grid_of(Kern kern, LaunchCfg c, long n) {
  if (!c.persistent) return grid_for(n, c.threads);
  const long want = (n + c.threads - 1) / c.threads;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c.threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long cap = (long)per_sm * device_sm_count();
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// The cached configuration of kernel fn at item count n, or the timed choice among the launch shapes times
// `variants` pencil lengths (run(cfg) launches the kernel with cfg on stream s).
template <class Run>
LaunchCfg choose_cfg(const void* fn, long n, int variants, cudaStream_t s, Run run) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return kDefaultCfg;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneEntry& e : g_tuned)
      if (e.dev == dev && e.fn == fn && e.n == n) return e.cfg;
  }
  if (stream_capturing(s)) return kDefaultCfg;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return kDefaultCfg;
  }
  LaunchCfg best = kDefaultCfg;
  float best_ms = 3.0e38f;
  run(kDefaultCfg);  // untimed: first-touch effects
  for (int v = 0; v < variants; v++)
    for (LaunchCfg c : kShapes) {
      c.variant = v;
      cudaEventRecord(e0, s);
      run(c);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaGetLastError() != cudaSuccess)
        continue;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned.push_back({dev, fn, n, best});
  return best;
}

// One launch of Body over the item space `kind`; for a chunked body, `kind_long` is the same item space in
// pencils of RCHUNK_LONG cells (-1: no choice of pencil length).
template <class Body>
void launch(const Single& t, const StageConsts& k0, int kind, cudaStream_t s, int kind_long = -1) {
  const long n = t.count(kind);
  if (n <= 0) return;
  auto kern = k_single<Body>;
  auto run = [&](LaunchCfg q) {
    StageConsts k = k0;
    const int kd = q.variant ? kind_long : kind;
    k.chunk = kind_chunk(kd);
    const long m = t.count(kd);
    kern<<<grid_of(kern, q, m), q.threads, 0, s>>>(t.r, k, m);
  };
  LaunchCfg c = kDefaultCfg;
  if (Tunable<Body>::value && autotune_on())
    c = choose_cfg(reinterpret_cast<const void*>(kern), n, kind_long >= 0 ? 2 : 1, s, run);
  else if (kind_long >= 0 && long_pencils())
    c.variant = 1;
  run(c);
}

template <class Body>
void launch(const Batch& t, const StageConsts& k0, int kind, cudaStream_t s, int kind_long = -1) {
  const long n = t.count(kind);
  if (n <= 0) return;
  auto kern = k_batch<Body>;
  auto run = [&](LaunchCfg q) {
    StageConsts k = k0;
    const int kd = q.variant ? kind_long : kind;
    k.chunk = kind_chunk(kd);
    const long m = t.count(kd);
    const long* off = t.off + (long)kd * (t.nb + 1);
    kern<<<grid_of(kern, q, m), q.threads, 0, s>>>(t.tab, off, t.nb, k);
  };
  LaunchCfg c = kDefaultCfg;
  if (Tunable<Body>::value && autotune_on())
    c = choose_cfg(reinterpret_cast<const void*>(kern), n, kind_long >= 0 ? 2 : 1, s, run);
  else if (kind_long >= 0 && long_pencils())
    c.variant = 1;
  run(c);
}

// ----------------------------------------------------------------------------------------------------------
// Ghost zones (Sec. 3.8): periodic wrap, or copy of the nearest owned value; the edge potential A is
// extrapolated linearly along the normal under copy BCs (when at least two owned layers exist).
// A field's owned index range along an axis is [g, g+n-1] if it is cell-like there (or periodic), [g, g+n]
// if it is vertex-like with copy BCs.  Sweeps run x, then y, then z, each over the full range of the others.

template <int AX, int NF>
__device__ __forceinline__ void ghost_point(const Blk& b, long t, double* const* f, const int* cell_like,
                                            const int* linear) {
  constexpr int A1 = (AX + 1) % 3, A2 = (AX + 2) % 3;
  const int g = b.g, n = b.n[AX], Nn = b.N[AX];
  const long m1 = b.N[A1] + 1;
  const int slots = 2 * g + 1;
  const long st = stride(b, AX);
  int q, q1, q2;
  unflatten3(t, (unsigned)slots, (unsigned)m1, q, q1, q2);
  const int i = (q < g) ? q : Nn - 2 * g + q;
  int p[3];
  p[AX] = 0;
  p[A1] = q1;
  p[A2] = q2;
  const long base = lin(b, p[0], p[1], p[2]);
#pragma unroll
  for (int fi = 0; fi < NF; fi++) {
    const bool cl = (cell_like[fi] >> AX) & 1;
    const int lo = g;
    const int hi = (cl || b.bc[AX] == 0) ? g + n - 1 : g + n;
    if (i >= lo && i <= hi) continue;
    if ((b.halo >> (2 * AX + (i < lo ? 0 : 1))) & 1) continue;  // filled from the neighbouring block
    double* __restrict__ a = f[fi] + base;
    double v;
    if (b.bc[AX] == 0) {
      const int src = lo + (((i - lo) % n) + n) % n;
      v = a[src * st];
    } else {
      const int e0 = (i < lo) ? lo : hi;
      const double f0 = a[e0 * st];
      if (linear[fi] && hi > lo) {
        const int e1 = (i < lo) ? lo + 1 : hi - 1;
        const double f1 = a[e1 * st];
        // unfused rounded operations: the extrapolated value is reproducible exactly
        v = __dadd_rn(f0, __dmul_rn((double)(i < lo ? lo - i : i - hi), __dsub_rn(f0, f1)));
      } else {
        v = f0;
      }
    }
    a[i * st] = v;
  }
}

template <int AX>
struct GhostState {  // the 9 state fields of U_s (record field Us)
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    const int cl[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};
    const int lin_[9] = {0, 0, 0, 0, 0, 1, 1, 1, 0};
    ghost_point<AX, 9>(r.b, t, r.Us.f, cl, lin_);
  }
};

template <int AX>
struct GhostPrims {  // the 5 primitives (record field P)
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    const int cl[5] = {7, 7, 7, 7, 7};
    const int lin_[5] = {0, 0, 0, 0, 0};
    ghost_point<AX, 5>(r.b, t, r.P.f, cl, lin_);
  }
};

// ----------------------------------------------------------------------------------------------------------
// Ghost exchange between the blocks of a tiled domain: a point outside the block's owned range whose domain
// position lies inside the domain (after the periodic wrap) takes the value of the block that owns that
// position, read at the owner's own index; points outside the domain along a copy-BC axis are left to the
// boundary-condition sweeps that follow (which then read exchanged values where a neighbour exists, exactly
// as the sweeps of one block covering the whole domain would).  Owned ranges as in the ghost fill.

template <int NF, bool STATE>
struct Exchange {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    const Blk& b = r.b;
    const Tiling& T = *k.til;
    Box box = make_box(0, b.N[0], 0, b.N[1], 0, b.N[2]);
    int p[3];
    box.at(t, p[0], p[1], p[2]);
    const long c = lin(b, p[0], p[1], p[2]);
    const int clm[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};  // bit a: cell-like along axis a
#pragma unroll 1
    for (int fi = 0; fi < NF; fi++) {
      const int cl_bits = STATE ? clm[fi] : 7;
      bool owned = true, outside = false;
      int own[3], loc[3];
      for (int a = 0; a < 3; a++) {
        const bool cl = (cl_bits >> a) & 1;
        const int hi = (cl || b.bc[a] == 0) ? b.g + b.n[a] - 1 : b.g + b.n[a];
        if (p[a] >= b.g && p[a] <= hi) {
          own[a] = b.coord[a];
          loc[a] = p[a];
          continue;
        }
        owned = false;
        const int Nt = T.ntot[a];
        int G = b.off[a] + p[a] - b.g;  // domain index along a
        if (T.bc[a] == 0) {
          G = ((G % Nt) + Nt) % Nt;
        } else if (G < 0 || G > (cl ? Nt - 1 : Nt)) {
          outside = true;
          break;
        }
        const int* cuts = T.cuts(a);
        int lo = 0, hi2 = T.nblk[a];  // largest lo with cuts[lo] <= G (the last block for G == Nt)
        while (hi2 - lo > 1) {
          const int mid = (lo + hi2) >> 1;
          if (cuts[mid] <= G) lo = mid;
          else hi2 = mid;
        }
        own[a] = lo;
        loc[a] = G - cuts[lo] + b.g;
      }
      if (owned || outside) continue;
      const BlockRec& o = k.tab[own[0] + T.nblk[0] * (own[1] + T.nblk[1] * own[2])];
      const long oc = lin(o.b, loc[0], loc[1], loc[2]);
      if (STATE) r.Us.f[fi][c] = o.Us.f[fi][oc];
      else r.P.f[fi][c] = o.P.f[fi][oc];
    }
  }
};
using ExchangeState = Exchange<9, true>;
using ExchangePrims = Exchange<5, false>;

// ----------------------------------------------------------------------------------------------------------
// B~^i = [ijk] d_j A_k on faces (Eq. BEulerian, second-order differences of the edge values), then the
// undensitised centre field B^i = (B~^i_- + B~^i_+) / (2 sqrt(gamma_c)) (Sec. 3.1).

struct BFace {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    const Blk& b = r.b;
    const double* __restrict__ Ax = r.Us.f[5];
    const double* __restrict__ Ay = r.Us.f[6];
    const double* __restrict__ Az = r.Us.f[7];
    double* __restrict__ bf = r.w.bf;
    Box box = make_box(0, b.N[0], 0, b.N[1], 0, b.N[2]);
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
};

struct BCentre {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    const Blk& b = r.b;
    const double* __restrict__ bf = r.w.bf;
    double* __restrict__ bc = r.w.bc;
    Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    const double sqg = r.w.cg[CG_SQG * b.V + c];
    // correctly rounded quotients, as the oracle divides, so that the centre field (and the reconstruction of its
    // transverse components) matches bit for bit given the same face field: one division, then corrections
    const double isqg = 1.0 / sqg;
    bc[c] = quotient_by(0.5 * (bf[c] + bf[c + 1]), sqg, isqg);
    bc[b.V + c] = quotient_by(0.5 * (bf[b.V + c] + bf[b.V + c + b.sy]), sqg, isqg);
    bc[2 * b.V + c] = quotient_by(0.5 * (bf[2 * b.V + c] + bf[2 * b.V + c + b.sz]), sqg, isqg);
  }
};

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
// Conserved variables from primitives at every cell (initial data, Eq. cons).  Writes record field Us.

struct Prim2Con {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    const Blk& b = r.b;
    Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
    int i, j, kk;
    box.at(t, i, j, kk);
    const long c = lin(b, i, j, kk);
    Geo m;
    load_geo_centre(b, r.w.cg, c, m);
    const double v[3] = {r.P.f[2][c], r.P.f[3][c], r.P.f[4][c]};
    const double W = 1.0 / sqrt(1.0 - contract_sym(m.g, v, v));
    const double u[3] = {W * v[0], W * v[1], W * v[2]};
    const double B[3] = {r.w.bc[c], r.w.bc[b.V + c], r.w.bc[2 * b.V + c]};
    SideOut o;
    face_side<double, false>(m, 1.0 / m.alp, m.alp * sqrt(m.gu[0]), 0, r.P.f[0][c], r.P.f[1][c], u, B, k.gamma,
                             k.gfac, o);
    for (int a = 0; a < 5; a++) r.Us.f[a][c] = o.U[a];
  }
};

// ----------------------------------------------------------------------------------------------------------
// Primitive recovery on interior cells (Sec. 3.5, 3.6): atmosphere if D~ < sqrt(gamma) rho_atm, else Noble 2D
// seeded by the previous primitives, Palenzuela 1D fallback, atmosphere with flag -1 if both fail.  The state
// is record field Us (atmosphere resets in place), the primitives field P.

struct C2PCount {
  unsigned long long noble, fb, atm, fail, it;
};

__device__ __forceinline__ C2PCount c2p_at(const BlockRec& r, const C2PParams& cp, long c) {
  const Blk& b = r.b;
  Geo m;
  load_geo_centre(b, r.w.cg, c, m);
  const F9& U = r.Us;
  const F5& P = r.P;
  const double Dt = U.f[0][c];
  const double B[3] = {r.w.bc[c], r.w.bc[b.V + c], r.w.bc[2 * b.V + c]};
  C2PResult res;
  res.iters = 0;
  bool ok = false;
  bool atm = !(Dt >= m.sqg * cp.rho_atm);
  int flag = 2;
  if (!atm) {
    // correctly rounded quotients, as the oracle divides: on the rim of the torus workload the stage's
    // right-hand side amplifies one-ulp differences of the recovered primitives to about 1e-12 of its magnitude
    const double isqg = 1.0 / m.sqg;
    const double D = quotient_by(Dt, m.sqg, isqg);
    const double S[3] = {quotient_by(U.f[1][c], m.sqg, isqg), quotient_by(U.f[2][c], m.sqg, isqg),
                         quotient_by(U.f[3][c], m.sqg, isqg)};
    const double tau = quotient_by(U.f[4][c], m.sqg, isqg);
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
    if (z0 > 0.0 && isfinite(z0)) ok = c2p_noble(m, D, S, tau, B, S2, B2, BS, z0, gv2, cp, res);
    flag = 0;
    if (!ok && cp.use_fallback) {
      ok = c2p_palenzuela(m, D, S, tau, B, S2, B2, BS, cp, res);
      flag = 1;
    }
    if (!ok) {
      flag = -1;
      atm = true;
    }
  }
  if (atm) {
    res.rho = cp.rho_atm;
    res.press = cp.K_atm * pow(cp.rho_atm, cp.gamma_atm);
    res.v[0] = res.v[1] = res.v[2] = 0.0;
    // conserved variables of the atmosphere state (v = 0, W = 1, b^2 = B^2), field kept (Sec. 3.6)
    double Bl[3];
    lower(m.g, B, Bl);
    const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
    U.f[0][c] = m.sqg * res.rho;
    U.f[1][c] = 0.0;
    U.f[2][c] = 0.0;
    U.f[3][c] = 0.0;
    U.f[4][c] = m.sqg * (res.press / (cp.gamma_atm - 1.0) + 0.5 * B2);
  }
  P.f[0][c] = res.rho;
  P.f[1][c] = res.press;
  P.f[2][c] = res.v[0];
  P.f[3][c] = res.v[1];
  P.f[4][c] = res.v[2];
  if (r.flags) r.flags[c] = (signed char)flag;
  C2PCount out = {0, 0, 0, 0, (unsigned long long)res.iters};
  if (flag == 0) out.noble = 1;
  else if (flag == 1) out.fb = 1;
  else if (flag == 2) out.atm = 1;
  else out.fail = 1;
  return out;
}

__device__ __forceinline__ C2PCount c2p_cell(const BlockRec& r, const C2PParams& cp, long t) {
  const Blk& b = r.b;
  Box box = make_box(b.g, b.g + b.n[0] - 1, b.g, b.g + b.n[1] - 1, b.g, b.g + b.n[2] - 1);
  int i, j, k;
  box.at(t, i, j, k);
  return c2p_at(r, cp, lin(b, i, j, k));
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void add_counts(C2PCount c, unsigned long long* stats) {
  c.noble = warp_sum(c.noble);
  c.fb = warp_sum(c.fb);
  c.atm = warp_sum(c.atm);
  c.fail = warp_sum(c.fail);
  c.it = warp_sum(c.it);
  if ((threadIdx.x & 31) == 0) {
    if (c.noble) atomicAdd(stats + 0, c.noble);
    if (c.fb) atomicAdd(stats + 1, c.fb);
    if (c.atm) atomicAdd(stats + 2, c.atm);
    if (c.fail) atomicAdd(stats + 3, c.fail);
    if (c.it) atomicAdd(stats + 4, c.it);
  }
}

// The grid-stride loops are padded to whole warps so that the counter reduction sees full warps (the block
// size is a multiple of 32 and so is the padded count).
__global__ void __launch_bounds__(128) k_c2p_single(BlockRec r, StageConsts k, long count) {
  const long padded = (count + 31) / 32 * 32;
  GRID_LOOP(t, padded) {
    C2PCount c = {0, 0, 0, 0, 0};
    if (t < count) c = c2p_cell(r, k.cp, t);
    if (k.stats) add_counts(c, k.stats);
  }
}

// the recovery on the cells lo..hi (inclusive, inside the interior) of one block, without counters
struct CellRange {
  int lo[3], hi[3];
};

__global__ void __launch_bounds__(128) k_c2p_range(BlockRec r, StageConsts k, CellRange q, long count) {
  const Box box = make_box(q.lo[0], q.hi[0], q.lo[1], q.hi[1], q.lo[2], q.hi[2]);
  GRID_LOOP(t, count) {
    int i, j, kk;
    box.at(t, i, j, kk);
    c2p_at(r, k.cp, lin(r.b, i, j, kk));
  }
}

__global__ void __launch_bounds__(128) k_c2p_batch(const BlockRec* __restrict__ tab, const long* __restrict__ off,
                                                     int nb, StageConsts k) {
  const long total = off[nb];
  const long padded = (total + 31) / 32 * 32;
  GRID_LOOP(T, padded) {
    C2PCount c = {0, 0, 0, 0, 0};
    if (T < total) {
      const int blk = find_block(off, nb, T);
      c = c2p_cell(tab[blk], k.cp, T - off[blk]);
    }
    if (k.stats) add_counts(c, k.stats);
  }
}

static void launch_c2p_kind(const Single& t, const StageConsts& k, cudaStream_t s) {
  const long n = t.count(KIND_INTERIOR);
  if (n > 0) k_c2p_single<<<grid_for(n, 128), 128, 0, s>>>(t.r, k, n);
}

static void launch_c2p_kind(const Batch& t, const StageConsts& k, cudaStream_t s) {
  const long n = t.count(KIND_INTERIOR);
  if (n > 0)
    k_c2p_batch<<<grid_for(n, 128), 128, 0, s>>>(t.tab, t.off + (long)KIND_INTERIOR * (t.nb + 1), t.nb, k);
}

// ----------------------------------------------------------------------------------------------------------
// u^i = W v^i at every cell (the reconstructed velocity variable).

struct UVel {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    const Blk& b = r.b;
    Box box = make_box(0, b.N[0] - 1, 0, b.N[1] - 1, 0, b.N[2] - 1);
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    double g6[6];
    for (int a = 0; a < 6; a++) g6[a] = r.w.cg[(CG_G + a) * b.V + c];
    const double v[3] = {r.P.f[2][c], r.P.f[3][c], r.P.f[4][c]};
    const double W = 1.0 / sqrt(1.0 - contract_sym(g6, v, v));
    r.w.uvel[c] = W * v[0];
    r.w.uvel[b.V + c] = W * v[1];
    r.w.uvel[2 * b.V + c] = W * v[2];
  }
};

// ----------------------------------------------------------------------------------------------------------
// Reconstruction along D of each cell once (cells g-1 .. g+n along D, all transverse cells): the values at the
// cell's lower and upper D-faces of rho, p, u^x, u^y, u^z and the two transverse centre B components.  Minmod
// and MP5 run per cell; PPM and WENO-Z run as ReconPPM and ReconWENO below (chunks with a sliding stencil).

template <int D, int SCHEME>
struct Recon {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts&, long t) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const Blk& b = r.b;
    int lo[3] = {0, 0, 0}, hi[3] = {b.N[0] - 1, b.N[1] - 1, b.N[2] - 1};
    lo[D] = b.g - 1;
    hi[D] = b.g + b.n[D];
    Box box = make_box(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
    const long st = stride(b, D);
    int i, j, k;
    box.at(t, i, j, k);
    const long c = lin(b, i, j, k);
    const double* src[NREC] = {r.P.f[0], r.P.f[1], r.w.uvel, r.w.uvel + b.V, r.w.uvel + 2 * b.V,
                               r.w.bc + T1 * b.V, r.w.bc + T2 * b.V};
#pragma unroll
    for (int v = 0; v < NREC; v++) {
      double a[5];
#pragma unroll
      for (int s = 0; s < 5; s++) a[s] = src[v][c + (s - 2) * st];
      double l, h;
      recon5<SCHEME>(a, l, h);
      r.w.rec[v * b.V + c] = l;
      r.w.rec[(NREC + v) * b.V + c] = h;
    }
  }
};

// PPM reconstruction along D by chunks: one work item is a run of RCHUNK cells along D (cells g-1 .. g+n, all
// transverse indices) that slides its 5-cell stencil, so each cell forms one new van Leer slope and one new
// interface value (the others carry over from the previous cell) and then applies the CW84 constraints; the
// results are those of Recon<D, 1>.  The transverse axis of smaller stride varies fastest across threads.
template <int D>
struct ReconPPM {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    constexpr int TA = (D == 0) ? 1 : 0, TB = (D == 2) ? 1 : 2;
    const Blk& b = r.b;
    const int lenD = b.n[D] + 2;
    int p[3];
    int ch;
    unflatten3(t, (unsigned)b.N[TA], (unsigned)b.N[TB], p[TA], p[TB], ch);
    const int i0 = b.g - 1 + ch * k.chunk;
    const int i1 = min(b.g - 1 + lenD, i0 + k.chunk);
    p[D] = i0;
    const long st = stride(b, D);
    const long c0 = lin(b, p[0], p[1], p[2]);
    const double* src[NREC] = {r.P.f[0], r.P.f[1], r.w.uvel, r.w.uvel + b.V, r.w.uvel + 2 * b.V,
                               r.w.bc + T1 * b.V, r.w.bc + T2 * b.V};
    for (int v = 0; v < NREC; v++) {
      const double* __restrict__ a = src[v];
      long c = c0;
      double fm2 = a[c - 2 * st], fm1 = a[c - st], f0 = a[c], fp1 = a[c + st], fp2 = a[c + 2 * st];
      double dm = ppm_dq(fm2, fm1, f0), d0 = ppm_dq(fm1, f0, fp1), dp = ppm_dq(f0, fp1, fp2);
      double alo = fm1 + 0.5 * (f0 - fm1) - (d0 - dm) * (1.0 / 6.0);
      for (int i = i0; i < i1; i++) {
        const double ahi = f0 + 0.5 * (fp1 - f0) - (dp - d0) * (1.0 / 6.0);
        double l = alo, h = ahi;
        ppm_limit(f0, l, h);
        r.w.rec[v * b.V + c] = l;
        r.w.rec[(NREC + v) * b.V + c] = h;
        if (i + 1 < i1) {
          fm1 = f0;
          f0 = fp1;
          fp1 = fp2;
          fp2 = a[c + 3 * st];
          d0 = dp;
          dp = ppm_dq(f0, fp1, fp2);
          alo = ahi;
          c += st;
        }
      }
    }
  }
};

// Face solve along D for faces g..g+n along D and all transverse indices: left state = upper value of cell
// f-1, right state = lower value of cell f; HLLE (Eq. HLLEfluxes) and the upwind velocities of Eq. uct1.
// ALT: the alternative schemes (Lax-Friedrichs fluxes, flux constrained transport), a separate instantiation
// (FacesAlt) so that the default kernel (Faces) keeps its register budget.
// Item t of the faces along D (faces g..g+n along D): first the faces whose two transverse indices are interior
// (returns true: their fluxes feed the cell update), then those with one transverse index in the ghost layers
// (returns false: only the edge fields read them, through c_max, c_min, the upwind velocities and, for flux
// constrained transport, the induction fluxes).  The (2g)^2 corner columns, which nothing reads, have no items.
// The first axis of each range varies fastest across items.
template <int D>
__device__ __forceinline__ bool face_item(const Blk& b, long t, int p[3]) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const int gw = 2 * b.g;
  int e[3];
  e[D] = b.n[D] + 1;
  e[T1] = b.n[T1];
  e[T2] = b.n[T2];
  int ghost = -1;  // the transverse axis whose index lies in the ghost layers
  const long nint = (long)e[0] * e[1] * e[2];
  if (t >= nint) {
    t -= nint;
    e[T1] = gw;
    const long na = (long)e[0] * e[1] * e[2];
    if (t < na) {
      ghost = T1;
    } else {
      t -= na;
      e[T1] = b.n[T1];
      e[T2] = gw;
      ghost = T2;
    }
  }
  unflatten3(t, (unsigned)e[0], (unsigned)e[1], p[0], p[1], p[2]);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a == ghost) p[a] = p[a] < b.g ? p[a] : p[a] + b.n[a];  // 0..g-1, then g+n..n+2g-1
    else p[a] += b.g;
  }
  return ghost < 0;
}

template <int D, bool ALT>
struct FaceSolve {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const Blk& b = r.b;
    const long st = stride(b, D);
    const double* __restrict__ fg = r.w.fg + (long)D * NFG * b.V;
    double* __restrict__ fd = r.w.face + (long)D * NFD * b.V;
    int p[3];
    const bool full = face_item<D>(b, t, p);
    const long c = lin(b, p[0], p[1], p[2]);
    Geo m;
    m.alp = fg[FG_ALP * b.V + c];
    for (int a = 0; a < 3; a++) m.beta[a] = fg[(FG_BETA + a) * b.V + c];
    for (int a = 0; a < 6; a++) m.g[a] = fg[(FG_G + a) * b.V + c];
    m.gu[sym(D, D)] = fg[FG_GUDD * b.V + c];  // the only inverse-metric component the face solve reads
    m.sqg = fg[FG_SQG * b.V + c];
    const double ia = fg[FG_IALP * b.V + c];
    const double width = fg[FG_WIDTH * b.V + c];
    const double Bn = r.w.bf[D * b.V + c] * fg[FG_ISQG * b.V + c];
    SideOut s[2];
    // Where the two sides' reconstructed inputs are equal bit for bit (uniform data), the second side's outputs are
    // the first side's, and are copied.  Otherwise, unless the adjoint keeps the four roots, the second side's
    // speeds are iterated only as far as HLLE needs them: it reads c_max = max(0, lambda_+^L, lambda_+^R) and
    // c_min = -min(0, lambda_-^L, lambda_-^R), so lambda_+^R stops once its iterate passes max(0, lambda_+^L) and
    // lambda_-^R once it passes min(0, lambda_-^L); c_max and c_min are those of the full iteration.
    const double* __restrict__ rside[2] = {r.w.rec + NREC * b.V + (c - st), r.w.rec + c};
    double Bt[2][2];  // transverse B^T1, B^T2 (undensitised) of each side
#pragma unroll
    for (int side = 0; side < 2; side++) {
      const double* __restrict__ rr = rside[side];
      double in[7];  // rho, p, u^x, u^y, u^z, B^T1, B^T2
#pragma unroll
      for (int v = 0; v < 7; v++) in[v] = rr[v * b.V];
      Bt[side][0] = in[5];
      Bt[side][1] = in[6];
      const double u[3] = {in[2], in[3], in[4]};
      double B[3];
      B[D] = Bn;
      B[T1] = in[5];
      B[T2] = in[6];
      if (side == 0) {
        face_side(m, ia, width, D, in[0], in[1], u, B, k.gamma, k.gfac, s[0], nullptr, full);
        continue;
      }
      bool same = true;  // bitwise, on the integer pipe
#pragma unroll
      for (int v = 0; v < 7; v++)
        same = same && __double_as_longlong(in[v]) == __double_as_longlong(rside[0][v * b.V]);
      if (same) {
        s[1] = s[0];
      } else {
        const bool keep = r.w.roots != nullptr;  // no cut: the roots are kept
        face_side<double, true, true>(m, ia, width, D, in[0], in[1], u, B, k.gamma, k.gfac, s[1], nullptr, full,
                                      keep ? -INFINITY : fmax(0.0, s[0].lp), keep ? INFINITY : fmin(0.0, s[0].lm));
      }
    }
    const double cmax = fmax(0.0, fmax(s[0].lp, s[1].lp));
    const double cmin = -fmin(0.0, fmin(s[0].lm, s[1].lm));
    const double den = cmax + cmin;
    if (den > 0.0) {
      const double iden = recip(den);
      if (full) {
        if (ALT && k.lxf) {  // Eq. LxFfluxes: c_wave = max(c_max, c_min)
          const double cw = fmax(cmax, cmin);
          for (int v = 0; v < 5; v++)
            fd[(FD_F + v) * b.V + c] = 0.5 * (s[1].F[v] + s[0].F[v] - cw * (s[1].U[v] - s[0].U[v]));
        } else {
          for (int v = 0; v < 5; v++)
            fd[(FD_F + v) * b.V + c] =
                (cmin * s[1].F[v] + cmax * s[0].F[v] - cmax * cmin * (s[1].U[v] - s[0].U[v])) * iden;
        }
      }
      fd[FD_VB1 * b.V + c] = (cmax * s[0].vt[T1] + cmin * s[1].vt[T1]) * iden;
      fd[FD_VB2 * b.V + c] = (cmax * s[0].vt[T2] + cmin * s[1].vt[T2]) * iden;
    } else {
      if (full)
        for (int v = 0; v < 5; v++) fd[(FD_F + v) * b.V + c] = 0.5 * (s[0].F[v] + s[1].F[v]);
      fd[FD_VB1 * b.V + c] = 0.5 * (s[0].vt[T1] + s[1].vt[T1]);
      fd[FD_VB2 * b.V + c] = 0.5 * (s[0].vt[T2] + s[1].vt[T2]);
    }
    if (ALT && k.fct) {
      // induction fluxes along D of B~^T1 and B~^T2 (v~^D B~^a - v~^a B~^D) with the same Riemann solver
      const double Bnt = r.w.bf[D * b.V + c];
      const double sqg = m.sqg;
#pragma unroll
      for (int q = 0; q < 2; q++) {
        const int a = q == 0 ? T1 : T2;
        const double BL = sqg * Bt[0][q], BR = sqg * Bt[1][q];
        const double FL = s[0].vt[D] * BL - s[0].vt[a] * Bnt;
        const double FR = s[1].vt[D] * BR - s[1].vt[a] * Bnt;
        double Fh;
        if (den > 0.0 && k.lxf) Fh = 0.5 * (FR + FL - fmax(cmax, cmin) * (BR - BL));
        else if (den > 0.0) Fh = (cmin * FR + cmax * FL - cmax * cmin * (BR - BL)) / den;
        else Fh = 0.5 * (FL + FR);
        fd[(FD_EB1 + q) * b.V + c] = Fh;
      }
    }
    fd[FD_CMAX * b.V + c] = cmax;
    fd[FD_CMIN * b.V + c] = cmin;
    if (r.w.roots) {  // kept for the adjoint
      double* rt = r.w.roots + (long)D * 4 * b.V + c;
      rt[0] = s[0].lp;
      rt[b.V] = s[0].lm;
      rt[2 * b.V] = s[1].lp;
      rt[3 * b.V] = s[1].lm;
    }
  }
};
template <int D>
struct Faces : FaceSolve<D, false> {};
template <int D>
struct FacesAlt : FaceSolve<D, true> {};

// ----------------------------------------------------------------------------------------------------------
// Stage combine: classical RK4 (stages 0..3) or RK2, the explicit midpoint method (stages 4 and 5); stage < 0
// writes dU/dt.

__device__ __forceinline__ void combine(int stage, double dt, long c, int v, double k, const BlockRec& r) {
  if (stage < 0) {
    r.dU.f[v][c] = k;
  } else if (stage == 0) {
    r.Uacc.f[v][c] = (1.0 / 6.0) * dt * k;
    r.Unext.f[v][c] = r.Un.f[v][c] + 0.5 * dt * k;
  } else if (stage == 1) {
    r.Uacc.f[v][c] = r.Uacc.f[v][c] + (1.0 / 3.0) * dt * k;
    r.Unext.f[v][c] = r.Un.f[v][c] + 0.5 * dt * k;
  } else if (stage == 2) {
    r.Uacc.f[v][c] = r.Uacc.f[v][c] + (1.0 / 3.0) * dt * k;
    r.Unext.f[v][c] = r.Un.f[v][c] + 1.0 * dt * k;
  } else if (stage == 3) {
    r.Unext.f[v][c] = r.Un.f[v][c] + r.Uacc.f[v][c] + (1.0 / 6.0) * dt * k;
  } else if (stage == 4) {  // RK2 (explicit midpoint), first stage
    r.Unext.f[v][c] = r.Un.f[v][c] + 0.5 * dt * k;
  } else {  // RK2, second stage
    r.Unext.f[v][c] = r.Un.f[v][c] + dt * k;
  }
}

// G_A = alpha Psi / sqrt(gamma) - beta^j A_j and F_Psi^j = alpha sqrt(gamma) gamma^jk A_k - beta^j Psi at
// vertices, with A_j averaged from the two adjacent j-edges (Sec. 3.4).
struct Vertex {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    const Blk& b = r.b;
    const Ws& w = r.w;
    const F9& U = r.Us;
    Box box = make_box(b.g - 1, b.g + b.n[0] + 1, b.g - 1, b.g + b.n[1] + 1, b.g - 1, b.g + b.n[2] + 1);
    int i, j, kk;
    box.at(t, i, j, kk);
    const long c = lin(b, i, j, kk);
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
    w.ga[c] = k.lorenz ? (alp * psi / sqg - bA) : 0.0;
    const double as = alp * sqg;
    w.fpsi[c] = as * (gu[0] * Av[0] + gu[1] * Av[1] + gu[2] * Av[2]) - bx * psi;
    w.fpsi[b.V + c] = as * (gu[1] * Av[0] + gu[3] * Av[1] + gu[4] * Av[2]) - by * psi;
    w.fpsi[2 * b.V + c] = as * (gu[2] * Av[0] + gu[4] * Av[1] + gu[5] * Av[2]) - bz * psi;
  }
};


// WENO-Z reconstruction along D by chunks: as ReconPPM, a run of RCHUNK cells along D slides its 5-cell stencil;
// the curvature part (13/12) (second difference)^2 of the Jiang-Shu indicators is shared by three consecutive
// cells, so each cell forms one new curvature term and the rest of its indicators and weights (wenoz_both).
template <int D>
struct ReconWENO {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    constexpr int TA = (D == 0) ? 1 : 0, TB = (D == 2) ? 1 : 2;
    const Blk& b = r.b;
    const int lenD = b.n[D] + 2;
    int p[3];
    int ch;
    unflatten3(t, (unsigned)b.N[TA], (unsigned)b.N[TB], p[TA], p[TB], ch);
    const int i0 = b.g - 1 + ch * k.chunk;
    const int i1 = min(b.g - 1 + lenD, i0 + k.chunk);
    p[D] = i0;
    const long st = stride(b, D);
    const long c0 = lin(b, p[0], p[1], p[2]);
    const double* src[NREC] = {r.P.f[0], r.P.f[1], r.w.uvel, r.w.uvel + b.V, r.w.uvel + 2 * b.V,
                               r.w.bc + T1 * b.V, r.w.bc + T2 * b.V};
    for (int v = 0; v < NREC; v++) {
      const double* __restrict__ a = src[v];
      long c = c0;
      double s[5] = {a[c - 2 * st], a[c - st], a[c], a[c + st], a[c + 2 * st]};
      double k0 = wenoz_curv(s[0], s[1], s[2]), k1 = wenoz_curv(s[1], s[2], s[3]), k2 = wenoz_curv(s[2], s[3], s[4]);
      // the lower face's mirrored candidates: formed here at the pencil's first cell, then carried over from the
      // previous cell's upper-face candidates (the same expressions on the same values, so the same bits)
      double l1 = weno_cand_m(s[1], s[2], s[3]), l2 = weno_cand_p(s[0], s[1], s[2]);
      for (int i = i0; i < i1; i++) {
        double tau5, e0, e1, e2;
        wenoz_indicators(s, k0, k1, k2, tau5, e0, e1, e2);
        const double h1 = weno_cand_p(s[1], s[2], s[3]), h2 = weno_cand_m(s[2], s[3], s[4]);
        double l, h;
        wenoz_combine(tau5, e0, e1, e2, weno_cand_0(s[0], s[1], s[2]), h1, h2, weno_cand_0(s[4], s[3], s[2]), l1, l2,
                      l, h);
        r.w.rec[v * b.V + c] = l;
        r.w.rec[(NREC + v) * b.V + c] = h;
        if (i + 1 < i1) {
          s[0] = s[1];
          s[1] = s[2];
          s[2] = s[3];
          s[3] = s[4];
          s[4] = a[c + 3 * st];
          k0 = k1;
          k1 = k2;
          k2 = wenoz_curv(s[2], s[3], s[4]);
          l1 = h2;
          l2 = h1;
          c += st;
        }
      }
    }
  }
};

// UCT edge inputs: for the faces normal to DF, the PPM lower and upper values along DR (chunked, sliding
// stencil as in ReconPPM) of the upwind velocity v~bar^DR and of the face field B~^DF, over the faces the edges
// use (g-1..g+n along DR, g..g+n along DF, g..g+n-1 along the third axis).  The edge between faces f-1 and f
// along DR takes the upper value of f-1 and the lower value of f: the values ppm_pair forms from f-3..f+2.
template <int DF, int K>
struct EdgeRecon {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    constexpr int DR = (DF + 1 + K) % 3, DE = 3 - DF - DR;
    constexpr int TA = (DF < DE) ? DF : DE, TB = (DF < DE) ? DE : DF;  // transverse axes, smaller stride first
    const Blk& b = r.b;
    const int ea = (TA == DF) ? b.n[DF] + 1 : b.n[DE];
    const int eb = (TB == DF) ? b.n[DF] + 1 : b.n[DE];
    int p[3];
    int ch;
    unflatten3(t, (unsigned)ea, (unsigned)eb, p[TA], p[TB], ch);
    p[TA] += b.g;
    p[TB] += b.g;
    const int i0 = b.g - 1 + ch * k.chunk;
    const int i1 = min(b.g + b.n[DR] + 1, i0 + k.chunk);
    p[DR] = i0;
    const long st = stride(b, DR);
    const long c0 = lin(b, p[0], p[1], p[2]);
    const int slot = (((DF + 1) % 3) == DR) ? FD_VB1 : FD_VB2;
    const double* srcs[2] = {r.w.face + ((long)DF * NFD + slot) * b.V, r.w.bf + (long)DF * b.V};
    double* out = r.w.erec + (long)(DF * 2 + K) * 4 * b.V;
    for (int qn = 0; qn < 2; qn++) {
      const double* __restrict__ a = srcs[qn];
      double* __restrict__ lo = out + (2 * qn) * b.V;
      double* __restrict__ hi = out + (2 * qn + 1) * b.V;
      long c = c0;
      double fm2 = a[c - 2 * st], fm1 = a[c - st], f0 = a[c], fp1 = a[c + st], fp2 = a[c + 2 * st];
      double dm = ppm_dq(fm2, fm1, f0), d0 = ppm_dq(fm1, f0, fp1), dp = ppm_dq(f0, fp1, fp2);
      double alo = fm1 + 0.5 * (f0 - fm1) - (d0 - dm) * (1.0 / 6.0);
      for (int i = i0; i < i1; i++) {
        const double ahi = f0 + 0.5 * (fp1 - f0) - (dp - d0) * (1.0 / 6.0);
        double l = alo, h = ahi;
        ppm_limit(f0, l, h);
        lo[c] = l;
        hi[c] = h;
        if (i + 1 < i1) {
          fm1 = f0;
          f0 = fp1;
          fp1 = fp2;
          fp2 = a[c + 3 * st];
          d0 = dp;
          dp = ppm_dq(f0, fp1, fp2);
          alo = ahi;
          c += st;
        }
      }
    }
  }
};

// Edges along E (owned range): UCT electric field (Sec. 3.4, Eqs. uct1, uct2, eq3.20) with (E, d1, d2) cyclic,
//   E_E = -HLL_d1(v~^d1 B~^d2) + HLL_d2(v~^d2 B~^d1),
// products reconstructed with PPM to the edge from the faces normal to d2 (resp. d1), speeds a_+- at the edge
// the maximum over the two faces sharing it; then dA_E/dt = -E_E - d_E G_A.
template <int E>
struct Edges {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    constexpr int D1 = (E + 1) % 3, D2 = (E + 2) % 3;
    const Blk& b = r.b;
    const Ws& w = r.w;
    int lo[3] = {b.g, b.g, b.g}, hi[3] = {b.g + b.n[0], b.g + b.n[1], b.g + b.n[2]};
    hi[E] -= 1;
    Box box = make_box(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
    int i, j, kk;
    box.at(t, i, j, kk);
    const long c = lin(b, i, j, kk);
    if (k.fct) {
      // flux constrained transport: the average of the induction fluxes on the four faces sharing the edge; the
      // flux along D1 of B~^D2 (slot EB1 of the D1-faces at c and c - e_D2) is -E, the flux along D2 of B~^D1
      // (slot EB2 of the D2-faces at c and c - e_D1) is +E
      const double* __restrict__ f1 = w.face + ((long)D1 * NFD + FD_EB1) * b.V;
      const double* __restrict__ f2 = w.face + ((long)D2 * NFD + FD_EB2) * b.V;
      const double Ee = 0.25 * ((f2[c] + f2[c - stride(b, D1)]) - (f1[c] + f1[c - stride(b, D2)]));
      const double dG = (w.ga[c + stride(b, E)] - w.ga[c]) * b.idx[E];
      combine(k.stage, k.dt, c, 5 + E, -Ee - dG, r);
      return;
    }
    double term[2];
#pragma unroll
    for (int tt = 0; tt < 2; tt++) {
      const int dr = tt == 0 ? D1 : D2;  // reconstruction / upwind direction
      const int df = tt == 0 ? D2 : D1;  // normal of the faces carrying v~^dr and B~^df
      const long sr = stride(b, dr);
      const long sf = stride(b, df);
      // component dr on df-faces: slot VB1 holds component (df+1)%3, VB2 holds (df+2)%3
      // the PPM values on both sides of the edge, from the UCT edge inputs of the faces normal to df
      const int kk = (((df + 1) % 3) == dr) ? 0 : 1;
      const double* __restrict__ er = w.erec + (long)(df * 2 + kk) * 4 * b.V;
      const double vL = er[b.V + c - sr], vR = er[c], BL = er[3 * b.V + c - sr], BR = er[2 * b.V + c];
      const double* __restrict__ fdr = w.face + (long)dr * NFD * b.V;
      const long c0 = c - sf;
      const double ap = fmax(fdr[FD_CMAX * b.V + c0], fdr[FD_CMAX * b.V + c]);
      const double am = fmax(fdr[FD_CMIN * b.V + c0], fdr[FD_CMIN * b.V + c]);
      const double den = ap + am;
      term[tt] = (den > 0.0) ? (ap * vL * BL + am * vR * BR - ap * am * (BR - BL)) / den : 0.5 * (vL * BL + vR * BR);
    }
    const double Ee = -term[0] + term[1];
    const double dG = (w.ga[c + stride(b, E)] - w.ga[c]) * b.idx[E];
    combine(k.stage, k.dt, c, 5 + E, -Ee - dG, r);
  }
};

// dPsi/dt = -d_j F_Psi^j - xi alpha Psi at vertices g..g+n (Eq. recastedScalarPot).
struct Psi {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    const Blk& b = r.b;
    const Ws& w = r.w;
    Box box = make_box(b.g, b.g + b.n[0], b.g, b.g + b.n[1], b.g, b.g + b.n[2]);
    int i, j, kk;
    box.at(t, i, j, kk);
    const long c = lin(b, i, j, kk);
    double rr = 0.0;
    if (k.lorenz) {
      const double div = (w.fpsi[c + 1] - w.fpsi[c - 1]) * (0.5 * b.idx[0]) +
                         (w.fpsi[b.V + c + b.sy] - w.fpsi[b.V + c - b.sy]) * (0.5 * b.idx[1]) +
                         (w.fpsi[2 * b.V + c + b.sz] - w.fpsi[2 * b.V + c - b.sz]) * (0.5 * b.idx[2]);
      rr = -div - k.xi * w.vg[VG_ALP * b.V + c] * r.Us.f[8][c];
    }
    combine(k.stage, k.dt, c, 8, rr, r);
  }
};

// Interior cells: dU/dt = -sum_d (F_d(+) - F_d(-)) / dx_d + S (Eq. fluxconseqs, densitised).
struct Cells {
  static __device__ __forceinline__ void run(const BlockRec& r, const StageConsts& k, long t) {
    const Blk& b = r.b;
    const Ws& w = r.w;
    Box box = make_box(b.g, b.g + b.n[0] - 1, b.g, b.g + b.n[1] - 1, b.g, b.g + b.n[2] - 1);
    int i, j, kk;
    box.at(t, i, j, kk);
    const long c = lin(b, i, j, kk);
    double rr[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double* __restrict__ fd = w.face + (long)d * NFD * b.V;
      const long c1 = c + stride(b, d);
#pragma unroll
      for (int v = 0; v < 5; v++) rr[v] -= (fd[(FD_F + v) * b.V + c1] - fd[(FD_F + v) * b.V + c]) * b.idx[d];
    }
    Geo m;
    load_geo_centre(b, w.cg, c, m);
    const double v[3] = {r.P.f[2][c], r.P.f[3][c], r.P.f[4][c]};
    const double B[3] = {w.bc[c], w.bc[b.V + c], w.bc[2 * b.V + c]};
    double src[5];
    sources(m, w.cg, b.V, c, r.P.f[0][c], r.P.f[1][c], v, B, k.gfac, src);
#pragma unroll
    for (int q = 0; q < 5; q++) combine(k.stage, k.dt, c, q, rr[q] + src[q], r);
  }
};

// ----------------------------------------------------------------------------------------------------------
// Measurement hook: when enabled, an event pair brackets every face-kernel launch on its own stream (not
// while the stream is being captured into a graph).
namespace {
struct FaceProfile {
  bool on = false;
  int cap = 0;
  int n = 0;
  cudaEvent_t* ev = nullptr;  // 2 * cap events
};
FaceProfile g_prof;

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}
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

// ----------------------------------------------------------------------------------------------------------
// Stage sequences, written once for both launch targets.

static StageConsts consts_of(const StageArgs& a, int stage, double dt, unsigned long long* stats) {
  StageConsts k;
  k.gamma = a.gamma;
  k.gfac = a.gfac;
  k.dt = dt;
  k.xi = a.xi > 0.0 ? a.xi : (dt > 0.0 ? 1.5 / dt : 0.0);
  k.stage = stage;
  k.lorenz = (a.gauge == 0);
  k.lxf = (a.flux == 1);
  k.fct = (a.efield == 1);
  k.cp.gamma = a.gamma;
  k.cp.rho_atm = a.rho_atm;
  k.cp.K_atm = a.K_atm;
  k.cp.gamma_atm = a.gamma_atm;
  k.cp.tol = a.c2p_tol;
  k.cp.W_max = a.W_max;
  k.cp.maxiter = a.c2p_maxiter;
  k.cp.brent_maxiter = a.brent_maxiter;
  k.cp.use_fallback = a.use_fallback;
  k.stats = stats;
  k.tab = nullptr;
  k.til = nullptr;
  k.chunk = RCHUNK;
  return k;
}

template <class T>
static void seq_ghost_state(const T& t, const StageConsts& k, cudaStream_t s) {
  launch<GhostState<0>>(t, k, KIND_GHOST_X, s);
  launch<GhostState<1>>(t, k, KIND_GHOST_Y, s);
  launch<GhostState<2>>(t, k, KIND_GHOST_Z, s);
}

template <class T>
static void seq_ghost_prims(const T& t, const StageConsts& k, cudaStream_t s) {
  launch<GhostPrims<0>>(t, k, KIND_GHOST_X, s);
  launch<GhostPrims<1>>(t, k, KIND_GHOST_Y, s);
  launch<GhostPrims<2>>(t, k, KIND_GHOST_Z, s);
}

template <class T>
static void seq_bfield(const T& t, const StageConsts& k, cudaStream_t s) {
  launch<BFace>(t, k, KIND_VERTS_ALL, s);
  launch<BCentre>(t, k, KIND_CELLS_ALL, s);
}

template <int D, class T>
static void seq_dir(const T& t, const StageConsts& k, int recon, cudaStream_t s) {
  if (recon == 0) launch<Recon<D, 0>>(t, k, KIND_RECON_X + D, s);
  else if (recon == 1) launch<ReconPPM<D>>(t, k, KIND_RCHUNK_X + D, s, KIND_RCHUNK16_X + D);
  else if (recon == 3) launch<Recon<D, 3>>(t, k, KIND_RECON_X + D, s);
  else launch<ReconWENO<D>>(t, k, KIND_RCHUNK_X + D, s, KIND_RCHUNK16_X + D);
  const bool mark = g_prof.on && g_prof.n < g_prof.cap && !capturing(s);
  if (mark) cudaEventRecord(g_prof.ev[2 * g_prof.n], s);
  if (k.lxf || k.fct) launch<FacesAlt<D>>(t, k, KIND_FACES_X + D, s);
  else launch<Faces<D>>(t, k, KIND_FACES_X + D, s);
  if (mark) cudaEventRecord(g_prof.ev[2 * g_prof.n++ + 1], s);
}

template <class T>
static void seq_erec(const T& t, const StageConsts& k, cudaStream_t s) {
  launch<EdgeRecon<0, 0>>(t, k, KIND_EREC + 0, s, KIND_EREC16 + 0);
  launch<EdgeRecon<0, 1>>(t, k, KIND_EREC + 1, s, KIND_EREC16 + 1);
  launch<EdgeRecon<1, 0>>(t, k, KIND_EREC + 2, s, KIND_EREC16 + 2);
  launch<EdgeRecon<1, 1>>(t, k, KIND_EREC + 3, s, KIND_EREC16 + 3);
  launch<EdgeRecon<2, 0>>(t, k, KIND_EREC + 4, s, KIND_EREC16 + 4);
  launch<EdgeRecon<2, 1>>(t, k, KIND_EREC + 5, s, KIND_EREC16 + 5);
}

template <class T>
static void seq_rhs_tail(const T& t, const StageConsts& k, cudaStream_t s) {
  if (!k.fct) seq_erec(t, k, s);  // UCT's edge reconstruction (flux constrained transport needs none)
  launch<Vertex>(t, k, KIND_VERTEX, s);
  launch<Edges<0>>(t, k, KIND_EDGES_X, s);
  launch<Edges<1>>(t, k, KIND_EDGES_Y, s);
  launch<Edges<2>>(t, k, KIND_EDGES_Z, s);
  launch<Psi>(t, k, KIND_PSI, s);
  launch<Cells>(t, k, KIND_INTERIOR, s);
}

template <class T>
static void seq_rhs(const T& t, const StageConsts& k, int recon, cudaStream_t s) {
  launch<UVel>(t, k, KIND_CELLS_ALL, s);
  seq_dir<0>(t, k, recon, s);
  seq_dir<1>(t, k, recon, s);
  seq_dir<2>(t, k, recon, s);
  if (!k.fct) seq_erec(t, k, s);
  launch<Vertex>(t, k, KIND_VERTEX, s);
  launch<Edges<0>>(t, k, KIND_EDGES_X, s);
  launch<Edges<1>>(t, k, KIND_EDGES_Y, s);
  launch<Edges<2>>(t, k, KIND_EDGES_Z, s);
  launch<Psi>(t, k, KIND_PSI, s);
  launch<Cells>(t, k, KIND_INTERIOR, s);
}

template <class T>
static void seq_stage(const T& t, const StageConsts& k, int recon, cudaStream_t s) {
  if (k.til) launch<ExchangeState>(t, k, KIND_VERTS_ALL, s);
  seq_ghost_state(t, k, s);
  seq_bfield(t, k, s);
  launch_c2p_kind(t, k, s);
  if (k.til) launch<ExchangePrims>(t, k, KIND_VERTS_ALL, s);
  seq_ghost_prims(t, k, s);
  seq_rhs(t, k, recon, s);
}

static Single single_of(const Blk& b, const Ws& w) {
  Single t;
  std::memset(&t.r, 0, sizeof(t.r));
  t.r.b = b;
  t.r.w = w;
  return t;
}

static StageConsts zero_consts() {
  StageConsts k;
  std::memset(&k, 0, sizeof(k));
  k.chunk = RCHUNK;
  return k;
}

// ----------------------------------------------------------------------------------------------------------
// Single-block launchers (used by the C ABI).

cudaError_t launch_ghost_state(const Blk& b, const F9& U, cudaStream_t s) {
  Ws w;
  std::memset(&w, 0, sizeof(w));
  Single t = single_of(b, w);
  t.r.Us = U;
  seq_ghost_state(t, zero_consts(), s);
  return cudaGetLastError();
}

cudaError_t launch_ghost_prims(const Blk& b, const F5& P, cudaStream_t s) {
  Ws w;
  std::memset(&w, 0, sizeof(w));
  Single t = single_of(b, w);
  t.r.P = P;
  seq_ghost_prims(t, zero_consts(), s);
  return cudaGetLastError();
}

cudaError_t launch_bfield(const Blk& b, const Ws& w, const F9& U, cudaStream_t s) {
  Single t = single_of(b, w);
  t.r.Us = U;
  seq_bfield(t, zero_consts(), s);
  return cudaGetLastError();
}

cudaError_t launch_uvel(const Blk& b, const Ws& w, const F5& P, cudaStream_t s) {
  Single t = single_of(b, w);
  t.r.P = P;
  launch<UVel>(t, zero_consts(), KIND_CELLS_ALL, s);
  return cudaGetLastError();
}

cudaError_t launch_prim2con(const StageArgs& a, const F9& U, const F5& P, cudaStream_t s) {
  Single t = single_of(a.b, a.w);
  t.r.Us = U;
  t.r.P = P;
  launch<Prim2Con>(t, consts_of(a, -1, 0.0, nullptr), KIND_CELLS_ALL, s);
  return cudaGetLastError();
}

cudaError_t launch_c2p(const StageArgs& a, const F9& U, const F5& P, signed char* flags,
                       unsigned long long* stats, cudaStream_t s) {
  Single t = single_of(a.b, a.w);
  t.r.Us = U;
  t.r.P = P;
  t.r.flags = flags;
  launch_c2p_kind(t, consts_of(a, -1, 0.0, stats), s);
  return cudaGetLastError();
}

cudaError_t launch_c2p_range(const StageArgs& a, const F9& U, const F5& P, const int lo[3], const int hi[3],
                             cudaStream_t s) {
  Single t = single_of(a.b, a.w);
  t.r.Us = U;
  t.r.P = P;
  CellRange q;
  long count = 1;
  for (int d = 0; d < 3; d++) {
    if (lo[d] < a.b.g || hi[d] > a.b.g + a.b.n[d] - 1 || hi[d] < lo[d]) return cudaErrorInvalidValue;
    q.lo[d] = lo[d];
    q.hi[d] = hi[d];
    count *= hi[d] - lo[d] + 1;
  }
  k_c2p_range<<<grid_for(count, 128), 128, 0, s>>>(t.r, consts_of(a, -1, 0.0, nullptr), q, count);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const StageArgs& a, const F9& Us, const F5& P, int stage, double dt, const F9& Un,
                       const F9& Unext, const F9& Uacc, const F9& dU, cudaStream_t s) {
  Single t = single_of(a.b, a.w);
  t.r.Us = Us;
  t.r.P = P;
  t.r.Un = Un;
  t.r.Unext = Unext;
  t.r.Uacc = Uacc;
  t.r.dU = dU;
  seq_rhs(t, consts_of(a, stage, dt, nullptr), a.recon, s);
  return cudaGetLastError();
}

cudaError_t launch_rhs_from_kept(const StageArgs& sa, const AdjWs& a, int stage, double dt, const F9& Un,
                                 const F9& Unext, const F9& Uacc, const F9& dU, cudaStream_t s) {
  Ws w = sa.w;
  w.bf = a.kbf;
  w.bc = a.kbc;
  w.uvel = a.kuvel;
  w.face = a.kface;
  Single t = single_of(sa.b, w);
  t.r.Us = a.Y;
  t.r.P = a.P;
  t.r.Un = Un;
  t.r.Unext = Unext;
  t.r.Uacc = Uacc;
  t.r.dU = dU;
  seq_rhs_tail(t, consts_of(sa, stage, dt, nullptr), s);
  return cudaGetLastError();
}

cudaError_t launch_face_data(const StageArgs& a, const F5& P, double* const rec[3], double* roots, cudaStream_t s) {
  Single t = single_of(a.b, a.w);
  t.r.P = P;
  t.r.w.roots = roots;
  const StageConsts k = consts_of(a, -1, 0.0, nullptr);
  launch<UVel>(t, k, KIND_CELLS_ALL, s);
  Single td[3] = {t, t, t};
  for (int d = 0; d < 3; d++) td[d].r.w.rec = rec[d];
  seq_dir<0>(td[0], k, a.recon, s);
  seq_dir<1>(td[1], k, a.recon, s);
  seq_dir<2>(td[2], k, a.recon, s);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------------------------
// Batched stage: every block of the table in one launch per kernel.

cudaError_t launch_batch_ghosts(const BlockRec* tab, const long* off, const long* host_total, int nb,
                                const Tiling* tiling, cudaStream_t s) {
  Batch t;
  t.tab = tab;
  t.off = off;
  t.host_total = host_total;
  t.nb = nb;
  StageConsts k = zero_consts();
  k.tab = tab;
  k.til = tiling;
  if (tiling) launch<ExchangeState>(t, k, KIND_VERTS_ALL, s);
  seq_ghost_state(t, k, s);
  return cudaGetLastError();
}

cudaError_t launch_batch_stage(const StageArgs& a, const BlockRec* tab, const long* off, const long* host_total,
                               int nb, int stage, double dt, unsigned long long* stats, cudaStream_t s,
                               const Tiling* tiling) {
  Batch t;
  t.tab = tab;
  t.off = off;
  t.host_total = host_total;
  t.nb = nb;
  StageConsts k = consts_of(a, stage, dt, stats);
  if (tiling) {
    k.tab = tab;
    k.til = tiling;
  }
  seq_stage(t, k, a.recon, s);
  return cudaGetLastError();
}

}  // namespace asterx
