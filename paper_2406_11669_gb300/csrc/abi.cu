// Host runtime of the C ABI declared in include/asterx.h: argument validation (before any launch), workspace
// layout, and the order of launches of one RK stage (Sec. 3.12 workflow of arXiv:2406.11669).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/asterx.h"
#include "kernels.h"
#include "validate.h"

using namespace asterx;

namespace {

constexpr int kAbiVersion = 2;
constexpr size_t kAlign = 256;

long padded_V(const asterx_block* b) { return check::padded_volume(b); }

// each field starts on a 256-byte boundary
long field_stride(long V) { return (V + 31) / 32 * 32; }

using check::block_ok;
using check::finite_pos;
using check::params_ok;
using check::ptr_ok;
using check::set_ok;

size_t ws_bytes_for(const asterx_block* b) {
  const long fs = field_stride(padded_V(b));
  return (size_t)WS_FIELDS * fs * sizeof(double) + 8 * sizeof(unsigned long long) + kAlign;
}

Blk make_blk(const asterx_block* in) {
  Blk b;
  std::memset(&b, 0, sizeof(b));
  b.g = in->g;
  for (int d = 0; d < 3; d++) {
    b.n[d] = in->n[d];
    b.N[d] = in->n[d] + 2 * in->g;
    b.bc[d] = in->bc[d];
    b.dx[d] = in->dx[d];
    b.idx[d] = 1.0 / in->dx[d];
  }
  b.sy = b.N[0] + 1;
  b.sz = (long)(b.N[0] + 1) * (b.N[1] + 1);
  b.V = (long)(b.N[0] + 1) * (b.N[1] + 1) * (b.N[2] + 1);
  return b;
}

Ws make_ws(const asterx_block* in, void* base) {
  const long fs = field_stride(padded_V(in));
  double* p = reinterpret_cast<double*>(base);
  Ws w;
  auto take = [&](int nf) {
    double* q = p;
    p += (long)nf * fs;
    return q;
  };
  // a group of nf fields starts on a 256-byte boundary and holds its fields at pitch V (kernels index
  // group + f * V); nf * fs >= nf * V leaves the padding at the group's end
  w.cg = take(NCG);
  w.fg = take(3 * NFG);
  w.vg = take(NVG);
  w.bf = take(3);
  w.bc = take(3);
  w.uvel = take(3);
  w.rec = take(2 * NREC);
  w.face = take(3 * NFD);
  w.ga = take(1);
  w.fpsi = take(3);
  w.uacc = take(9);
  w.ustage = take(18);
  w.erec = take(24);
  w.counters = reinterpret_cast<unsigned long long*>(p);
  w.roots = nullptr;
  return w;
}

StageArgs make_args(const asterx_params* p, const asterx_block* blk, void* ws) {
  StageArgs a;
  a.b = make_blk(blk);
  a.w = make_ws(blk, ws);
  a.recon = p->recon;
  a.gauge = p->gauge;
  a.gamma = p->gamma;
  a.gfac = p->gamma / (p->gamma - 1.0);
  a.rho_atm = p->rho_atm;
  a.K_atm = p->K_atm;
  a.gamma_atm = p->gamma_atm;
  a.c2p_tol = p->c2p_tol;
  a.W_max = p->W_max;
  a.xi = p->xi_lorenz;
  a.c2p_maxiter = p->c2p_maxiter;
  a.brent_maxiter = p->brent_maxiter;
  a.use_fallback = p->use_fallback;
  a.flux = p->flux;
  a.efield = p->efield;
  return a;
}

F9 f9(const asterx_state* s) {
  F9 f;
  std::memcpy(f.f, s, sizeof(f.f));
  return f;
}
F5 f5(const asterx_prims* s) {
  F5 f;
  std::memcpy(f.f, s, sizeof(f.f));
  return f;
}

asterx_status common_checks(const asterx_params* p, const asterx_block* blk, void* ws, size_t ws_bytes) {
  if (!params_ok(p) || !block_ok(blk)) return ASTERX_EINVAL;
  if (!ws || ((uintptr_t)ws % kAlign) != 0) return ASTERX_EINVAL;
  if (ws_bytes < ws_bytes_for(blk)) return ASTERX_ENOMEM;
  return ASTERX_OK;
}

asterx_status cuda_status(cudaError_t e) { return e == cudaSuccess ? ASTERX_OK : ASTERX_ECUDA; }

}  // namespace

// One RK4 step of a batch captured as a CUDA graph (112 launches), replayed by later calls.  The graph bakes in the
// launch parameters (tables, per-kind totals, dt, counters, physics parameters), so an entry is reused only
// when all of them match; asterx_batch_prepare and asterx_batch_release drop the entries of their workspace.
namespace {
struct StepGraph {
  int device;
  void* ws;
  int nb;
  double dt;
  void* stats;
  asterx_params p;
  std::vector<long> totals;
  cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::vector<StepGraph> g_graphs;
std::vector<void*> g_tiled;  // batch workspaces prepared as a tiled domain (guarded by g_graph_mu)

void set_tiled(void* ws, bool tiled) {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  g_tiled.erase(std::remove(g_tiled.begin(), g_tiled.end(), ws), g_tiled.end());
  if (tiled) g_tiled.push_back(ws);
}

bool is_tiled(void* ws) {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  return std::find(g_tiled.begin(), g_tiled.end(), ws) != g_tiled.end();
}

void drop_graphs(void* ws) {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (size_t i = 0; i < g_graphs.size();) {
    if (g_graphs[i].ws == ws) {
      cudaGraphExecDestroy(g_graphs[i].exec);
      g_graphs.erase(g_graphs.begin() + i);
    } else {
      i++;
    }
  }
}

// the cached step graph for these launch parameters (null if there is none)
cudaGraphExec_t cached_graph(const asterx_params* p, void* ws, const long* totals, int nb, double dt,
                             unsigned long long* stats) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (const StepGraph& g : g_graphs)
    if (g.device == dev && g.ws == ws && g.nb == nb && g.dt == dt && g.stats == stats &&
        std::memcmp(&g.p, p, sizeof(*p)) == 0 && std::equal(g.totals.begin(), g.totals.end(), totals))
      return g.exec;
  return nullptr;
}

// the cached step graph for these launch parameters, captured on a private stream if there is none (null if
// capture is not possible, e.g. inside the caller's own capture)
cudaGraphExec_t step_graph(const StageArgs& a, const asterx_params* p, void* ws, const BlockRec* tab, const long* off,
                           const long* totals, int nb, double dt, unsigned long long* stats, const Tiling* til) {
  if (cudaGraphExec_t g = cached_graph(p, ws, totals, nb, dt, stats)) return g;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_graph_mu);
  cudaStream_t ps = nullptr;
  if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int stage = 0; stage < 4 && e == cudaSuccess; stage++)
      e = launch_batch_stage(a, tab + (size_t)stage * nb, off, totals, nb, stage, dt, stats, ps, til);
    const cudaError_t e2 = cudaStreamEndCapture(ps, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(ps);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  StepGraph g;
  g.device = dev;
  g.ws = ws;
  g.nb = nb;
  g.dt = dt;
  g.stats = stats;
  g.p = *p;
  g.totals.assign(totals, totals + NKIND);
  g.exec = exec;
  g_graphs.push_back(g);
  return exec;
}
}  // namespace

extern "C" {

int asterx_abi_version(void) { return kAbiVersion; }

const char* asterx_status_str(asterx_status s) {
  switch (s) {
    case ASTERX_OK: return "ok";
    case ASTERX_EINVAL: return "invalid argument";
    case ASTERX_ECUDA: return "CUDA error";
    case ASTERX_ENOMEM: return "workspace too small";
    case ASTERX_EC2P: return "primitive recovery failed";
    case ASTERX_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

size_t asterx_workspace_size(const asterx_block* blk) {
  if (!block_ok(blk)) return 0;
  return ws_bytes_for(blk);
}

asterx_status asterx_prepare(const asterx_params* p, const asterx_block* blk, const asterx_metric* metric,
                             void* ws, size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_metric, 16>(metric)) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  CF16 m;
  std::memcpy(m.f, metric, sizeof(m.f));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(a.w.counters, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return ASTERX_ECUDA;
  return cuda_status(launch_prepare(a.b, m, a.w, s));
}

asterx_status asterx_prim2con(const asterx_params* p, const asterx_block* blk, asterx_state* U,
                              const asterx_prims* P, void* ws, size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P)) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  F9 u = f9(U);
  cudaError_t e = launch_bfield(a.b, a.w, u, s);
  if (e == cudaSuccess) e = launch_prim2con(a, u, f5(P), s);
  return cuda_status(e);
}

asterx_status asterx_fill_ghosts(const asterx_params* p, const asterx_block* blk, asterx_state* U, void* ws,
                                 size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U)) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  return cuda_status(launch_ghost_state(a.b, f9(U), reinterpret_cast<cudaStream_t>(stream)));
}

asterx_status asterx_con2prim(const asterx_params* p, const asterx_block* blk, asterx_state* U,
                              asterx_prims* P, signed char* flags, asterx_c2p_stats* stats, void* ws,
                              size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P)) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  F9 u = f9(U);
  cudaError_t e = launch_bfield(a.b, a.w, u, s);
  if (e == cudaSuccess)
    e = launch_c2p(a, u, f5(P), flags, reinterpret_cast<unsigned long long*>(stats), s);
  return cuda_status(e);
}

asterx_status asterx_rhs(const asterx_params* p, const asterx_block* blk, const asterx_state* U,
                         const asterx_prims* P, asterx_state* dUdt, double dt, void* ws, size_t ws_bytes,
                         asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P) || !set_ok<asterx_state, 9>(dUdt))
    return ASTERX_EINVAL;
  if (!finite_pos(dt)) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  F9 u = f9(U), d = f9(dUdt);
  cudaError_t e = launch_bfield(a.b, a.w, u, s);
  if (e == cudaSuccess) e = launch_rhs(a, u, f5(P), -1, dt, u, u, u, d, s);
  return cuda_status(e);
}

// prims_ready, when given, is recorded once the stage's primitives are final (after the recovery and their ghost
// fill; the right-hand side only reads them).
static asterx_status stage_impl(const StageArgs& a, int stage, double dt, const F9& un, const F9& us,
                                const F9& unext, const F9& uacc, const F5& pr, signed char* flags,
                                unsigned long long* stats, cudaStream_t s, cudaEvent_t prims_ready = nullptr) {
  cudaError_t e = launch_ghost_state(a.b, us, s);
  if (e == cudaSuccess) e = launch_bfield(a.b, a.w, us, s);
  if (e == cudaSuccess) e = launch_c2p(a, us, pr, flags, stats, s);
  if (e == cudaSuccess) e = launch_ghost_prims(a.b, pr, s);
  if (e == cudaSuccess && prims_ready) e = cudaEventRecord(prims_ready, s);
  if (e == cudaSuccess) e = launch_rhs(a, us, pr, stage, dt, un, unext, uacc, unext, s);
  return cuda_status(e);
}

asterx_status asterx_rk_stage(const asterx_params* p, const asterx_block* blk, int stage, double dt,
                              const asterx_state* Un, asterx_state* Us, asterx_state* Unext, asterx_state* Uacc,
                              asterx_prims* P, signed char* flags, asterx_c2p_stats* stats, void* ws,
                              size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (stage < 0 || stage > 3 || !finite_pos(dt)) return ASTERX_EINVAL;
  if (!set_ok<asterx_state, 9>(Un) || !set_ok<asterx_state, 9>(Us) || !set_ok<asterx_state, 9>(Unext) ||
      !set_ok<asterx_state, 9>(Uacc) || !set_ok<asterx_prims, 5>(P))
    return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  return stage_impl(a, stage, dt, f9(Un), f9(Us), f9(Unext), f9(Uacc), f5(P), flags,
                    reinterpret_cast<unsigned long long*>(stats), reinterpret_cast<cudaStream_t>(stream));
}

// The four stages of one classical RK4 step; prims_ready (optional) is recorded when the last stage's primitives
// are final.
static asterx_status rk4_impl(const asterx_params* p, const asterx_block* blk, double dt, asterx_state* U,
                              asterx_prims* P, signed char* flags, asterx_c2p_stats* stats, void* ws,
                              cudaStream_t s, cudaEvent_t prims_ready) {
  StageArgs a = make_args(p, blk, ws);
  const long V = a.b.V;
  F9 un = f9(U), acc, sb[2];
  for (int v = 0; v < 9; v++) {
    acc.f[v] = a.w.uacc + v * V;
    sb[0].f[v] = a.w.ustage + v * V;
    sb[1].f[v] = a.w.ustage + (9 + v) * V;
  }
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  for (int stage = 0; stage < 4; stage++) {
    const F9& us = stage == 0 ? un : sb[(stage - 1) % 2];
    const F9& unext = stage == 3 ? un : sb[stage % 2];
    const asterx_status st =
        stage_impl(a, stage, dt, un, us, unext, acc, f5(P), flags, cnt, s, stage == 3 ? prims_ready : nullptr);
    if (st != ASTERX_OK) return st;
  }
  return ASTERX_OK;
}

asterx_status asterx_rk4_step(const asterx_params* p, const asterx_block* blk, double dt, asterx_state* U,
                              asterx_prims* P, signed char* flags, asterx_c2p_stats* stats, void* ws,
                              size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || !set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P)) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  return rk4_impl(p, blk, dt, U, P, flags, stats, ws, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

// the fine block nested in the coarse one as asterx_prolong requires; L = the coarse cell of the fine corner
static bool nesting_ok(const asterx_block* c, const asterx_block* f, int L[3]) {
  if (!block_ok(c) || !block_ok(f)) return false;
  for (int d = 0; d < 3; d++) {
    if (f->dx[d] * 2.0 != c->dx[d] || (f->n[d] % 2) != 0) return false;
    const double q = (f->x0[d] - c->x0[d]) / c->dx[d];
    L[d] = (int)std::lround(q);
    if (std::fabs(q - L[d]) > 1e-9 || L[d] < 0 || L[d] + f->n[d] / 2 > c->n[d]) return false;
  }
  return true;
}

asterx_status asterx_prolong(const asterx_block* coarse, const asterx_block* fine, const asterx_state* Uc,
                             const asterx_prims* Pc, asterx_state* Uf, asterx_prims* Pf, int all,
                             asterx_stream stream) {
  int L[3];
  if (!nesting_ok(coarse, fine, L)) return ASTERX_EINVAL;
  if (!set_ok<asterx_state, 9>(Uc) || !set_ok<asterx_prims, 5>(Pc) || !set_ok<asterx_state, 9>(Uf) ||
      !set_ok<asterx_prims, 5>(Pf))
    return ASTERX_EINVAL;
  return cuda_status(launch_prolong(make_blk(coarse), make_blk(fine), L, f9(Uc), f5(Pc), f9(Uf), f5(Pf), all != 0,
                                    reinterpret_cast<cudaStream_t>(stream)));
}

// a stage whose ghost layers (state and primitives) are given: the fine level's, prolonged from the coarse one
static asterx_status stage_given_ghosts(const StageArgs& a, int stage, double dt, const F9& un, const F9& us,
                                        const F9& unext, const F9& uacc, const F5& pr, unsigned long long* stats,
                                        cudaStream_t s) {
  cudaError_t e = launch_bfield(a.b, a.w, us, s);
  if (e == cudaSuccess) e = launch_c2p(a, us, pr, nullptr, stats, s);
  if (e == cudaSuccess) e = launch_rhs(a, us, pr, stage, dt, un, unext, uacc, unext, s);
  return cuda_status(e);
}

asterx_status asterx_rk4_step_refined(const asterx_params* p, const asterx_block* coarse, const asterx_block* fine,
                                      double dt, asterx_state* Uc, asterx_prims* Pc, asterx_state* Uf,
                                      asterx_prims* Pf, asterx_c2p_stats* stats, void* ws_c, size_t ws_c_bytes,
                                      void* ws_f, size_t ws_f_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, coarse, ws_c, ws_c_bytes);
  if (st == ASTERX_OK) st = common_checks(p, fine, ws_f, ws_f_bytes);
  if (st != ASTERX_OK) return st;
  int L[3];
  if (!nesting_ok(coarse, fine, L) || !finite_pos(dt)) return ASTERX_EINVAL;
  if (!set_ok<asterx_state, 9>(Uc) || !set_ok<asterx_prims, 5>(Pc) || !set_ok<asterx_state, 9>(Uf) ||
      !set_ok<asterx_prims, 5>(Pf))
    return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  StageArgs ac = make_args(p, coarse, ws_c), af = make_args(p, fine, ws_f);
  F9 unc = f9(Uc), unf = f9(Uf), accc, accf, sbc[2], sbf[2];
  for (int v = 0; v < 9; v++) {
    accc.f[v] = ac.w.uacc + v * ac.b.V;
    accf.f[v] = af.w.uacc + v * af.b.V;
    for (int q = 0; q < 2; q++) {
      sbc[q].f[v] = ac.w.ustage + (9 * q + v) * ac.b.V;
      sbf[q].f[v] = af.w.ustage + (9 * q + v) * af.b.V;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  const F5 pc = f5(Pc), pf = f5(Pf);
  for (int stage = 0; stage < 4; stage++) {
    const F9& usc = stage == 0 ? unc : sbc[(stage - 1) % 2];
    const F9& unxc = stage == 3 ? unc : sbc[stage % 2];
    const F9& usf = stage == 0 ? unf : sbf[(stage - 1) % 2];
    const F9& unxf = stage == 3 ? unf : sbf[stage % 2];
    st = stage_impl(ac, stage, dt, unc, usc, unxc, accc, pc, nullptr, cnt, s);
    if (st != ASTERX_OK) return st;
    if (launch_prolong(ac.b, af.b, L, usc, pc, usf, pf, false, s) != cudaSuccess) return ASTERX_ECUDA;
    st = stage_given_ghosts(af, stage, dt, unf, usf, unxf, accf, pf, cnt, s);
    if (st != ASTERX_OK) return st;
  }
  return cuda_status(launch_restrict(ac.b, af.b, L, unc, unf, s));
}

// Subcycling (Sec. 3.10): the weights of the coarse slopes h k_i in the fine ghost data at stage s of fine
// substep m.  The coarse step's continuous extension u(t_n + theta h) = u_n + h sum_i b_i(theta) k_i, with
// b_1 = theta - 3/2 theta^2 + 2/3 theta^3, b_2 = b_3 = theta^2 - 2/3 theta^3, b_4 = -1/2 theta^2 + 2/3 theta^3,
// gives u and its first three time derivatives at the substep start theta = m / 2.  The fine stage states of a
// linear problem are u, u + (h_f/2) u', u + (h_f/2) u' + (h_f^2/4) u'' and u + h_f u' + (h_f^2/2) u'' +
// (h_f^3/4) u'''; with h_f = h / 2 they weight the theta-derivatives by 1/4, 1/16 (stages 1, 2) and by
// 1/2, 1/8, 1/32 (stage 3).
static void subcycle_weights(int m, int s, double beta[4]) {
  const double t = 0.5 * m;
  const double b0[4] = {t - 1.5 * t * t + 2.0 * (t * t * t) / 3.0, t * t - 2.0 * (t * t * t) / 3.0,
                        t * t - 2.0 * (t * t * t) / 3.0, -0.5 * t * t + 2.0 * (t * t * t) / 3.0};
  const double b1[4] = {1.0 - 3.0 * t + 2.0 * t * t, 2.0 * t - 2.0 * t * t, 2.0 * t - 2.0 * t * t, -t + 2.0 * t * t};
  const double b2[4] = {-3.0 + 4.0 * t, 2.0 - 4.0 * t, 2.0 - 4.0 * t, -1.0 + 4.0 * t};
  const double b3[4] = {4.0, -4.0, -4.0, 4.0};
  static const double w1[4] = {0.0, 0.25, 0.25, 0.5}, w2[4] = {0.0, 0.0, 1.0 / 16.0, 0.125},
                      w3[4] = {0.0, 0.0, 0.0, 1.0 / 32.0};
  for (int i = 0; i < 4; i++) beta[i] = b0[i] + w1[s] * b1[i] + w2[s] * b2[i] + w3[s] * b3[i];
}

static size_t subcycle_bytes_for(const asterx_block* coarse) {
  const size_t fields = 5 * 9 + 5;  // U_n, Y_1, Y_2, Y_3, the interpolated state; its primitives
  return (fields * (size_t)padded_V(coarse) * sizeof(double) + kAlign - 1) / kAlign * kAlign;
}

size_t asterx_subcycle_workspace_size(const asterx_block* coarse) {
  if (!block_ok(coarse)) return 0;
  return subcycle_bytes_for(coarse);
}

asterx_status asterx_rk4_step_subcycled(const asterx_params* p, const asterx_block* coarse,
                                        const asterx_block* fine, double dt, asterx_state* Uc, asterx_prims* Pc,
                                        asterx_state* Uf, asterx_prims* Pf, asterx_c2p_stats* stats, void* ws_c,
                                        size_t ws_c_bytes, void* ws_f, size_t ws_f_bytes, void* ws_t,
                                        size_t ws_t_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, coarse, ws_c, ws_c_bytes);
  if (st == ASTERX_OK) st = common_checks(p, fine, ws_f, ws_f_bytes);
  if (st != ASTERX_OK) return st;
  int L[3];
  if (!nesting_ok(coarse, fine, L) || !finite_pos(dt)) return ASTERX_EINVAL;
  if (!set_ok<asterx_state, 9>(Uc) || !set_ok<asterx_prims, 5>(Pc) || !set_ok<asterx_state, 9>(Uf) ||
      !set_ok<asterx_prims, 5>(Pf))
    return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  if (!ws_t || ((uintptr_t)ws_t % kAlign) != 0) return ASTERX_EINVAL;
  if (ws_t_bytes < subcycle_bytes_for(coarse)) return ASTERX_ENOMEM;
  StageArgs ac = make_args(p, coarse, ws_c), af = make_args(p, fine, ws_f);
  const long Vc = ac.b.V;
  double* t = static_cast<double*>(ws_t);
  F9 unc = f9(Uc), unf = f9(Uf), accc, accf, sbf[2], un, y[3], yt;
  F5 pt;
  for (int v = 0; v < 9; v++) {
    accc.f[v] = ac.w.uacc + v * Vc;
    accf.f[v] = af.w.uacc + v * af.b.V;
    for (int q = 0; q < 2; q++) sbf[q].f[v] = af.w.ustage + (9 * q + v) * af.b.V;
    un.f[v] = t + v * Vc;
    for (int q = 0; q < 3; q++) y[q].f[v] = t + (9 * (q + 1) + v) * Vc;
    yt.f[v] = t + (36 + v) * Vc;
  }
  for (int v = 0; v < 5; v++) pt.f[v] = t + (45 + v) * Vc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  const F5 pc = f5(Pc), pf = f5(Pf);
  // the coarse step, keeping its stage states and its base (as the first stage's recovery leaves it)
  for (int stage = 0; stage < 4; stage++) {
    const F9& us = stage == 0 ? unc : y[stage - 1];
    const F9& unext = stage == 3 ? unc : y[stage];
    st = stage_impl(ac, stage, dt, unc, us, unext, accc, pc, nullptr, cnt, s);
    if (st != ASTERX_OK) return st;
    if (stage == 0)
      for (int v = 0; v < 9; v++)
        if (cudaMemcpyAsync(un.f[v], unc.f[v], Vc * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          return ASTERX_ECUDA;
  }
  for (int v = 0; v < 5; v++)
    if (cudaMemcpyAsync(pt.f[v], pc.f[v], Vc * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return ASTERX_ECUDA;
  // the coarse cells whose primitives the prolongation reads (cells L - 3 .. L + n_fine/2 + 2 of the interior,
  // one more on each side kept as margin); an axis where that range would leave the interior is recovered
  // whole, so that the ghost fill (periodic wrap included) reads recovered cells only
  // the interpolated state itself is formed on those cells and two more points on each side (the face and
  // centre field of the recovery reach one point beyond them, the prolongation of the potentials one more), or
  // along the whole padded axis where the recovery covers the whole axis
  int rlo[3], rhi[3], clo[3], chi[3];
  for (int d = 0; d < 3; d++) {
    rlo[d] = ac.b.g + L[d] - 4;
    rhi[d] = ac.b.g + L[d] + fine->n[d] / 2 + 3;
    clo[d] = rlo[d] - 2;
    chi[d] = rhi[d] + 2;
    if (rlo[d] < ac.b.g || rhi[d] > ac.b.g + ac.b.n[d] - 1) {
      rlo[d] = ac.b.g;
      rhi[d] = ac.b.g + ac.b.n[d] - 1;
      clo[d] = 0;
      chi[d] = ac.b.N[d];
    }
  }
  // two fine steps of dt / 2, their ghost data from the coarse step by time interpolation
  for (int m = 0; m < 2; m++) {
    for (int stage = 0; stage < 4; stage++) {
      double beta[4];
      subcycle_weights(m, stage, beta);
      cudaError_t e = launch_subcycle_combine(ac.b, clo, chi, un, y[0], y[1], y[2], unc, yt, beta, s);
      if (e == cudaSuccess) e = launch_ghost_state(ac.b, yt, s);
      if (e == cudaSuccess) e = launch_bfield(ac.b, ac.w, yt, s);
      if (e == cudaSuccess) e = launch_c2p_range(ac, yt, pt, rlo, rhi, s);
      if (e == cudaSuccess) e = launch_ghost_prims(ac.b, pt, s);
      const F9& usf = stage == 0 ? unf : sbf[(stage - 1) % 2];
      const F9& unxf = stage == 3 ? unf : sbf[stage % 2];
      if (e == cudaSuccess) e = launch_prolong(ac.b, af.b, L, yt, pt, usf, pf, false, s);
      if (e != cudaSuccess) return ASTERX_ECUDA;
      st = stage_given_ghosts(af, stage, 0.5 * dt, unf, usf, unxf, accf, pf, cnt, s);
      if (st != ASTERX_OK) return st;
    }
  }
  return cuda_status(launch_restrict(ac.b, af.b, L, unc, unf, s));
}

asterx_status asterx_rk2_step(const asterx_params* p, const asterx_block* blk, double dt, asterx_state* U,
                              asterx_prims* P, signed char* flags, asterx_c2p_stats* stats, void* ws,
                              size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || !set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P)) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  const long V = a.b.V;
  F9 un = f9(U), acc, mid;
  for (int v = 0; v < 9; v++) {
    acc.f[v] = a.w.uacc + v * V;  // unused by the RK2 combine
    mid.f[v] = a.w.ustage + v * V;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  st = stage_impl(a, 4, dt, un, un, mid, acc, f5(P), flags, cnt, s);  // U_1 = U_n + dt/2 L(U_n)
  if (st != ASTERX_OK) return st;
  return stage_impl(a, 5, dt, un, mid, un, acc, f5(P), flags, cnt, s);  // U_{n+1} = U_n + dt L(U_1)
}

asterx_status asterx_tmunu(const asterx_params* p, const asterx_block* blk, const asterx_metric* metric,
                           const asterx_state* U, const asterx_prims* P, asterx_tmunu_fields* T, void* ws,
                           size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_metric, 16>(metric) || !set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P) ||
      !set_ok<asterx_tmunu_fields, 10>(T))
    return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  CF16 m;
  std::memcpy(m.f, metric, sizeof(m.f));
  double* t[10];
  std::memcpy(t, T, sizeof(t));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = launch_bfield(a.b, a.w, f9(U), s);
  if (e == cudaSuccess) e = launch_uvel(a.b, a.w, f5(P), s);
  if (e == cudaSuccess) e = launch_tmunu(a.b, a.w, a.gamma, m, f5(P), t, s);
  return cuda_status(e);
}

asterx_status asterx_rk4_step_metrics(const asterx_params* p, const asterx_block* blk, double dt,
                                      const asterx_metric* const* metric, asterx_state* U, asterx_prims* P,
                                      signed char* flags, asterx_c2p_stats* stats, void* ws, size_t ws_bytes,
                                      asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || !set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P) || !metric)
    return ASTERX_EINVAL;
  for (int q = 0; q < 4; q++)
    if (!set_ok<asterx_metric, 16>(metric[q])) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  StageArgs a = make_args(p, blk, ws);
  const long V = a.b.V;
  F9 un = f9(U), acc, sb[2];
  for (int v = 0; v < 9; v++) {
    acc.f[v] = a.w.uacc + v * V;
    sb[0].f[v] = a.w.ustage + v * V;
    sb[1].f[v] = a.w.ustage + (9 + v) * V;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  for (int stage = 0; stage < 4; stage++) {
    CF16 m;
    std::memcpy(m.f, metric[stage], sizeof(m.f));
    if (launch_prepare(a.b, m, a.w, s) != cudaSuccess) return ASTERX_ECUDA;
    const F9& us = stage == 0 ? un : sb[(stage - 1) % 2];
    const F9& unext = stage == 3 ? un : sb[stage % 2];
    st = stage_impl(a, stage, dt, un, us, unext, acc, f5(P), flags, cnt, s);
    if (st != ASTERX_OK) return st;
  }
  return ASTERX_OK;
}

asterx_status asterx_rk4_step_host(const asterx_params* p, const asterx_block* blk, double dt,
                                   double* const* h_U9, double* const* h_P5, asterx_state* dU, asterx_prims* dP,
                                   asterx_c2p_stats* stats, void* ws, size_t ws_bytes, asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || !h_U9 || !h_P5 || !set_ok<asterx_state, 9>(dU) || !set_ok<asterx_prims, 5>(dP))
    return ASTERX_EINVAL;
  for (int v = 0; v < 9; v++)
    if (!h_U9[v]) return ASTERX_EINVAL;
  for (int v = 0; v < 5; v++)
    if (!h_P5[v]) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)padded_V(blk) * sizeof(double);
  F9 u = f9(dU);
  F5 pr = f5(dP);
  // one copy per run of fields that are consecutive on both sides (a stacked array is one copy)
  auto copy_fields = [&](double* const* dst, double* const* src, int nf, cudaMemcpyKind kind, cudaStream_t q) {
    for (int v = 0; v < nf;) {
      int e = v + 1;
      while (e < nf && dst[e] == dst[e - 1] + bytes / sizeof(double) && src[e] == src[e - 1] + bytes / sizeof(double))
        e++;
      if (cudaMemcpyAsync(dst[v], src[v], (size_t)(e - v) * bytes, kind, q) != cudaSuccess) return false;
      v = e;
    }
    return true;
  };
  // The primitives are final once the last stage's recovery has run (its right-hand side only reads them), so
  // their copy to the host runs on a second stream while that right-hand side and the state update run.
  cudaStream_t s2 = nullptr;
  cudaEvent_t prims_ready = nullptr;
  if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) return ASTERX_ECUDA;
  if (cudaEventCreateWithFlags(&prims_ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(s2);
    return ASTERX_ECUDA;
  }
  auto finish = [&](asterx_status r) {
    cudaStreamSynchronize(s2);
    cudaEventDestroy(prims_ready);
    cudaStreamDestroy(s2);
    return r;
  };
  if (!copy_fields(u.f, h_U9, 9, cudaMemcpyHostToDevice, s) ||
      !copy_fields(pr.f, h_P5, 5, cudaMemcpyHostToDevice, s))
    return finish(ASTERX_ECUDA);
  st = rk4_impl(p, blk, dt, dU, dP, nullptr, stats, ws, s, prims_ready);
  if (st != ASTERX_OK) return finish(st);
  if (cudaStreamWaitEvent(s2, prims_ready, 0) != cudaSuccess ||
      !copy_fields(h_P5, pr.f, 5, cudaMemcpyDeviceToHost, s2) ||
      !copy_fields(h_U9, u.f, 9, cudaMemcpyDeviceToHost, s))
    return finish(ASTERX_ECUDA);
  const cudaError_t e1 = cudaStreamSynchronize(s);
  const cudaError_t e2 = cudaStreamSynchronize(s2);
  return finish(cuda_status(e1 != cudaSuccess ? e1 : e2));
}

// ----------------------------------------------------------------------------------------------------------
// Batched step.  Pooled workspace layout: [4 stage tables of nb BlockRec | NKIND x (nb+1) item offsets |
// per-block workspaces, each on a 256-byte boundary].

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// header: 4 stage tables, the item offsets, then room for a tiling (struct and up to 3 (nb + 1) cut offsets)
static size_t batch_tiling_offset(int nb) {
  return round_up(4 * (size_t)nb * sizeof(BlockRec) + (size_t)NKIND * (nb + 1) * sizeof(long), 16);
}

static size_t batch_header_bytes(int nb) {
  return round_up(batch_tiling_offset(nb) + sizeof(Tiling) + 3 * (size_t)(nb + 1) * sizeof(int), kAlign);
}

static bool batch_blocks_ok(const asterx_batch_block* blocks, int nb) {
  if (!blocks || nb < 1 || nb > (1 << 20)) return false;
  for (int i = 0; i < nb; i++)
    if (!block_ok(&blocks[i].blk) || !set_ok<asterx_state, 9>(&blocks[i].U) ||
        !set_ok<asterx_prims, 5>(&blocks[i].P) || !set_ok<asterx_metric, 16>(&blocks[i].metric))
      return false;
  return true;
}

static size_t batch_bytes(const asterx_batch_block* blocks, int nb) {
  size_t tot = batch_header_bytes(nb);
  for (int i = 0; i < nb; i++) tot += round_up(ws_bytes_for(&blocks[i].blk), kAlign);
  return tot + kAlign;
}

// start of block i's workspace inside the pool
static char* block_ws(const asterx_batch_block* blocks, int nb, void* ws, int i) {
  size_t off = batch_header_bytes(nb);
  for (int q = 0; q < i; q++) off += round_up(ws_bytes_for(&blocks[q].blk), kAlign);
  return static_cast<char*>(ws) + off;
}

static asterx_status batch_checks(const asterx_params* p, const asterx_batch_block* blocks, int nb, void* ws,
                                  size_t ws_bytes) {
  if (!params_ok(p) || !batch_blocks_ok(blocks, nb)) return ASTERX_EINVAL;
  if (!ws || ((uintptr_t)ws % kAlign) != 0) return ASTERX_EINVAL;
  if (ws_bytes < batch_bytes(blocks, nb)) return ASTERX_ENOMEM;
  return ASTERX_OK;
}

static void batch_totals(const asterx_batch_block* blocks, int nb, long* totals, long* offsets /* may be null */) {
  for (int k = 0; k < NKIND; k++) {
    long acc = 0;
    for (int i = 0; i < nb; i++) {
      if (offsets) offsets[(long)k * (nb + 1) + i] = acc;
      acc += kind_count(k, make_blk(&blocks[i].blk));
    }
    if (offsets) offsets[(long)k * (nb + 1) + nb] = acc;
    totals[k] = acc;
  }
}

size_t asterx_batch_workspace_size(const asterx_batch_block* blocks, int nblocks) {
  if (!batch_blocks_ok(blocks, nblocks)) return 0;
  return batch_bytes(blocks, nblocks);
}

static asterx_status batch_prepare_impl(const asterx_params* p, const asterx_batch_block* blocks, int nblocks,
                                        const asterx_tiling* tl, void* ws, asterx_stream stream) {
  drop_graphs(ws);  // new tables: cached step graphs of this workspace no longer apply
  set_tiled(ws, tl != nullptr);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nb = nblocks;
  std::vector<BlockRec> tabs(4 * (size_t)nb);
  std::vector<long> offsets((size_t)NKIND * (nb + 1));
  long totals[NKIND];
  batch_totals(blocks, nb, totals, offsets.data());
  for (int i = 0; i < nb; i++) {
    const asterx_batch_block& bb = blocks[i];
    StageArgs a = make_args(p, &bb.blk, block_ws(blocks, nb, ws, i));
    CF16 m;
    std::memcpy(m.f, &bb.metric, sizeof(m.f));
    cudaError_t e = launch_prepare(a.b, m, a.w, s);
    if (e != cudaSuccess) return ASTERX_ECUDA;
    F9 u = f9(&bb.U), acc, sb[2];
    for (int v = 0; v < 9; v++) {
      acc.f[v] = a.w.uacc + v * a.b.V;
      sb[0].f[v] = a.w.ustage + v * a.b.V;
      sb[1].f[v] = a.w.ustage + (9 + v) * a.b.V;
    }
    if (tl) {  // position in the block grid; sides with a neighbour (or a periodic wrap) take exchanged ghosts
      const int c3[3] = {i % tl->nblk[0], (i / tl->nblk[0]) % tl->nblk[1], i / (tl->nblk[0] * tl->nblk[1])};
      for (int d = 0; d < 3; d++) {
        a.b.coord[d] = c3[d];
        a.b.off[d] = tl->cuts[d][c3[d]];
        if (c3[d] > 0 || a.b.bc[d] == ASTERX_BC_PERIODIC) a.b.halo |= 1 << (2 * d);
        if (c3[d] < tl->nblk[d] - 1 || a.b.bc[d] == ASTERX_BC_PERIODIC) a.b.halo |= 1 << (2 * d + 1);
      }
    }
    for (int stage = 0; stage < 4; stage++) {
      BlockRec& r = tabs[(size_t)stage * nb + i];
      std::memset(&r, 0, sizeof(r));
      r.b = a.b;
      r.w = a.w;
      r.Un = u;
      r.Us = stage == 0 ? u : sb[(stage - 1) % 2];
      r.Unext = stage == 3 ? u : sb[stage % 2];
      r.Uacc = acc;
      r.dU = r.Unext;
      r.P = f5(&bb.P);
      r.flags = nullptr;
    }
  }
  char* hdr = static_cast<char*>(ws);
  cudaError_t e = cudaMemcpyAsync(hdr, tabs.data(), tabs.size() * sizeof(BlockRec), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hdr + 4 * (size_t)nb * sizeof(BlockRec), offsets.data(), offsets.size() * sizeof(long),
                        cudaMemcpyHostToDevice, s);
  std::vector<char> tbuf;
  if (tl && e == cudaSuccess) {
    Tiling t;
    int at = 0;
    for (int d = 0; d < 3; d++) {
      t.nblk[d] = tl->nblk[d];
      t.ntot[d] = tl->cuts[d][tl->nblk[d]];
      t.bc[d] = blocks[0].blk.bc[d];
      t.cut_at[d] = at;
      at += tl->nblk[d] + 1;
    }
    tbuf.resize(sizeof(Tiling) + (size_t)at * sizeof(int));
    std::memcpy(tbuf.data(), &t, sizeof(t));
    int* cuts = reinterpret_cast<int*>(tbuf.data() + sizeof(Tiling));
    for (int d = 0; d < 3; d++)
      for (int q = 0; q <= tl->nblk[d]; q++) cuts[t.cut_at[d] + q] = tl->cuts[d][q];
    e = cudaMemcpyAsync(hdr + batch_tiling_offset(nb), tbuf.data(), tbuf.size(), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables go out of scope
  return cuda_status(e);
}

asterx_status asterx_batch_prepare(const asterx_params* p, const asterx_batch_block* blocks, int nblocks,
                                   void* ws, size_t ws_bytes, asterx_stream stream) {
  asterx_status st = batch_checks(p, blocks, nblocks, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  return batch_prepare_impl(p, blocks, nblocks, nullptr, ws, stream);
}

// the blocks tile one domain: nblk[0] nblk[1] nblk[2] blocks listed x fastest, each block's interior the cells
// between consecutive cuts, common spacing and boundary conditions, origins consistent with the cuts
static bool tiling_ok(const asterx_batch_block* blocks, int nb, const asterx_tiling* t) {
  if (!t) return false;
  long count = 1;
  for (int d = 0; d < 3; d++) {
    if (t->nblk[d] < 1 || !t->cuts[d] || t->cuts[d][0] != 0) return false;
    for (int q = 0; q < t->nblk[d]; q++)
      if (t->cuts[d][q + 1] - t->cuts[d][q] < blocks[0].blk.g) return false;  // at least g cells per block
    count *= t->nblk[d];
  }
  if (count != nb) return false;
  for (int i = 0; i < nb; i++) {
    const asterx_block& b = blocks[i].blk;
    const int c3[3] = {i % t->nblk[0], (i / t->nblk[0]) % t->nblk[1], i / (t->nblk[0] * t->nblk[1])};
    for (int d = 0; d < 3; d++) {
      if (b.n[d] != t->cuts[d][c3[d] + 1] - t->cuts[d][c3[d]]) return false;
      if (b.dx[d] != blocks[0].blk.dx[d] || b.bc[d] != blocks[0].blk.bc[d]) return false;
      const double x0 = blocks[0].blk.x0[d] + t->cuts[d][c3[d]] * b.dx[d];
      if (std::fabs(b.x0[d] - x0) > 1e-9 * b.dx[d]) return false;
    }
  }
  return true;
}

asterx_status asterx_batch_prepare_tiled(const asterx_params* p, const asterx_batch_block* blocks, int nblocks,
                                         const asterx_tiling* tiling, void* ws, size_t ws_bytes,
                                         asterx_stream stream) {
  asterx_status st = batch_checks(p, blocks, nblocks, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!tiling_ok(blocks, nblocks, tiling)) return ASTERX_EINVAL;
  return batch_prepare_impl(p, blocks, nblocks, tiling, ws, stream);
}

asterx_status asterx_batch_prim2con(const asterx_params* p, const asterx_batch_block* blocks, int nblocks,
                                    void* ws, size_t ws_bytes, asterx_stream stream) {
  asterx_status st = batch_checks(p, blocks, nblocks, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool tiled = is_tiled(ws);
  if (tiled) {  // the potentials' ghosts from the neighbouring blocks (stage-0 records: U_s = U)
    long totals[NKIND];
    batch_totals(blocks, nblocks, totals, nullptr);
    const BlockRec* tab = reinterpret_cast<const BlockRec*>(ws);
    const long* off =
        reinterpret_cast<const long*>(static_cast<char*>(ws) + 4 * (size_t)nblocks * sizeof(BlockRec));
    const Tiling* til = reinterpret_cast<const Tiling*>(static_cast<char*>(ws) + batch_tiling_offset(nblocks));
    if (launch_batch_ghosts(tab, off, totals, nblocks, til, s) != cudaSuccess) return ASTERX_ECUDA;
  }
  for (int i = 0; i < nblocks; i++) {
    StageArgs a = make_args(p, &blocks[i].blk, block_ws(blocks, nblocks, ws, i));
    F9 u = f9(&blocks[i].U);
    cudaError_t e = tiled ? cudaSuccess : launch_ghost_state(a.b, u, s);
    if (e == cudaSuccess) e = launch_bfield(a.b, a.w, u, s);
    if (e == cudaSuccess) e = launch_prim2con(a, u, f5(&blocks[i].P), s);
    if (e != cudaSuccess) return ASTERX_ECUDA;
  }
  return ASTERX_OK;
}


asterx_status asterx_batch_release(void* ws) {
  if (!ws) return ASTERX_EINVAL;
  drop_graphs(ws);
  set_tiled(ws, false);
  return ASTERX_OK;
}

asterx_status asterx_batched_step(const asterx_params* p, const asterx_batch_block* blocks, int nblocks, double dt,
                                  int nsteps, asterx_c2p_stats* stats, void* ws, size_t ws_bytes,
                                  asterx_stream stream) {
  asterx_status st = batch_checks(p, blocks, nblocks, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || nsteps < 0) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;
  const int nb = nblocks;
  long totals[NKIND];
  batch_totals(blocks, nb, totals, nullptr);
  // the stage-independent parameters are those of the first block's arguments (the same params for all)
  StageArgs a = make_args(p, &blocks[0].blk, block_ws(blocks, nb, ws, 0));
  const BlockRec* tab = reinterpret_cast<const BlockRec*>(ws);
  const long* off = reinterpret_cast<const long*>(static_cast<char*>(ws) + 4 * (size_t)nb * sizeof(BlockRec));
  const Tiling* til =
      is_tiled(ws) ? reinterpret_cast<const Tiling*>(static_cast<char*>(ws) + batch_tiling_offset(nb)) : nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(stats);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  int first = 0;  // steps launched directly
  if (nsteps > 0 && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
    if (!cached_graph(p, ws, totals, nb, dt, cnt)) {
      // the first step of new launch parameters runs directly, which lets the launch autotuner time its
      // kernels on the live data; the graph captured after it bakes in the chosen launch shapes
      for (int stage = 0; stage < 4; stage++) {
        cudaError_t e = launch_batch_stage(a, tab + (size_t)stage * nb, off, totals, nb, stage, dt, cnt, s, til);
        if (e != cudaSuccess) return ASTERX_ECUDA;
      }
      first = 1;
    }
    cudaGraphExec_t exec = step_graph(a, p, ws, tab, off, totals, nb, dt, cnt, til);
    if (exec) {
      for (int step = first; step < nsteps; step++)
        if (cudaGraphLaunch(exec, s) != cudaSuccess) return ASTERX_ECUDA;
      return ASTERX_OK;
    }
  }
  for (int step = first; step < nsteps; step++)
    for (int stage = 0; stage < 4; stage++) {
      cudaError_t e = launch_batch_stage(a, tab + (size_t)stage * nb, off, totals, nb, stage, dt, cnt, s, til);
      if (e != cudaSuccess) return ASTERX_ECUDA;
    }
  return ASTERX_OK;
}

// ----------------------------------------------------------------------------------------------------------
// Adjoint.  Adjoint workspace: RK4 stage states Y0..Y3 (36 fields), forward accumulator (9), running adjoint
// lambda (9), stage adjoint kbar (9), sum (9), the right-hand-side adjoint accumulators (ADJ_ACC_FIELDS),
// reconstructed-value adjoints (2 NREC), a state copy (9), and the kept forward intermediates of the four stages
// (4 KEEP_FIELDS: recovered primitives and flags, B~ and B, u, face data, reconstruction, roots).

namespace {
constexpr int ADJ_BASE_FIELDS = 36 + 9 + 9 + 9 + 9 + ADJ_ACC_FIELDS + 2 * NREC + 9;
constexpr int ADJ_FIELDS = ADJ_BASE_FIELDS + 4 * KEEP_FIELDS;

struct Keep {
  F5 P;
  signed char* flags;
  double *bf, *bc, *uvel, *face, *rec3[3], *roots;
};

struct AdjLayout {
  F9 Ys[4], acc, lam, kbar, sum, ycopy;
  double* accum;
  double* lrec;
  Keep keep[4];
};

size_t adj_bytes_for(const asterx_block* b) {
  const long V = padded_V(b);
  const long fs = field_stride(V);
  return (size_t)ADJ_FIELDS * fs * sizeof(double) + kAlign;
}

AdjLayout make_adj(const asterx_block* in, void* base) {
  const long V = padded_V(in);
  const long fs = field_stride(V);
  double* p = reinterpret_cast<double*>(base);
  auto take = [&](int nf) {
    double* q = p;
    p += (long)nf * fs;
    return q;
  };
  auto take9 = [&]() {
    F9 f;
    double* q = take(9);
    for (int v = 0; v < 9; v++) f.f[v] = q + v * V;
    return f;
  };
  AdjLayout L;
  for (int s = 0; s < 4; s++) L.Ys[s] = take9();
  L.acc = take9();
  L.lam = take9();
  L.kbar = take9();
  L.sum = take9();
  L.accum = take(ADJ_ACC_FIELDS);
  L.lrec = take(2 * NREC);
  L.ycopy = take9();
  for (int s = 0; s < 4; s++) {
    Keep& k = L.keep[s];
    double* q = take(5);
    for (int v = 0; v < 5; v++) k.P.f[v] = q + v * V;
    k.bf = take(3);
    k.bc = take(3);
    k.uvel = take(3);
    k.face = take(3 * NFD);
    for (int d = 0; d < 3; d++) k.rec3[d] = take(2 * NREC);
    k.roots = take(12);
    k.flags = reinterpret_cast<signed char*>(take(1));
  }
  return L;
}

// the adjoint arguments of one stage: state Y, weights mu, the kept intermediates of stage `ks`
AdjWs adj_ws(const AdjLayout& L, const Blk& b, const F9& Y, int ks, const F9& mu) {
  AdjWs a;
  const Keep& k = L.keep[ks];
  a.Y = Y;
  a.mu = mu;
  a.P = k.P;
  a.flags = k.flags;
  a.kbf = k.bf;
  a.kbc = k.bc;
  a.kuvel = k.uvel;
  a.kface = k.face;
  for (int d = 0; d < 3; d++) a.rec3[d] = k.rec3[d];
  a.roots = k.roots;
  double* q = L.accum;
  a.lY_base = q;
  a.lY = q; q += 9 * b.V;
  a.lP = q; q += 5 * b.V;
  a.lu = q; q += 3 * b.V;
  a.lBc = q; q += 3 * b.V;
  a.lBf = q; q += 3 * b.V;
  a.lface = q; q += 3L * NFD * b.V;
  a.lGA = q; q += b.V;
  a.lFpsi = q; q += 3 * b.V;
  a.lAv = q;
  a.lrec = L.lrec;
  return a;
}

F9 f9_from(double* base, long V) {
  F9 f;
  for (int v = 0; v < 9; v++) f.f[v] = base + v * V;
  return f;
}

cudaError_t copy9(const F9& dst, const F9& src, long V, cudaStream_t s) {
  for (int v = 0; v < 9; v++) {
    cudaError_t e = cudaMemcpyAsync(dst.f[v], src.f[v], V * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t copy5(const F5& dst, const F5& src, long V, cudaStream_t s) {
  for (int v = 0; v < 5; v++) {
    cudaError_t e = cudaMemcpyAsync(dst.f[v], src.f[v], V * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

size_t asterx_adjoint_workspace_size(const asterx_block* blk) {
  if (!block_ok(blk)) return 0;
  return adj_bytes_for(blk);
}

static asterx_status adj_checks(const asterx_params* p, const asterx_block* blk, double dt, void* ws,
                                size_t ws_bytes, void* aws, size_t aws_bytes) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt)) return ASTERX_EINVAL;
  if (!aws || ((uintptr_t)aws % kAlign) != 0) return ASTERX_EINVAL;
  if (aws_bytes < adj_bytes_for(blk)) return ASTERX_ENOMEM;
  return ASTERX_OK;
}


asterx_status asterx_rhs_adjoint(const asterx_params* p, const asterx_block* blk, double dt, const asterx_state* U,
                                 asterx_prims* P, const asterx_state* mu, asterx_state* lam, void* ws,
                                 size_t ws_bytes, void* aws, size_t aws_bytes, asterx_stream stream) {
  asterx_status st = adj_checks(p, blk, dt, ws, ws_bytes, aws, aws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P) || !set_ok<asterx_state, 9>(mu) ||
      !set_ok<asterx_state, 9>(lam))
    return ASTERX_EINVAL;
  StageArgs sa = make_args(p, blk, ws);
  AdjLayout L = make_adj(blk, aws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long V = sa.b.V;
  cudaError_t e = copy9(L.ycopy, f9(U), V, s);
  if (e == cudaSuccess) e = copy9(L.kbar, f9(mu), V, s);
  if (e == cudaSuccess) e = launch_mask_owned9(sa.b, L.kbar, s);
  if (e == cudaSuccess) e = copy5(L.keep[0].P, f5(P), V, s);  // the recovery's guess
  AdjWs a = adj_ws(L, sa.b, L.ycopy, 0, L.kbar);
  if (e == cudaSuccess) e = launch_rhs_adjoint(sa, a, dt, s);
  if (e == cudaSuccess) e = copy9(f9(lam), f9_from(a.lY, V), V, s);
  if (e == cudaSuccess) e = copy5(f5(P), L.keep[0].P, V, s);
  return cuda_status(e);
}

asterx_status asterx_rk_stage_adjoint(const asterx_params* p, const asterx_block* blk, int stage, double dt,
                                      const asterx_state* Us, asterx_prims* P, const asterx_state* lam_next,
                                      const asterx_state* lam_acc, asterx_state* lam_s, void* ws, size_t ws_bytes,
                                      void* aws, size_t aws_bytes, asterx_stream stream) {
  asterx_status st = adj_checks(p, blk, dt, ws, ws_bytes, aws, aws_bytes);
  if (st != ASTERX_OK) return st;
  if (stage < 0 || stage > 3) return ASTERX_EINVAL;
  if (!set_ok<asterx_state, 9>(Us) || !set_ok<asterx_prims, 5>(P) || !set_ok<asterx_state, 9>(lam_next) ||
      !set_ok<asterx_state, 9>(lam_s) || (stage < 3 && !set_ok<asterx_state, 9>(lam_acc)))
    return ASTERX_EINVAL;
  StageArgs sa = make_args(p, blk, ws);
  const Blk& b = sa.b;
  AdjLayout L = make_adj(blk, aws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // kbar = c dt lam_next + b dt lam_acc (stages 0..2), dt/6 lam_next (stage 3)
  const double c[3] = {0.5, 0.5, 1.0}, w[3] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0};
  cudaError_t e = copy9(L.kbar, f9(lam_next), b.V, s);
  if (e == cudaSuccess && stage < 3) {
    e = copy9(L.lam, f9(lam_acc), b.V, s);
    if (e == cudaSuccess) e = launch_axpby9(b, w[stage] * dt, L.lam, c[stage] * dt, L.kbar, s);
  } else if (e == cudaSuccess) {
    e = launch_axpby9(b, 0.0, L.kbar, dt / 6.0, L.kbar, s);
  }
  if (e == cudaSuccess) e = launch_mask_owned9(b, L.kbar, s);
  if (e == cudaSuccess) e = copy9(L.ycopy, f9(Us), b.V, s);
  if (e == cudaSuccess) e = copy5(L.keep[0].P, f5(P), b.V, s);
  AdjWs a = adj_ws(L, b, L.ycopy, 0, L.kbar);
  if (e == cudaSuccess) e = launch_rhs_adjoint(sa, a, dt, s);
  if (e == cudaSuccess) e = copy9(f9(lam_s), f9_from(a.lY, b.V), b.V, s);
  if (e == cudaSuccess) e = copy5(f5(P), L.keep[0].P, b.V, s);
  return cuda_status(e);
}

asterx_status asterx_rk4_step_adjoint(const asterx_params* p, const asterx_block* blk, double dt,
                                      const asterx_state* Un, asterx_prims* P, asterx_state* lam, void* ws,
                                      size_t ws_bytes, void* aws, size_t aws_bytes, asterx_stream stream) {
  asterx_status st = adj_checks(p, blk, dt, ws, ws_bytes, aws, aws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(Un) || !set_ok<asterx_prims, 5>(P) || !set_ok<asterx_state, 9>(lam))
    return ASTERX_EINVAL;
  StageArgs sa = make_args(p, blk, ws);
  const Blk& b = sa.b;
  AdjLayout L = make_adj(blk, aws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // forward pass from the checkpoint, keeping each stage's intermediates: the stage states Y0..Y3 and, per
  // stage, the recovery, face data and reconstruction (the recovery's guess carries from stage to stage)
  cudaError_t e = copy9(L.Ys[0], f9(Un), b.V, s);
  if (e == cudaSuccess) e = copy5(L.keep[0].P, f5(P), b.V, s);
  for (int stage = 0; stage < 4 && e == cudaSuccess; stage++) {
    AdjWs a = adj_ws(L, b, L.Ys[stage], stage, L.kbar);
    if (stage > 0) e = copy5(L.keep[stage].P, L.keep[stage - 1].P, b.V, s);
    if (e == cudaSuccess) e = launch_adjoint_forward(sa, a, s);
    if (stage < 3 && e == cudaSuccess)
      e = launch_rhs_from_kept(sa, a, stage, dt, L.Ys[0], L.Ys[stage + 1], L.acc, L.Ys[stage + 1], s);
  }
  // reverse sweep: kbar_3 = dt/6 lam, Ybar_s = J_s^T kbar_s, kbar_{s-1} = b_{s-1} dt lam + c_s dt Ybar_s
  if (e == cudaSuccess) e = copy9(L.lam, f9(lam), b.V, s);
  if (e == cudaSuccess) e = launch_mask_owned9(b, L.lam, s);
  if (e == cudaSuccess) e = copy9(L.sum, L.lam, b.V, s);
  if (e == cudaSuccess) e = copy9(L.kbar, L.lam, b.V, s);
  if (e == cudaSuccess) e = launch_axpby9(b, 0.0, L.lam, dt / 6.0, L.kbar, s);
  const double blam[3] = {dt / 6.0, dt / 3.0, dt / 3.0};  // weight of lam in kbar_{s}, s = 0, 1, 2
  const double cy[3] = {0.5 * dt, 0.5 * dt, dt};          // weight of Ybar_{s+1} in kbar_{s}
  for (int stage = 3; stage >= 0 && e == cudaSuccess; stage--) {
    AdjWs a = adj_ws(L, b, L.Ys[stage], stage, L.kbar);
    e = launch_adjoint_reverse(sa, a, dt, s);
    const F9 ybar = f9_from(a.lY, b.V);
    if (e == cudaSuccess) e = launch_axpby9(b, 1.0, ybar, 1.0, L.sum, s);
    if (stage > 0 && e == cudaSuccess) {
      // kbar_{stage-1} = blam * lam + cy * ybar
      e = copy9(L.kbar, ybar, b.V, s);
      if (e == cudaSuccess) e = launch_axpby9(b, blam[stage - 1], L.lam, cy[stage - 1], L.kbar, s);
    }
  }
  if (e == cudaSuccess) e = copy9(f9(lam), L.sum, b.V, s);
  if (e == cudaSuccess) e = copy5(f5(P), L.keep[0].P, b.V, s);
  return cuda_status(e);
}

asterx_status asterx_prim2con_adjoint(const asterx_params* p, const asterx_block* blk, const asterx_state* U,
                                      const asterx_prims* P, asterx_state* lam, asterx_prims* lamP, void* ws,
                                      size_t ws_bytes, void* aws, size_t aws_bytes, asterx_stream stream) {
  asterx_status st = adj_checks(p, blk, 1.0, ws, ws_bytes, aws, aws_bytes);
  if (st != ASTERX_OK) return st;
  if (!set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P) || !set_ok<asterx_state, 9>(lam) ||
      !set_ok<asterx_prims, 5>(lamP))
    return ASTERX_EINVAL;
  StageArgs sa = make_args(p, blk, ws);
  AdjLayout L = make_adj(blk, aws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = copy9(L.ycopy, f9(U), sa.b.V, s);
  if (e == cudaSuccess) e = copy9(L.kbar, f9(lam), sa.b.V, s);
  if (e == cudaSuccess) e = launch_mask_owned9(sa.b, L.kbar, s);
  if (e == cudaSuccess) e = copy5(L.keep[0].P, f5(P), sa.b.V, s);
  AdjWs a = adj_ws(L, sa.b, L.ycopy, 0, L.kbar);
  if (e == cudaSuccess) e = launch_prim2con_adjoint(sa, a, L.kbar, f5(lamP), s);
  if (e == cudaSuccess) e = copy9(f9(lam), f9_from(a.lY, sa.b.V), sa.b.V, s);
  return cuda_status(e);
}

asterx_status asterx_rk4_steps_checkpointed(const asterx_params* p, const asterx_block* blk, double dt, int nsteps,
                                            asterx_state* U, asterx_prims* P, const asterx_state* ckpt,
                                            asterx_c2p_stats* stats, void* ws, size_t ws_bytes,
                                            asterx_stream stream) {
  asterx_status st = common_checks(p, blk, ws, ws_bytes);
  if (st != ASTERX_OK) return st;
  if (!finite_pos(dt) || nsteps < 1 || !ckpt || !set_ok<asterx_state, 9>(U) || !set_ok<asterx_prims, 5>(P))
    return ASTERX_EINVAL;
  for (int k = 0; k < nsteps; k++)
    if (!set_ok<asterx_state, 9>(&ckpt[k])) return ASTERX_EINVAL;
  const long V = padded_V(blk);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int k = 0; k < nsteps; k++) {
    if (copy9(f9(&ckpt[k]), f9(U), V, s) != cudaSuccess) return ASTERX_ECUDA;
    st = asterx_rk4_step(p, blk, dt, U, P, nullptr, stats, ws, ws_bytes, stream);
    if (st != ASTERX_OK) return st;
  }
  return ASTERX_OK;
}

asterx_status asterx_rk4_adjoint_steps(const asterx_params* p, const asterx_block* blk, double dt, int nsteps,
                                       const asterx_state* ckpt, asterx_prims* P, asterx_state* lam, void* ws,
                                       size_t ws_bytes, void* aws, size_t aws_bytes, asterx_stream stream) {
  asterx_status st = adj_checks(p, blk, dt, ws, ws_bytes, aws, aws_bytes);
  if (st != ASTERX_OK) return st;
  if (nsteps < 1 || !ckpt) return ASTERX_EINVAL;
  for (int k = 0; k < nsteps; k++)
    if (!set_ok<asterx_state, 9>(&ckpt[k])) return ASTERX_EINVAL;
  for (int k = nsteps - 1; k >= 0; k--) {
    st = asterx_rk4_step_adjoint(p, blk, dt, &ckpt[k], P, lam, ws, ws_bytes, aws, aws_bytes, stream);
    if (st != ASTERX_OK) return st;
  }
  return ASTERX_OK;
}

asterx_status asterx_profile_enable(int max_launches) {
  if (max_launches < 1 || max_launches > (1 << 20)) return ASTERX_EINVAL;
  return cuda_status(profile_enable(max_launches));
}

asterx_status asterx_profile_read(int* launches, double* total_ms) {
  if (!launches || !total_ms) return ASTERX_EINVAL;
  return cuda_status(profile_read(launches, total_ms));
}

void asterx_profile_disable(void) { profile_disable(); }

asterx_status asterx_dfma_probe(double* out, int blocks, int threads, long iters, asterx_stream stream) {
  if (!ptr_ok(out) || blocks < 1 || threads < 32 || threads > 1024 || (threads % 32) != 0 || iters < 1)
    return ASTERX_EINVAL;
  return cuda_status(launch_dfma_probe(out, blocks, threads, iters, reinterpret_cast<cudaStream_t>(stream)));
}

asterx_status asterx_newton_rcp(const double* d, double* out, long n, asterx_stream stream) {
  if (n < 0 || (n > 0 && (!ptr_ok(d) || !ptr_ok(out)))) return ASTERX_EINVAL;
  if (n == 0) return ASTERX_OK;
  return cuda_status(launch_newton_rcp(d, out, n, reinterpret_cast<cudaStream_t>(stream)));
}

asterx_status asterx_quotient(const double* a, const double* b, double* out, long n, asterx_stream stream) {
  if (n < 0 || (n > 0 && (!ptr_ok(a) || !ptr_ok(b) || !ptr_ok(out)))) return ASTERX_EINVAL;
  if (n == 0) return ASTERX_OK;
  return cuda_status(launch_quotient(a, b, out, n, reinterpret_cast<cudaStream_t>(stream)));
}

asterx_status asterx_recip(const double* d, double* out, long n, asterx_stream stream) {
  if (n < 0 || (n > 0 && (!ptr_ok(d) || !ptr_ok(out)))) return ASTERX_EINVAL;
  if (n == 0) return ASTERX_OK;
  return cuda_status(launch_recip(d, out, n, reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
