// Primitive recovery without any device allocation by the caller or the library: the scratch memory the
// recovery needs (centre geometry, face field, centre field) lives in one fixed-size array in the library's
// own device memory.  See asterx_con2prim_noalloc in include/asterx.h for who needs this and its limits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/asterx.h"
#include "kernels.h"

using namespace asterx;

namespace {

constexpr long kMaxEntries = ASTERX_NOALLOC_MAX_ENTRIES;  // padded entries per field
constexpr int kFields = NCG + 3 + 3;                       // centre record, face B~, centre B

// Shared by every call on a device and kept until the process exits.  In host code this name is only a
// stand-in for the device symbol: its device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) double g_noalloc_scratch[(long)kFields * kMaxEntries];

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }
bool aligned8(const void* q) { return q && ((uintptr_t)q % 8 == 0); }

}  // namespace

extern "C" asterx_status asterx_con2prim_noalloc(const asterx_params* p, const asterx_block* blk,
                                                 const asterx_metric* metric, asterx_state* U, asterx_prims* P,
                                                 signed char* flags, asterx_c2p_stats* stats,
                                                 asterx_stream stream) {
  // argument checks (the same rules as the workspace entry points)
  if (!p || !blk || !metric || !U || !P) return ASTERX_EINVAL;
  if (!(std::isfinite(p->gamma) && p->gamma > 1.0) || !finite_pos(p->rho_atm) || !(p->K_atm >= 0.0) ||
      !(p->gamma_atm > 1.0) || !finite_pos(p->c2p_tol) || p->c2p_maxiter < 1 || p->brent_maxiter < 1 ||
      !(p->W_max > 1.0) || (p->use_fallback != 0 && p->use_fallback != 1))
    return ASTERX_EINVAL;
  if (blk->g != 3) return ASTERX_EINVAL;
  long V = 1;
  for (int d = 0; d < 3; d++) {
    if (blk->n[d] < 1 || !finite_pos(blk->dx[d]) || (blk->bc[d] != 0 && blk->bc[d] != 1)) return ASTERX_EINVAL;
    V *= (long)(blk->n[d] + 2 * blk->g + 1);
  }
  if (V > kMaxEntries) return ASTERX_EINVAL;  // the block does not fit the fixed scratch array
  const double* const* mf = reinterpret_cast<const double* const*>(metric);
  for (int f = 0; f < 16; f++)
    if (!aligned8(mf[f])) return ASTERX_EINVAL;
  double* const* uf = reinterpret_cast<double* const*>(U);
  for (int f = 0; f < 9; f++)
    if (!aligned8(uf[f])) return ASTERX_EINVAL;
  double* const* pf = reinterpret_cast<double* const*>(P);
  for (int f = 0; f < 5; f++)
    if (!aligned8(pf[f])) return ASTERX_EINVAL;
  if (stats && ((uintptr_t)stats % 8) != 0) return ASTERX_EINVAL;

  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return ASTERX_ECUDA;

  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.b.g = blk->g;
  for (int d = 0; d < 3; d++) {
    a.b.n[d] = blk->n[d];
    a.b.N[d] = blk->n[d] + 2 * blk->g;
    a.b.bc[d] = blk->bc[d];
    a.b.dx[d] = blk->dx[d];
    a.b.idx[d] = 1.0 / blk->dx[d];
  }
  a.b.sy = a.b.N[0] + 1;
  a.b.sz = (long)(a.b.N[0] + 1) * (a.b.N[1] + 1);
  a.b.V = V;
  // scratch layout: centre record (NCG fields), face B~ (3), centre B (3), each field at pitch V.  Every
  // entry the recovery reads is written earlier in the same call, so nothing needs clearing.
  a.w.cg = base;
  a.w.bf = base + (long)NCG * V;
  a.w.bc = base + (long)(NCG + 3) * V;
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
  a.recon = p->recon;
  a.gauge = p->gauge;

  CF16 m;
  std::memcpy(m.f, metric, sizeof(m.f));
  F9 u;
  std::memcpy(u.f, U, sizeof(u.f));
  F5 pr;
  std::memcpy(pr.f, P, sizeof(pr.f));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = launch_prepare_centre(a.b, m, a.w.cg, s);
  if (e == cudaSuccess) e = launch_bfield(a.b, a.w, u, s);
  if (e == cudaSuccess) e = launch_c2p(a, u, pr, flags, reinterpret_cast<unsigned long long*>(stats), s);
  return e == cudaSuccess ? ASTERX_OK : ASTERX_ECUDA;
}
