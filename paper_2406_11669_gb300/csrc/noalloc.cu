// Primitive recovery without any device allocation by the caller or the library: the scratch memory the
// recovery needs (centre geometry, face field, centre field) lives in one fixed-size array in the library's
// own device memory.  See asterx_con2prim_noalloc in include/asterx.h for who needs this and its limits.
#include <cuda.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/asterx.h"
#include "kernels.h"
#include "validate.h"

using namespace asterx;

namespace {

constexpr long kMaxEntries = ASTERX_NOALLOC_MAX_ENTRIES;  // padded entries per field
constexpr int kFields = NCG + 3 + 3;                       // centre record, face B~, centre B

// Shared by every call on a device and kept until the process exits.  In host code this name is only a
// stand-in for the device symbol: its device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) double g_noalloc_scratch[(long)kFields * kMaxEntries];

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  unsigned long long ctx_id;  // the CUDA context the address belongs to (0: not looked up yet)
  double* ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the current context, through the driver entry points the runtime hands out (the library
// links no driver library).  A device reset ends the context; the next one has a new id.
cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f = nullptr;
    void* g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f) return e != cudaSuccess ? e : cudaErrorUnknown;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !g) return e != cudaSuccess ? e : cudaErrorUnknown;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    get_id = reinterpret_cast<CtxGetIdFn>(g);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array on the current device.  It is looked up (cudaGetSymbolAddress, which
// also creates the device's context if the process has none yet) on the first call on each device and again
// whenever the device's context has changed since, e.g. after the host application reset the device.  If the
// context cannot be identified, the address is looked up on every call.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned long long id = 0;
  const bool known = g_scratch_addr[dev].ctx_id != 0 && current_context_id(&id) == cudaSuccess &&
                     id == g_scratch_addr[dev].ctx_id;
  if (!known) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev].ctx_id = (current_context_id(&id) == cudaSuccess) ? id : 0;
    g_scratch_addr[dev].ptr = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev].ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" asterx_status asterx_con2prim_noalloc(const asterx_params* p, const asterx_block* blk,
                                                 const asterx_metric* metric, asterx_state* U, asterx_prims* P,
                                                 signed char* flags, asterx_c2p_stats* stats,
                                                 asterx_stream stream) {
  // argument checks: the same rules as the workspace entry points, then the size of the fixed array
  if (!check::params_ok(p) || !check::block_ok(blk)) return ASTERX_EINVAL;
  const long V = check::padded_volume(blk);  // bounded factors: each n + 7 <= 2^20 + 7, product < 4e9
  if (V > kMaxEntries) return ASTERX_EINVAL;  // the block does not fit the fixed scratch array
  if (!metric || !check::set_ok<asterx_metric, 16>(metric) || !check::set_ok<asterx_state, 9>(U) ||
      !check::set_ok<asterx_prims, 5>(P))
    return ASTERX_EINVAL;
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
