// Host-side argument checks shared by every entry point of the C ABI (include/asterx.h): each call rejects
// invalid arguments with ASTERX_EINVAL before it launches anything.
#pragma once
#include <cmath>
#include <cstdint>

#include "../../include/asterx.h"

namespace asterx {
namespace check {

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// A block: 3 ghost layers, 1..2^20 interior cells per axis, positive finite spacing, finite origin, a known
// boundary condition per axis, and a padded volume (n + 7)^3 below 4e9 entries (32-bit item arithmetic).
inline bool block_ok(const asterx_block* b) {
  if (!b) return false;
  if (b->g != 3) return false;
  for (int d = 0; d < 3; d++) {
    if (b->n[d] < 1 || b->n[d] > (1 << 20)) return false;
    if (!finite_pos(b->dx[d]) || !std::isfinite(b->x0[d])) return false;
    if (b->bc[d] != ASTERX_BC_PERIODIC && b->bc[d] != ASTERX_BC_COPY) return false;
  }
  const double V = (double)(b->n[0] + 7) * (b->n[1] + 7) * (b->n[2] + 7);
  return V < 4.0e9;
}

// Padded entries per field, (n + 2g + 1) per axis; only for blocks that passed block_ok.
inline long padded_volume(const asterx_block* b) {
  long V = 1;
  for (int d = 0; d < 3; d++) V *= (long)(b->n[d] + 2 * b->g + 1);
  return V;
}

inline bool params_ok(const asterx_params* p) {
  if (!p) return false;
  if (!(std::isfinite(p->gamma) && p->gamma > 1.0)) return false;
  if (!finite_pos(p->rho_atm) || !(std::isfinite(p->K_atm) && p->K_atm >= 0.0)) return false;
  if (!(std::isfinite(p->gamma_atm) && p->gamma_atm > 1.0)) return false;
  if (!finite_pos(p->c2p_tol) || p->c2p_maxiter < 1 || p->brent_maxiter < 1) return false;
  if (!(std::isfinite(p->W_max) && p->W_max > 1.0)) return false;
  if (p->recon < ASTERX_RECON_MINMOD || p->recon > ASTERX_RECON_MP5) return false;
  if (p->gauge != ASTERX_GAUGE_LORENZ && p->gauge != ASTERX_GAUGE_ALGEBRAIC) return false;
  if (!(std::isfinite(p->xi_lorenz) && p->xi_lorenz >= 0.0)) return false;
  if (p->flux != ASTERX_FLUX_HLLE && p->flux != ASTERX_FLUX_LXF) return false;
  if (p->efield != ASTERX_EFIELD_UCT && p->efield != ASTERX_EFIELD_FCT) return false;
  return p->use_fallback == 0 || p->use_fallback == 1;
}

inline bool ptr_ok(const void* q) { return q && ((uintptr_t)q % 8 == 0); }

// every pointer of a struct of N double pointers is non-null and 8-byte aligned
template <class S, int N>
bool set_ok(const S* s) {
  if (!s) return false;
  const double* const* f = reinterpret_cast<const double* const*>(s);
  for (int i = 0; i < N; i++)
    if (!ptr_ok(f[i])) return false;
  return true;
}

}  // namespace check
}  // namespace asterx
