// Two refinement levels (the fixed BoxInBox refinement of Sec. 3.9, with the prolongation the AMR
// magnetic-rotor test of arXiv:2406.11669, Sec. 4.4, describes; the time interpolation of subcycling, Sec. 3.10,
// at the end): a fine block of half the spacing whose interior covers the coarse interior
// cells L .. L + n_fine/2 - 1 along each axis.
//
// Prolongation to the fine block's ghost points (or to all its points), axis by axis in the order x, y, z: along
// an axis where the variable is cell-centred, third-order conservative, u_I -/+ (u_{I+1} - u_{I-1}) / 8 for the
// two halves of coarse cell I, replaced for both halves by the limited linear u_I -/+ minmod(u_I - u_{I-1},
// u_{I+1} - u_I) / 4 where either would leave the range of the three coarse averages; along a vertex-centred axis,
// a fine point on a coarse point copies it, a midpoint takes (-u_{J-1} + 9 u_J + 9 u_{J+1} - u_{J+2}) / 16.
// Restriction: the mean of the fine points covering a coarse point (two halves along a cell-centred axis, the
// coincident point along a vertex-centred one).
//
// One thread per fine point (prolongation) or coarse point (restriction), each field in turn; the 3x3x3 (at most
// 4x4x4) coarse stencil of neighbouring fine points overlaps, so the gathers hit the caches.
#include "kernels.h"

namespace asterx {

namespace {

__device__ __forceinline__ int floor_div2(int f) { return (f >= 0) ? f / 2 : -((-f + 1) / 2); }

template <class Get>
__device__ __forceinline__ double prolong_1d(bool cell, int f, const Get& get) {
  if (cell) {
    const int I = floor_div2(f);
    const bool right = (f - 2 * I) == 1;
    const double um = get(I - 1), u0 = get(I), up = get(I + 1);
    const double d = (up - um) * 0.125;
    const double lo = fmin(um, fmin(u0, up)), hi = fmax(um, fmax(u0, up));
    const double vl = u0 - d, vr = u0 + d;
    if (vl < lo || vl > hi || vr < lo || vr > hi) {
      const double a = u0 - um, b = up - u0;
      const double s = (a * b <= 0.0) ? 0.0 : (fabs(a) <= fabs(b) ? a : b);
      return right ? u0 + 0.25 * s : u0 - 0.25 * s;
    }
    return right ? vr : vl;
  }
  if ((f & 1) == 0) return get(f / 2);
  const int J = floor_div2(f - 1);
  return (-get(J - 1) + 9.0 * get(J) + 9.0 * get(J + 1) - get(J + 2)) * 0.0625;
}

struct RefineArgs {
  Blk C, F;
  int L[3];
  F9 Uc, Uf;
  F5 Pc, Pf;
  int all;
};

__device__ __forceinline__ long clin(const Blk& b, int i, int j, int k) { return i + b.sy * j + b.sz * k; }

// the points of the fine padded array outside its cell interior [g, g+n) along some axis (every ghost point of
// every field lies there): the planes before and after the interior along z, then along y within the interior
// z range, then along x within the interior y and z ranges
__host__ __device__ inline long shell_count(const Blk& F) {
  return F.V - (long)F.n[0] * F.n[1] * F.n[2];
}

__device__ __forceinline__ void shell_point(const Blk& F, long t, int& i, int& j, int& k) {
  const long e0 = F.N[0] + 1, e1 = F.N[1] + 1;
  const long zA = (long)(F.N[2] + 1 - F.n[2]) * e1 * e0;
  if (t < zA) {
    const long pl = t / (e1 * e0), r = t % (e1 * e0);
    k = (int)(pl < F.g ? pl : pl + F.n[2]);
    j = (int)(r / e0);
    i = (int)(r % e0);
    return;
  }
  t -= zA;
  const long yw = (long)(F.N[1] + 1 - F.n[1]) * e0;
  const long zB = (long)F.n[2] * yw;
  if (t < zB) {
    k = F.g + (int)(t / yw);
    const long r = t % yw, q = r / e0;
    j = (int)(q < F.g ? q : q + F.n[1]);
    i = (int)(r % e0);
    return;
  }
  t -= zB;
  const long xw = F.N[0] + 1 - F.n[0];
  k = F.g + (int)(t / ((long)F.n[1] * xw));
  const long r = t % ((long)F.n[1] * xw);
  j = F.g + (int)(r / xw);
  const long q = r % xw;
  i = (int)(q < F.g ? q : q + F.n[0]);
}

__global__ void __launch_bounds__(128) k_prolong(RefineArgs a) {
  const Blk& F = a.F;
  const Blk& C = a.C;
  const long count = a.all ? F.V : shell_count(F);
  const int clm[14] = {7, 7, 7, 7, 7, 1, 2, 4, 0, 7, 7, 7, 7, 7};  // bit a: cell-centred along axis a
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    if (a.all) {
      i = (int)(t % F.sy);
      j = (int)((t / F.sy) % (F.N[1] + 1));
      k = (int)(t / F.sz);
    } else {
      shell_point(F, t, i, j, k);
    }
    const long c = clin(F, i, j, k);
    const int p[3] = {i, j, k};
    const int fr[3] = {i - F.g, j - F.g, k - F.g};
#pragma unroll 1
    for (int v = 0; v < 14; v++) {
      bool owned = true, inside = true;
      int cl[3];
      for (int ax = 0; ax < 3; ax++) {
        cl[ax] = (clm[v] >> ax) & 1;
        const int hi = cl[ax] ? F.g + F.n[ax] - 1 : F.g + F.n[ax];
        owned = owned && p[ax] >= F.g && p[ax] <= hi;
        inside = inside && p[ax] < F.N[ax] + (cl[ax] ? 0 : 1);
      }
      if ((owned && !a.all) || !inside) continue;
      const double* __restrict__ src = v < 9 ? a.Uc.f[v] : a.Pc.f[v - 9];
      auto along_z = [&](int qz) {
        auto along_y = [&](int qy) {
          auto along_x = [&](int qx) {
            return src[clin(C, C.g + a.L[0] + qx, C.g + a.L[1] + qy, C.g + a.L[2] + qz)];
          };
          return prolong_1d(cl[0], fr[0], along_x);
        };
        return prolong_1d(cl[1], fr[1], along_y);
      };
      const double val = prolong_1d(cl[2], fr[2], along_z);
      if (v < 9) a.Uf.f[v][c] = val;
      else a.Pf.f[v - 9][c] = val;
    }
  }
}

__global__ void __launch_bounds__(128) k_restrict(RefineArgs a) {
  const Blk& F = a.F;
  const Blk& C = a.C;
  const int m[3] = {F.n[0] / 2, F.n[1] / 2, F.n[2] / 2};
  const long e0 = m[0] + 1, e1 = m[1] + 1;
  const long count = e0 * e1 * (m[2] + 1);
  const int clm[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
    const int q[3] = {(int)(t % e0), (int)((t / e0) % e1), (int)(t / (e0 * e1))};
#pragma unroll 1
    for (int v = 0; v < 9; v++) {
      int cl[3];
      bool in = true;
      for (int ax = 0; ax < 3; ax++) {
        cl[ax] = (clm[v] >> ax) & 1;
        in = in && q[ax] <= (cl[ax] ? m[ax] - 1 : m[ax]);
      }
      if (!in) continue;
      double sum = 0.0;
      int cnt = 0;
      for (int dz = 0; dz <= cl[2]; dz++)
        for (int dy = 0; dy <= cl[1]; dy++)
          for (int dx = 0; dx <= cl[0]; dx++) {
            sum += a.Uf.f[v][clin(F, F.g + 2 * q[0] + dx, F.g + 2 * q[1] + dy, F.g + 2 * q[2] + dz)];
            cnt++;
          }
      a.Uc.f[v][clin(C, C.g + a.L[0] + q[0], C.g + a.L[1] + q[1], C.g + a.L[2] + q[2])] = sum / cnt;
    }
  }
}

// Subcycling (Sec. 3.10): the coarse state that feeds the fine ghost points at one fine stage, U_n + sum_i beta_i
// h k_i over every point of the padded coarse block, with the coarse RK4 slopes recovered from the step's base
// U_n, stage states Y_1..Y_3 and result U_1 (h k_1 = 2 (Y_1 - U_n), h k_2 = 2 (Y_2 - U_n), h k_3 = Y_3 - U_n,
// h k_4 = 6 (U_1 - U_n) - h k_1 - 2 h k_2 - 2 h k_3); individually rounded operations in a fixed order.
struct CombineArgs {
  long V;
  F9 un, y1, y2, y3, u1, out;
  double beta[4];
};

__global__ void __launch_bounds__(256) k_subcycle_combine(CombineArgs a) {
  const long total = 9 * a.V;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int v = (int)(t / a.V);
    const long c = t - (long)v * a.V;
    const double un = a.un.f[v][c];
    const double g0 = __dmul_rn(2.0, __dsub_rn(a.y1.f[v][c], un));
    const double g1 = __dmul_rn(2.0, __dsub_rn(a.y2.f[v][c], un));
    const double g2 = __dsub_rn(a.y3.f[v][c], un);
    const double g3 = __dsub_rn(__dsub_rn(__dsub_rn(__dmul_rn(6.0, __dsub_rn(a.u1.f[v][c], un)), g0),
                                          __dmul_rn(2.0, g1)),
                                __dmul_rn(2.0, g2));
    const double sum = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.beta[0], g0), __dmul_rn(a.beta[1], g1)),
                                           __dmul_rn(a.beta[2], g2)),
                                 __dmul_rn(a.beta[3], g3));
    a.out.f[v][c] = __dadd_rn(un, sum);
  }
}

int refine_grid(long count) {
  long blocks = (count + 127) / 128;
  if (blocks > 152L * 64) blocks = 152L * 64;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

cudaError_t launch_prolong(const Blk& C, const Blk& F, const int L[3], const F9& Uc, const F5& Pc, const F9& Uf,
                           const F5& Pf, bool all, cudaStream_t s) {
  RefineArgs a;
  a.C = C;
  a.F = F;
  for (int d = 0; d < 3; d++) a.L[d] = L[d];
  a.Uc = Uc;
  a.Pc = Pc;
  a.Uf = Uf;
  a.Pf = Pf;
  a.all = all;
  k_prolong<<<refine_grid(all ? F.V : shell_count(F)), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_subcycle_combine(const Blk& b, const F9& un, const F9& y1, const F9& y2, const F9& y3,
                                    const F9& u1, const F9& out, const double beta[4], cudaStream_t s) {
  CombineArgs a;
  a.V = b.V;
  a.un = un;
  a.y1 = y1;
  a.y2 = y2;
  a.y3 = y3;
  a.u1 = u1;
  a.out = out;
  for (int i = 0; i < 4; i++) a.beta[i] = beta[i];
  long blocks = (9 * b.V + 255) / 256;
  if (blocks > 152L * 32) blocks = 152L * 32;
  k_subcycle_combine<<<(int)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Blk& C, const Blk& F, const int L[3], const F9& Uc, const F9& Uf, cudaStream_t s) {
  RefineArgs a;
  a.C = C;
  a.F = F;
  for (int d = 0; d < 3; d++) a.L[d] = L[d];
  a.Uc = Uc;
  a.Uf = Uf;
  a.Pc = F5{};
  a.Pf = F5{};
  a.all = 0;
  const long count = (long)(F.n[0] / 2 + 1) * (F.n[1] / 2 + 1) * (F.n[2] / 2 + 1);
  k_restrict<<<refine_grid(count), 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace asterx
