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
// Prolongation: one thread per coarse parent cell, each field in turn, writing the parent's up to eight fine
// children from its 3x3x3 (at most 4x4x4) coarse stencil with the 1D steps shared among them; restriction: one
// thread per coarse point.
#include "kernels.h"

namespace asterx {

namespace {

struct RefineArgs {
  Blk C, F;
  int L[3];
  F9 Uc, Uf;
  F5 Pc, Pf;
  int all;
};

__device__ __forceinline__ long clin(const Blk& b, int i, int j, int k) { return i + b.sy * j + b.sz * k; }

// The 1D operator for both fine halves of parent P at once, from the parent's stencil u[0..3] = u_{P-1}, u_P,
// u_{P+1}, u_{P+2}: cell-centred, u_P -/+ (u_{P+1} - u_{P-1}) / 8, or for both halves the limited linear
// u_P -/+ minmod(u_P - u_{P-1}, u_{P+1} - u_P) / 4 where either value would leave the range of the three;
// vertex-centred, the coincident point u_P and the midpoint (-u_{P-1} + 9 u_P + 9 u_{P+1} - u_{P+2}) / 16.
template <bool CELL>
__device__ __forceinline__ void prolong_pair(const double u[4], double& lo, double& hi) {
  if (CELL) {
    const double um = u[0], u0 = u[1], up = u[2];
    const double d = (up - um) * 0.125;
    const double mn = fmin(um, fmin(u0, up)), mx = fmax(um, fmax(u0, up));
    const double vl = u0 - d, vr = u0 + d;
    if (vl < mn || vl > mx || vr < mn || vr > mx) {
      const double a = u0 - um, b = up - u0;
      const double s = (a * b <= 0.0) ? 0.0 : (fabs(a) <= fabs(b) ? a : b);
      lo = u0 - 0.25 * s;
      hi = u0 + 0.25 * s;
    } else {
      lo = vl;
      hi = vr;
    }
  } else {
    lo = u[1];
    hi = (-u[0] + 9.0 * u[1] + 9.0 * u[2] - u[3]) * 0.0625;
  }
}

// The up to eight fine children (2P + h along each axis, h = 0, 1) of coarse parent P = (P0, P1, P2) (indices
// relative to the fine box's first coarse cell) for one field centred as CL (bit a: cell-centred along axis a):
// the 1D operator along x on every stencil line, then along y on those results, then along z, each computed
// once and shared by the children (a per-point evaluation repeats the x and y steps up to eight times).
template <int CL>
__device__ __forceinline__ void prolong_children(const RefineArgs& a, const double* __restrict__ src,
                                                 double* __restrict__ dst, const int P[3]) {
  constexpr bool C0 = CL & 1, C1 = (CL >> 1) & 1, C2 = (CL >> 2) & 1;
  constexpr int S1 = C1 ? 3 : 4, S2 = C2 ? 3 : 4;  // stencil lengths along y and z
  const Blk& F = a.F;
  const Blk& C = a.C;
  const int b0 = C.g + a.L[0] + P[0] - 1, b1 = C.g + a.L[1] + P[1] - 1, b2 = C.g + a.L[2] + P[2] - 1;
  double Y[2][2][4];
#pragma unroll
  for (int iz = 0; iz < S2; iz++) {
    double X[2][4];
#pragma unroll
    for (int iy = 0; iy < S1; iy++) {
      const double* __restrict__ row = src + clin(C, b0, b1 + iy, b2 + iz);
      const double u[4] = {row[0], row[1], row[2], C0 ? 0.0 : row[3]};
      prolong_pair<C0>(u, X[0][iy], X[1][iy]);
    }
#pragma unroll
    for (int hx = 0; hx < 2; hx++) {
      const double u[4] = {X[hx][0], X[hx][1], X[hx][2], C1 ? 0.0 : X[hx][3]};
      prolong_pair<C1>(u, Y[hx][0][iz], Y[hx][1][iz]);
    }
  }
  bool owned[3][2], inside[3][2];
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
    const bool cell = (CL >> ax) & 1;
    const int hi = cell ? F.g + F.n[ax] - 1 : F.g + F.n[ax];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int p = F.g + 2 * P[ax] + h;
      owned[ax][h] = p >= F.g && p <= hi;
      inside[ax][h] = p >= 0 && p < F.N[ax] + (cell ? 0 : 1);
    }
  }
#pragma unroll
  for (int hx = 0; hx < 2; hx++)
#pragma unroll
    for (int hy = 0; hy < 2; hy++) {
      const double u[4] = {Y[hx][hy][0], Y[hx][hy][1], Y[hx][hy][2], C2 ? 0.0 : Y[hx][hy][3]};
      double z[2];
      prolong_pair<C2>(u, z[0], z[1]);
#pragma unroll
      for (int hz = 0; hz < 2; hz++) {
        if (!(inside[0][hx] && inside[1][hy] && inside[2][hz])) continue;
        if (!a.all && owned[0][hx] && owned[1][hy] && owned[2][hz]) continue;
        dst[clin(F, F.g + 2 * P[0] + hx, F.g + 2 * P[1] + hy, F.g + 2 * P[2] + hz)] = z[hz];
      }
    }
}

// Parents: coarse cells P with children in the fine padded array, P = -2 .. n_fine/2 + 1 along each axis for
// three ghost layers (floor((-g)/2) .. floor((n_fine + g)/2) in general); for the ghost shell only those with
// an axis outside 0 .. n_fine/2 - 1 (a parent inside that range along every axis has owned children only).
struct ParentGrid {
  int lo[3], E[3];  // first parent and parent count per axis
  int il[3], ih[3];  // the interior parents, relative to lo (inclusive)
  __host__ __device__ long total() const { return (long)E[0] * E[1] * E[2]; }
  __host__ __device__ long shell() const {
    return total() - (long)(ih[0] - il[0] + 1) * (ih[1] - il[1] + 1) * (ih[2] - il[2] + 1);
  }
};

__host__ __device__ inline ParentGrid parent_grid(const Blk& F) {
  ParentGrid q;
  for (int ax = 0; ax < 3; ax++) {
    const int first = -((F.g + 1) / 2), last = (F.n[ax] + F.g) / 2;  // floor division for g >= 0
    q.lo[ax] = first;
    q.E[ax] = last - first + 1;
    q.il[ax] = -first;
    q.ih[ax] = F.n[ax] / 2 - 1 - first;
  }
  return q;
}

// t-th parent of the full grid (all) or of the shell: planes outside the interior along z, then rows outside it
// along y within the interior z range, then points outside it along x within the interior y and z ranges
__device__ __forceinline__ void parent_at(const ParentGrid& q, bool all, long t, int P[3]) {
  int i, j, k;
  const long e0 = q.E[0], e1 = q.E[1];
  if (all) {
    unflatten3(t, (unsigned)e0, (unsigned)e1, i, j, k);
  } else {
    const int nz = q.ih[2] - q.il[2] + 1, ny = q.ih[1] - q.il[1] + 1, nx = q.ih[0] - q.il[0] + 1;
    const long zA = (long)(q.E[2] - nz) * e1 * e0;
    if (t < zA) {
      const long pl = t / (e1 * e0), r = t % (e1 * e0);
      k = (int)(pl < q.il[2] ? pl : pl + nz);
      j = (int)(r / e0);
      i = (int)(r % e0);
    } else {
      t -= zA;
      const long yw = (long)(q.E[1] - ny) * e0;
      const long zB = (long)nz * yw;
      if (t < zB) {
        k = q.il[2] + (int)(t / yw);
        const long r = t % yw, qq = r / e0;
        j = (int)(qq < q.il[1] ? qq : qq + ny);
        i = (int)(r % e0);
      } else {
        t -= zB;
        const long xw = q.E[0] - nx;
        k = q.il[2] + (int)(t / ((long)ny * xw));
        const long r = t % ((long)ny * xw);
        j = q.il[1] + (int)(r / xw);
        const long qq = r % xw;
        i = (int)(qq < q.il[0] ? qq : qq + nx);
      }
    }
  }
  P[0] = q.lo[0] + i;
  P[1] = q.lo[1] + j;
  P[2] = q.lo[2] + k;
}

__global__ void __launch_bounds__(128, 3) k_prolong(RefineArgs a) {
  const ParentGrid q = parent_grid(a.F);
  const long count = a.all ? q.total() : q.shell();
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
    int P[3];
    parent_at(q, a.all, t, P);
#pragma unroll 1
    for (int v = 0; v < 14; v++) {
      const double* __restrict__ src = v < 9 ? a.Uc.f[v] : a.Pc.f[v - 9];
      double* __restrict__ dst = v < 9 ? a.Uf.f[v] : a.Pf.f[v - 9];
      if (v < 5 || v >= 9) prolong_children<7>(a, src, dst, P);
      else if (v == 5) prolong_children<1>(a, src, dst, P);
      else if (v == 6) prolong_children<2>(a, src, dst, P);
      else if (v == 7) prolong_children<4>(a, src, dst, P);
      else prolong_children<0>(a, src, dst, P);
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
    int q[3];
    unflatten3(t, (unsigned)e0, (unsigned)e1, q[0], q[1], q[2]);
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
// h k_i over a box of points of the padded coarse block, with the coarse RK4 slopes recovered from the step's base
// U_n, stage states Y_1..Y_3 and result U_1 (h k_1 = 2 (Y_1 - U_n), h k_2 = 2 (Y_2 - U_n), h k_3 = Y_3 - U_n,
// h k_4 = 6 (U_1 - U_n) - h k_1 - 2 h k_2 - 2 h k_3); individually rounded operations in a fixed order.
struct CombineArgs {
  Blk b;
  int lo[3], e[3];  // the points lo .. lo + e - 1 of the padded block
  F9 un, y1, y2, y3, u1, out;
  double beta[4];
};

// grid: x strides over the points, y = the field
__global__ void __launch_bounds__(256) k_subcycle_combine(CombineArgs a) {
  const int v = blockIdx.y;
  const double* __restrict__ pn = a.un.f[v];
  const double* __restrict__ p1 = a.y1.f[v];
  const double* __restrict__ p2 = a.y2.f[v];
  const double* __restrict__ p3 = a.y3.f[v];
  const double* __restrict__ pu = a.u1.f[v];
  double* __restrict__ po = a.out.f[v];
  const long count = (long)a.e[0] * a.e[1] * a.e[2];
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(t, (unsigned)a.e[0], (unsigned)a.e[1], i, j, k);
    const long c = clin(a.b, a.lo[0] + i, a.lo[1] + j, a.lo[2] + k);
    const double un = pn[c];
    const double g0 = __dmul_rn(2.0, __dsub_rn(p1[c], un));
    const double g1 = __dmul_rn(2.0, __dsub_rn(p2[c], un));
    const double g2 = __dsub_rn(p3[c], un);
    const double g3 = __dsub_rn(__dsub_rn(__dsub_rn(__dmul_rn(6.0, __dsub_rn(pu[c], un)), g0),
                                          __dmul_rn(2.0, g1)),
                                __dmul_rn(2.0, g2));
    const double sum = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.beta[0], g0), __dmul_rn(a.beta[1], g1)),
                                           __dmul_rn(a.beta[2], g2)),
                                 __dmul_rn(a.beta[3], g3));
    po[c] = __dadd_rn(un, sum);
  }
}

int refine_grid(long count) {
  long blocks = (count + 127) / 128;
  if (blocks > 64L * device_sm_count()) blocks = 64L * device_sm_count();
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
  const ParentGrid q = parent_grid(F);
  k_prolong<<<refine_grid(all ? q.total() : q.shell()), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_subcycle_combine(const Blk& b, const int lo[3], const int hi[3], const F9& un, const F9& y1,
                                    const F9& y2, const F9& y3, const F9& u1, const F9& out, const double beta[4],
                                    cudaStream_t s) {
  CombineArgs a;
  a.b = b;
  long count = 1;
  for (int d = 0; d < 3; d++) {
    if (lo[d] < 0 || hi[d] > b.N[d] || hi[d] < lo[d]) return cudaErrorInvalidValue;
    a.lo[d] = lo[d];
    a.e[d] = hi[d] - lo[d] + 1;
    count *= a.e[d];
  }
  a.un = un;
  a.y1 = y1;
  a.y2 = y2;
  a.y3 = y3;
  a.u1 = u1;
  a.out = out;
  for (int i = 0; i < 4; i++) a.beta[i] = beta[i];
  long blocks = (count + 255) / 256;
  if (blocks > 8L * device_sm_count()) blocks = 8L * device_sm_count();
  k_subcycle_combine<<<dim3((unsigned)blocks, 9), 256, 0, s>>>(a);
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
