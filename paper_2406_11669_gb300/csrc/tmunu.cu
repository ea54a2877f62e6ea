// Stress-energy tensor at vertices (Eq. tmunu of arXiv:2406.11669; T_{mu nu} is stored at vertices, Sec. 3.1),
// the matter input of a spacetime solver coupled to the GRMHD stage.
//
// At every vertex of the owned range (g..g+n per axis) the rest-mass density, pressure, u^i = W v^i and centre
// field B^i of the eight cells around it are averaged to the vertex.  With the vertex metric (alpha, beta^i,
// gamma_ij read directly from the caller's metric arrays): W = sqrt(1 + gamma_ij u^i u^j), v^i = u^i / W, the
// comoving field of Eq. eulerianB, and
//   T_{mu nu} = (rho h + b^2) u_mu u_nu + (p + b^2/2) g_{mu nu} - b_mu b_nu
// with the covariant u_i = gamma_ij u^j, u_0 = -alpha W + beta^i u_i, b_i = B_i / W + alpha b^0 v_i,
// b_0 = -alpha^2 b^0 + beta^i b_i, g_00 = -alpha^2 + beta^i beta_i, g_0i = beta_i, g_ij = gamma_ij.
//
// Memory: one thread per vertex, x fastest, so the eight-cell gathers of neighbouring threads share cache
// lines; per vertex 8 cell fields (rho, p, u, B) shared among 8 vertices, 10 metric values and 10 outputs.
#include "kernels.h"

namespace asterx {

namespace {

struct TmunuArgs {
  Blk b;
  const double* rho;
  const double* press;
  const double* u;  // 3 fields at pitch V
  const double* B;  // 3 fields at pitch V
  const double* m[10];  // alpha, beta^x,y,z, gamma_xx,xy,xz,yy,yz,zz at vertices
  double* T[10];
  double gfac;  // Gamma / (Gamma - 1): rho h = rho + gfac p
};

__global__ void __launch_bounds__(128) k_tmunu(TmunuArgs a) {
  const Blk& b = a.b;
  const int e0 = b.n[0] + 1, e1 = b.n[1] + 1;
  const long count = (long)e0 * e1 * (b.n[2] + 1);
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(t, (unsigned)e0, (unsigned)e1, i, j, k);
    i += b.g;
    j += b.g;
    k += b.g;
    const long v = i + b.sy * j + b.sz * k;
    const long c0 = v - 1 - b.sy - b.sz;  // cell (i-1, j-1, k-1)
    const long off[8] = {0, 1, b.sy, b.sy + 1, b.sz, b.sz + 1, b.sz + b.sy, b.sz + b.sy + 1};
    double rho = 0.0, p = 0.0, uu[3] = {0.0, 0.0, 0.0}, BB[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const long c = c0 + off[q];
      rho += a.rho[c];
      p += a.press[c];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        uu[d] += a.u[d * b.V + c];
        BB[d] += a.B[d * b.V + c];
      }
    }
    rho *= 0.125;
    p *= 0.125;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      uu[d] *= 0.125;
      BB[d] *= 0.125;
    }
    const double al = a.m[0][v];
    const double be[3] = {a.m[1][v], a.m[2][v], a.m[3][v]};
    double g[3][3];
    g[0][0] = a.m[4][v];
    g[0][1] = g[1][0] = a.m[5][v];
    g[0][2] = g[2][0] = a.m[6][v];
    g[1][1] = a.m[7][v];
    g[1][2] = g[2][1] = a.m[8][v];
    g[2][2] = a.m[9][v];
    double blo[3], ulo[3], Blo[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      blo[d] = g[d][0] * be[0] + g[d][1] * be[1] + g[d][2] * be[2];
      ulo[d] = g[d][0] * uu[0] + g[d][1] * uu[1] + g[d][2] * uu[2];
      Blo[d] = g[d][0] * BB[0] + g[d][1] * BB[1] + g[d][2] * BB[2];
    }
    const double W = sqrt(1.0 + uu[0] * ulo[0] + uu[1] * ulo[1] + uu[2] * ulo[2]);
    const double iW = 1.0 / W;
    const double B2 = BB[0] * Blo[0] + BB[1] * Blo[1] + BB[2] * Blo[2];
    const double Bu = BB[0] * ulo[0] + BB[1] * ulo[1] + BB[2] * ulo[2];  // B^i u_i = W B^i v_i
    const double ab0 = Bu;                                               // alpha b^0 = W B^i v_i
    double bl[3];
#pragma unroll
    for (int d = 0; d < 3; d++) bl[d] = (Blo[d] + ab0 * ulo[d]) * iW;  // B_i / W + alpha b^0 v_i, v_i = u_i / W
    const double b2 = (B2 + ab0 * ab0) * iW * iW;
    const double u0 = -al * W + be[0] * ulo[0] + be[1] * ulo[1] + be[2] * ulo[2];
    const double bt = -al * ab0 + be[0] * bl[0] + be[1] * bl[1] + be[2] * bl[2];
    const double e = rho + a.gfac * p + b2;
    const double pt = p + 0.5 * b2;
    const double g00 = -al * al + be[0] * blo[0] + be[1] * blo[1] + be[2] * blo[2];
    a.T[0][v] = e * u0 * u0 + pt * g00 - bt * bt;
#pragma unroll
    for (int d = 0; d < 3; d++) a.T[1 + d][v] = e * u0 * ulo[d] + pt * blo[d] - bt * bl[d];
    int q = 4;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
      for (int f = d; f < 3; f++) a.T[q++][v] = e * ulo[d] * ulo[f] + pt * g[d][f] - bl[d] * bl[f];
  }
}

}  // namespace

cudaError_t launch_tmunu(const Blk& b, const Ws& w, double gamma, const CF16& m, const F5& P, double* const T[10],
                         cudaStream_t s) {
  TmunuArgs a;
  a.b = b;
  a.rho = P.f[0];
  a.press = P.f[1];
  a.u = w.uvel;
  a.B = w.bc;
  for (int q = 0; q < 10; q++) {
    a.m[q] = m.f[q];
    a.T[q] = T[q];
  }
  a.gfac = gamma / (gamma - 1.0);
  const long count = (long)(b.n[0] + 1) * (b.n[1] + 1) * (b.n[2] + 1);
  long blocks = (count + 127) / 128;
  if (blocks > 64L * device_sm_count()) blocks = 64L * device_sm_count();
  k_tmunu<<<(int)blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace asterx
