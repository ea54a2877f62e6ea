// Adjoint (vector-Jacobian product) of the right-hand side of one RK stage, and of a classical RK4 step.
//
// Given mu = dJ/d(dU/dt) on the owned ranges, the kernels below return lambda = (dL/dY)^T mu for the stage
// operator L(Y) of the forward path (ghost fill, B~ = curl A, recovery, reconstruction, face solve, UCT,
// potentials, sources).  Each forward kernel has a reverse kernel, run in reverse order:
//   cells (flux divergence, sources) -> scalar potential -> edges (UCT, grad G_A) -> vertex potentials ->
//   face solves and reconstruction (per direction) -> u = W v -> primitive ghost fill -> recovery ->
//   centre field -> curl -> state ghost fill.
// Linear maps are transposed by hand.  The heavy nonlinear maps are reversed by hand (reverse mode): the face
// solve (face_side_vjp, the wave speeds by the implicit-function theorem at the converged roots), the source
// terms (sources_vjp), minmod and PPM (recon5_vjp).  The others take their local Jacobian from the same
// templated device code as the forward path run with forward-mode dual numbers: u = W v, WENO-Z, and
// prim->cons, whose Jacobian inverted at the recovered primitives differentiates the recovery (implicit-function
// theorem).
// Limiters, max/min and branch choices take the derivative of the branch taken.  Atmosphere cells (constant
// primitives) pass no derivative through the recovery.
//
// Accumulations that several threads share use FP64 atomics, so the summation order (and the last bits of
// lambda) may vary between runs.
#include <cstring>

#include "kernels.h"
#include "physics.cuh"

namespace asterx {

static __host__ int agrid(long count, int threads) {
  long blocks = (count + threads - 1) / threads;
  const long cap = 64L * device_sm_count();
  return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

#define ALOOP(t, count) \
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (count); t += (long)gridDim.x * blockDim.x)

__device__ __forceinline__ long alin(const Blk& b, int i, int j, int k) { return i + b.sy * j + b.sz * k; }
__device__ __forceinline__ long astr(const Blk& b, int d) { return d == 0 ? 1 : (d == 1 ? b.sy : b.sz); }

__device__ __forceinline__ void decode(long t, int lo0, int e0, int lo1, int e1, int lo2, int& i, int& j, int& k) {
  unflatten3(t, (unsigned)e0, (unsigned)e1, i, j, k);
  i += lo0;
  j += lo1;
  k += lo2;
}

// ----------------------------------------------------------------------------------------------------------
// Cells: dU_v/dt = -sum_d (F_d,v(c + e_d) - F_d,v(c)) / dx_d + S_v(P, B).  Flux part: each face gathers the
// adjoints of its two cells (zero outside the interior).  Source part: Jacobian of the sources in (rho, p, v,
// B) by dual numbers.

__global__ void ka_flux_div(Blk b, AdjWs a, F9 mu, int D) {
  // faces g..g+n along D, interior transverse
  int lo[3] = {b.g, b.g, b.g}, e[3] = {b.n[0], b.n[1], b.n[2]};
  e[D] = b.n[D] + 1;
  const long count = (long)e[0] * e[1] * e[2];
  const long st = astr(b, D);
  ALOOP(t, count) {
    int p[3];
    decode(t, lo[0], e[0], lo[1], e[1], lo[2], p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    const bool left_in = p[D] - 1 >= b.g;          // cell c - e_D is interior
    const bool right_in = p[D] <= b.g + b.n[D] - 1;  // cell c is interior
    for (int v = 0; v < 5; v++) {
      const double ml = left_in ? mu.f[v][c - st] : 0.0;
      const double mr = right_in ? mu.f[v][c] : 0.0;
      // F(c) enters dU(c) with +1/dx and dU(c - e_D) with -1/dx
      a.lface[((long)D * NFD + FD_F + v) * b.V + c] = (mr - ml) * b.idx[D];
    }
  }
}

__device__ __forceinline__ void load_geo(const Blk& b, const double* __restrict__ cg, long c, Geo& m) {
  m.alp = cg[CG_ALP * b.V + c];
  for (int q = 0; q < 3; q++) m.beta[q] = cg[(CG_BETA + q) * b.V + c];
  for (int q = 0; q < 6; q++) {
    m.g[q] = cg[(CG_G + q) * b.V + c];
    m.gu[q] = cg[(CG_GU + q) * b.V + c];
  }
  m.sqg = cg[CG_SQG * b.V + c];
}

__global__ void ka_sources(Blk b, Ws w, AdjWs a, F5 P, F9 mu, double gfac) {
  const long count = (long)b.n[0] * b.n[1] * b.n[2];
  ALOOP(t, count) {
    int i, j, k;
    decode(t, b.g, b.n[0], b.g, b.n[1], b.g, i, j, k);
    const long c = alin(b, i, j, k);
    Geo m;
    load_geo(b, w.cg, c, m);
    const double v[3] = {P.f[2][c], P.f[3][c], P.f[4][c]};
    const double B[3] = {w.bc[c], w.bc[b.V + c], w.bc[2 * b.V + c]};
    const double mq[5] = {0.0, mu.f[1][c], mu.f[2][c], mu.f[3][c], mu.f[4][c]};
    double g8[8];
    sources_vjp(m, w.cg, b.V, c, P.f[0][c], P.f[1][c], v, B, gfac, mq, g8);
    for (int r = 0; r < 5; r++) a.lP[r * b.V + c] += g8[r];
    for (int r = 0; r < 3; r++) a.lBc[r * b.V + c] += g8[5 + r];
  }
}

// ----------------------------------------------------------------------------------------------------------
// Scalar potential: dPsi = -sum_j (F^j(v+e_j) - F^j(v-e_j)) / (2 dx_j) - xi alpha Psi on vertices g..g+n.
// lambda_FPsi^j(w) gathers the two vertices that difference it.

__global__ void ka_psi(Blk b, Ws w, AdjWs a, F9 mu, double xi) {
  // vertices g-1 .. g+n+1 (the F_Psi range)
  const int n0 = b.n[0] + 3, n1 = b.n[1] + 3, n2 = b.n[2] + 3;
  const long count = (long)n0 * n1 * n2;
  ALOOP(t, count) {
    int p[3];
    decode(t, b.g - 1, n0, b.g - 1, n1, b.g - 1, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    auto owned = [&](const int q[3]) {
      return q[0] >= b.g && q[0] <= b.g + b.n[0] && q[1] >= b.g && q[1] <= b.g + b.n[1] && q[2] >= b.g &&
             q[2] <= b.g + b.n[2];
    };
    for (int d = 0; d < 3; d++) {
      int qm[3] = {p[0], p[1], p[2]}, qp[3] = {p[0], p[1], p[2]};
      qm[d] -= 1;
      qp[d] += 1;
      const double mm = owned(qm) ? mu.f[8][c - astr(b, d)] : 0.0;
      const double mp = owned(qp) ? mu.f[8][c + astr(b, d)] : 0.0;
      // F^d(c) enters dPsi(c + e_d) with +1/(2dx) and dPsi(c - e_d) with -1/(2dx)
      a.lFpsi[d * b.V + c] = (mp - mm) * (0.5 * b.idx[d]);
    }
    if (owned(p)) a.lY[8 * b.V + c] += -xi * w.vg[VG_ALP * b.V + c] * mu.f[8][c];
  }
}

// ----------------------------------------------------------------------------------------------------------
// Edges: dA_E = -E_E - (G_A(c + e_E) - G_A(c)) / dx_E.  lambda_G_A(v) gathers the edges that difference it.

__global__ void ka_grad_ga(Blk b, AdjWs a, F9 mu) {
  const int n0 = b.n[0] + 3, n1 = b.n[1] + 3, n2 = b.n[2] + 3;
  const long count = (long)n0 * n1 * n2;
  ALOOP(t, count) {
    int p[3];
    decode(t, b.g - 1, n0, b.g - 1, n1, b.g - 1, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    double acc = 0.0;
    for (int E = 0; E < 3; E++) {
      // edges along E at q: owned range g..g+n-1 along E, g..g+n across
      auto owned = [&](const int q[3]) {
        for (int d = 0; d < 3; d++) {
          const int hi = (d == E) ? b.g + b.n[d] - 1 : b.g + b.n[d];
          if (q[d] < b.g || q[d] > hi) return false;
        }
        return true;
      };
      int qm[3] = {p[0], p[1], p[2]};
      qm[E] -= 1;
      const double m_here = owned(p) ? mu.f[5 + E][c] : 0.0;               // edge at c: +G(c)/dx
      const double m_below = owned(qm) ? mu.f[5 + E][c - astr(b, E)] : 0.0;  // edge at c-e: -G(c)/dx
      acc += (m_here - m_below) * b.idx[E];
    }
    a.lGA[c] = acc;
  }
}

// UCT: E_E = -HLL_d1(v~^d1 B~^d2) + HLL_d2(v~^d2 B~^d1); lambda_E = -mu_A.  Each term reversed by hand: the HLL
// formula, the PPM interface values (reverse-mode recon5), a_+- = max over the two faces (branch taken).
template <int E>
__global__ void ka_edges(Blk b, Ws w, AdjWs a, F9 mu, int fct) {
  constexpr int D1 = (E + 1) % 3, D2 = (E + 2) % 3;
  int lo[3] = {b.g, b.g, b.g}, ex[3] = {b.n[0] + 1, b.n[1] + 1, b.n[2] + 1};
  ex[E] = b.n[E];
  const long count = (long)ex[0] * ex[1] * ex[2];
  ALOOP(t, count) {
    int p[3];
    decode(t, lo[0], ex[0], lo[1], ex[1], lo[2], p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    const double lE = -mu.f[5 + E][c];
    if (fct) {  // E = (F_D2(B~^D1) at c and c - e_D1  -  F_D1(B~^D2) at c and c - e_D2) / 4
      const double q = 0.25 * lE;
      const long f2 = ((long)D2 * NFD + FD_EB2) * b.V, f1 = ((long)D1 * NFD + FD_EB1) * b.V;
      atomicAdd(&a.lface[f2 + c], q);
      atomicAdd(&a.lface[f2 + c - astr(b, D1)], q);
      atomicAdd(&a.lface[f1 + c], -q);
      atomicAdd(&a.lface[f1 + c - astr(b, D2)], -q);
      continue;
    }
#pragma unroll
    for (int tt = 0; tt < 2; tt++) {
      const double sgn = tt == 0 ? -1.0 : 1.0;  // E = -term0 + term1
      const int dr = tt == 0 ? D1 : D2;
      const int df = tt == 0 ? D2 : D1;
      const long sr = astr(b, dr);
      const long sf = astr(b, df);
      const int slot = (((df + 1) % 3) == dr) ? FD_VB1 : FD_VB2;
      const long vb_off = ((long)df * NFD + slot) * b.V;
      const long bn_off = (long)df * b.V;
      double vs[6], bs[6];
      for (int s = 0; s < 6; s++) {
        const long q = c + (s - 3) * sr;
        vs[s] = w.face[vb_off + q];
        bs[s] = w.bf[bn_off + q];
      }
      PpmPair pv, pb;
      pv.values(vs);
      pb.values(bs);
      const double vL = pv.L, vR = pv.R, BL = pb.L, BR = pb.R;
      const long fdr = (long)dr * NFD * b.V;
      const long c0 = c - sf;
      const double apa = w.face[fdr + FD_CMAX * b.V + c0], apb = w.face[fdr + FD_CMAX * b.V + c];
      const double ama = w.face[fdr + FD_CMIN * b.V + c0], amb = w.face[fdr + FD_CMIN * b.V + c];
      const double ap = fmax(apa, apb), am = fmax(ama, amb);
      const double den = ap + am;
      const double lt = sgn * lE;  // adjoint of this term
      double gvL, gvR, gBL, gBR, gap = 0.0, gam = 0.0;
      if (den > 0.0) {
        const double term = (ap * vL * BL + am * vR * BR - ap * am * (BR - BL)) / den;
        gvL = ap * BL / den;
        gBL = (ap * vL + ap * am) / den;
        gvR = am * BR / den;
        gBR = (am * vR - ap * am) / den;
        gap = (vL * BL - am * (BR - BL) - term) / den;
        gam = (vR * BR - ap * (BR - BL) - term) / den;
      } else {
        gvL = 0.5 * BL;
        gBL = 0.5 * vL;
        gvR = 0.5 * BR;
        gBR = 0.5 * vR;
      }
      // the PPM interface values by reverse mode: the upper value of stencil cell 2, the lower of cell 3
      double gv[6], gb[6];
      pv.vjp(gvL * lt, gvR * lt, gv);
      pb.vjp(gBL * lt, gBR * lt, gb);
      for (int s = 0; s < 6; s++) {
        const long q = c + (s - 3) * sr;
        if (gv[s] != 0.0) atomicAdd(&a.lface[vb_off + q], gv[s]);
        if (gb[s] != 0.0) atomicAdd(&a.lBf[bn_off + q], gb[s]);
      }
      if (gap != 0.0) atomicAdd(&a.lface[fdr + FD_CMAX * b.V + (apb > apa ? c : c0)], gap * lt);
      if (gam != 0.0) atomicAdd(&a.lface[fdr + FD_CMIN * b.V + (amb > ama ? c : c0)], gam * lt);
    }
  }
}

// Vertex potentials: G_A = alpha Psi / sqrt(g) - beta^j Av_j, F^j = alpha sqrt(g) gamma^jk Av_k - beta^j Psi,
// Av_j = (A_j(v - e_j) + A_j(v)) / 2.  First the vertex adjoints of Av and Psi, then each edge gathers the two
// vertices that average it.
__global__ void ka_vertex(Blk b, Ws w, AdjWs a, int lorenz) {
  const int n0 = b.n[0] + 3, n1 = b.n[1] + 3, n2 = b.n[2] + 3;
  const long count = (long)n0 * n1 * n2;
  ALOOP(t, count) {
    int p[3];
    decode(t, b.g - 1, n0, b.g - 1, n1, b.g - 1, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    const double alp = w.vg[VG_ALP * b.V + c];
    const double be[3] = {w.vg[(VG_BETA + 0) * b.V + c], w.vg[(VG_BETA + 1) * b.V + c],
                          w.vg[(VG_BETA + 2) * b.V + c]};
    const double sqg = w.vg[VG_SQG * b.V + c];
    double gu[6];
    for (int q = 0; q < 6; q++) gu[q] = w.vg[(VG_GU + q) * b.V + c];
    const double lg = lorenz ? a.lGA[c] : 0.0;
    const double lf[3] = {a.lFpsi[c], a.lFpsi[b.V + c], a.lFpsi[2 * b.V + c]};
    double lpsi = lorenz ? alp / sqg * lg : 0.0;
    for (int d = 0; d < 3; d++) lpsi -= be[d] * lf[d];
    a.lY[8 * b.V + c] += lpsi;
    const double as = alp * sqg;
    for (int k = 0; k < 3; k++) {
      const double lak = -(lorenz ? be[k] * lg : 0.0) + as * (gu[sym(0, k)] * lf[0] + gu[sym(1, k)] * lf[1] +
                                                             gu[sym(2, k)] * lf[2]);
      a.lAv[k * b.V + c] = lak;
    }
  }
}

__global__ void ka_vertex_to_edges(Blk b, AdjWs a) {
  // edges whose averaging vertex lies in g-1 .. g+n+1: along k the edge index g-2 .. g+n+1
  const int n0 = b.n[0] + 4, n1 = b.n[1] + 4, n2 = b.n[2] + 4;
  const long count = (long)n0 * n1 * n2;
  ALOOP(t, count) {
    int p[3];
    decode(t, b.g - 2, n0, b.g - 2, n1, b.g - 2, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    for (int k = 0; k < 3; k++) {
      // edge A_k at p feeds Av_k at vertices p and p + e_k
      double acc = 0.0;
      for (int s = 0; s < 2; s++) {
        int q[3] = {p[0], p[1], p[2]};
        q[k] += s;
        bool in = true;
        for (int d = 0; d < 3; d++) in = in && q[d] >= b.g - 1 && q[d] <= b.g + b.n[d] + 1;
        if (!in) continue;
        acc += 0.5 * a.lAv[k * b.V + alin(b, q[0], q[1], q[2])];
      }
      if (acc != 0.0) a.lY[(5 + k) * b.V + c] += acc;
    }
  }
}

// ----------------------------------------------------------------------------------------------------------
// Face solve along D (faces g..g+n along D, all transverse): adjoints of (F^, v~bar, c_max, c_min) -> adjoints
// of the reconstructed left/right states and of the face field B~.  The primal side solves run first (their
// speeds set the HLLE weights), then HLLE is reversed by hand and each side by its reverse-mode VJP.
// ALT: with the alternative schemes (Lax-Friedrichs, flux constrained transport) a separate instantiation, so
// that the default one keeps its register budget.
template <int D, bool ALT>
__global__ void ka_faces(Blk b, Ws w, AdjWs a, double gamma, double gfac, int lxf_, int fct_) {
  const bool lxf = ALT && lxf_, fct = ALT && fct_;
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  int lo[3] = {0, 0, 0}, ex[3] = {b.N[0], b.N[1], b.N[2]};
  lo[D] = b.g;
  ex[D] = b.n[D] + 1;
  const long count = (long)ex[0] * ex[1] * ex[2];
  const long st = astr(b, D);
  const double* __restrict__ fg = w.fg + (long)D * NFG * b.V;
  ALOOP(t, count) {
    int p[3];
    decode(t, lo[0], ex[0], lo[1], ex[1], lo[2], p[0], p[1], p[2]);
    // the corner columns (both transverse indices in the ghost layers) feed nothing: no roots were kept there
    if ((p[T1] < b.g || p[T1] >= b.g + b.n[T1]) && (p[T2] < b.g || p[T2] >= b.g + b.n[T2])) continue;
    const long c = alin(b, p[0], p[1], p[2]);
    Geo m;
    m.alp = fg[FG_ALP * b.V + c];
    for (int q = 0; q < 3; q++) m.beta[q] = fg[(FG_BETA + q) * b.V + c];
    for (int q = 0; q < 6; q++) m.g[q] = fg[(FG_G + q) * b.V + c];
    m.gu[sym(D, D)] = fg[FG_GUDD * b.V + c];  // the only inverse-metric component the face solve reads
    m.sqg = fg[FG_SQG * b.V + c];
    const double ia = fg[FG_IALP * b.V + c];
    const double width = fg[FG_WIDTH * b.V + c];
    const double isqg = fg[FG_ISQG * b.V + c];
    SideOut s[2];
    double rho[2], press[2], u[2][3], B[2][3];
    for (int side = 0; side < 2; side++) {
      const long cc = side == 0 ? c - st : c;
      const double* __restrict__ rr = w.rec + (side == 0 ? NREC : 0) * b.V + cc;
      rho[side] = rr[0];
      press[side] = rr[b.V];
      for (int q = 0; q < 3; q++) u[side][q] = rr[(2 + q) * b.V];
      B[side][D] = w.bf[D * b.V + c] * isqg;
      B[side][T1] = rr[5 * b.V];
      B[side][T2] = rr[6 * b.V];
      // the roots the recompute's face solve found (no Newton iteration here)
      const double rt[2] = {a.roots[((long)D * 4 + 2 * side) * b.V + c], a.roots[((long)D * 4 + 2 * side + 1) * b.V + c]};
      face_side(m, ia, width, D, rho[side], press[side], u[side], B[side], gamma, gfac, s[side], rt);
    }
    const double* lf = a.lface + (long)D * NFD * b.V + c;
    double lF[5], lvb[2];
    for (int v = 0; v < 5; v++) lF[v] = lf[(FD_F + v) * b.V];
    lvb[0] = lf[FD_VB1 * b.V];
    lvb[1] = lf[FD_VB2 * b.V];
    double lcmax = lf[FD_CMAX * b.V], lcmin = lf[FD_CMIN * b.V];
    const double lpL = s[0].lp, lpR = s[1].lp, lmL = s[0].lm, lmR = s[1].lm;
    const double cmax = fmax(0.0, fmax(lpL, lpR));
    const double cmin = -fmin(0.0, fmin(lmL, lmR));
    const double den = cmax + cmin;
    SideBar wb[2];
    for (int side = 0; side < 2; side++) {
      wb[side].lp = wb[side].lm = 0.0;
      for (int q = 0; q < 3; q++) wb[side].vt[q] = 0.0;
    }
    // Lax-Friedrichs: c_wave = max(c_max, c_min), its derivative to c_max on ties
    const bool cw_max = cmax >= cmin;
    const double cw = cw_max ? cmax : cmin;
    double extraB[2][2] = {{0.0, 0.0}, {0.0, 0.0}};  // adjoints of the sides' transverse B (induction fluxes)
    double gBnt = 0.0;                               // adjoint of the densitised face field (induction fluxes)
    if (fct) {
      // the induction fluxes along D of B~^T1, B~^T2 (v~^D B~^a - v~^a B~^D), reversed: the solver, then the
      // products of the sides' v~ and densitised B~
      const double Bnt = w.bf[D * b.V + c];
      for (int q = 0; q < 2; q++) {
        const int ax = q == 0 ? T1 : T2;
        const double lFb = lf[(FD_EB1 + q) * b.V];
        if (lFb == 0.0) continue;
        const double BL = m.sqg * B[0][ax], BR = m.sqg * B[1][ax];
        const double FL = s[0].vt[D] * BL - s[0].vt[ax] * Bnt, FR = s[1].vt[D] * BR - s[1].vt[ax] * Bnt;
        double gFL, gFR, gBL, gBR;
        if (den > 0.0 && lxf) {
          gFL = gFR = 0.5;
          gBL = 0.5 * cw;
          gBR = -0.5 * cw;
          if (cw_max) lcmax += -0.5 * (BR - BL) * lFb;
          else lcmin += -0.5 * (BR - BL) * lFb;
        } else if (den > 0.0) {
          const double id = 1.0 / den;
          const double Fh = (cmin * FR + cmax * FL - cmax * cmin * (BR - BL)) * id;
          gFL = cmax * id;
          gFR = cmin * id;
          gBL = cmax * cmin * id;
          gBR = -cmax * cmin * id;
          lcmax += (FL - cmin * (BR - BL) - Fh) * id * lFb;
          lcmin += (FR - cmax * (BR - BL) - Fh) * id * lFb;
        } else {
          gFL = gFR = 0.5;
          gBL = gBR = 0.0;
        }
        const double wFL = gFL * lFb, wFR = gFR * lFb;
        wb[0].vt[D] += wFL * BL;
        wb[0].vt[ax] -= wFL * Bnt;
        wb[1].vt[D] += wFR * BR;
        wb[1].vt[ax] -= wFR * Bnt;
        extraB[0][q] += m.sqg * (wFL * s[0].vt[D] + gBL * lFb);
        extraB[1][q] += m.sqg * (wFR * s[1].vt[D] + gBR * lFb);
        gBnt -= wFL * s[0].vt[ax] + wFR * s[1].vt[ax];
      }
    }
    if (den > 0.0) {
      const double id = 1.0 / den;
      if (lxf) {
        double lcw = 0.0;
        for (int v = 0; v < 5; v++) {
          const double dU = s[1].U[v] - s[0].U[v];
          wb[0].F[v] = 0.5 * lF[v];
          wb[1].F[v] = 0.5 * lF[v];
          wb[0].U[v] = 0.5 * cw * lF[v];
          wb[1].U[v] = -0.5 * cw * lF[v];
          lcw -= 0.5 * dU * lF[v];
        }
        if (cw_max) lcmax += lcw;
        else lcmin += lcw;
      } else {
        for (int v = 0; v < 5; v++) {
          const double dU = s[1].U[v] - s[0].U[v];
          const double Fh = (cmin * s[1].F[v] + cmax * s[0].F[v] - cmax * cmin * dU) * id;
          wb[0].F[v] = cmax * id * lF[v];
          wb[1].F[v] = cmin * id * lF[v];
          wb[0].U[v] = cmax * cmin * id * lF[v];
          wb[1].U[v] = -cmax * cmin * id * lF[v];
          lcmax += (s[0].F[v] - cmin * dU - Fh) * id * lF[v];
          lcmin += (s[1].F[v] - cmax * dU - Fh) * id * lF[v];
        }
      }
      const int tq[2] = {T1, T2};
      for (int q = 0; q < 2; q++) {
        const double vtL = s[0].vt[tq[q]], vtR = s[1].vt[tq[q]];
        const double vb = (cmax * vtL + cmin * vtR) * id;
        wb[0].vt[tq[q]] += cmax * id * lvb[q];
        wb[1].vt[tq[q]] += cmin * id * lvb[q];
        lcmax += (vtL - vb) * id * lvb[q];
        lcmin += (vtR - vb) * id * lvb[q];
      }
    } else {
      for (int v = 0; v < 5; v++) {
        wb[0].F[v] = wb[1].F[v] = 0.5 * lF[v];
        wb[0].U[v] = wb[1].U[v] = 0.0;
      }
      for (int side = 0; side < 2; side++) {
        wb[side].vt[T1] += 0.5 * lvb[0];
        wb[side].vt[T2] += 0.5 * lvb[1];
      }
    }
    // c_max = max(0, lp_L, lp_R), c_min = -min(0, lm_L, lm_R): the branch taken carries the derivative
    if (cmax > 0.0) {
      if (lpR > lpL) wb[1].lp = lcmax;
      else wb[0].lp = lcmax;
    }
    if (cmin > 0.0) {
      if (lmR < lmL) wb[1].lm = -lcmin;
      else wb[0].lm = -lcmin;
    }
    // left state = upper values of cell c - e_D, right state = lower values of cell c (each used once)
    double gBn = 0.0;
    for (int side = 0; side < 2; side++) {
      double gr, gp, gu[3], gB[3];
      face_side_vjp(m, ia, D, rho[side], press[side], u[side], B[side], gamma, gfac, s[side].lp, s[side].lm,
                    wb[side], gr, gp, gu, gB);
      double* lr = a.lrec + (side == 0 ? NREC * b.V + c - st : c);
      lr[0] = gr;
      lr[b.V] = gp;
      for (int q = 0; q < 3; q++) lr[(2 + q) * b.V] = gu[q];
      lr[5 * b.V] = gB[T1] + extraB[side][0];
      lr[6 * b.V] = gB[T2] + extraB[side][1];
      gBn += gB[D];
    }
    a.lBf[D * b.V + c] += gBn * isqg + gBnt;
  }
}

// Reconstruction along D (cells g-1 .. g+n along D, all transverse): each cell's (lower, upper) values of the 7
// variables from its 5-cell stencil; the adjoints scatter to the stencil cells.
template <int D, int SCHEME>
__global__ void ka_recon(Blk b, Ws w, AdjWs a) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  int lo[3] = {0, 0, 0}, ex[3] = {b.N[0], b.N[1], b.N[2]};
  lo[D] = b.g - 1;
  ex[D] = b.n[D] + 2;
  const long count = (long)ex[0] * ex[1] * ex[2];
  const long st = astr(b, D);
  ALOOP(t, count) {
    int p[3];
    decode(t, lo[0], ex[0], lo[1], ex[1], lo[2], p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    const double* src[NREC] = {a.P.f[0], a.P.f[1], w.uvel, w.uvel + b.V, w.uvel + 2 * b.V, w.bc + T1 * b.V,
                               w.bc + T2 * b.V};
    double* dst[NREC] = {a.lP, a.lP + b.V, a.lu, a.lu + b.V, a.lu + 2 * b.V, a.lBc + T1 * b.V, a.lBc + T2 * b.V};
    for (int v = 0; v < NREC; v++) {
      const double glo = a.lrec[v * b.V + c], ghi = a.lrec[(NREC + v) * b.V + c];
      if (glo == 0.0 && ghi == 0.0) continue;
      double g[5];
      if constexpr (SCHEME < 2) {  // minmod, PPM: reverse mode
        double a5[5];
        for (int s = 0; s < 5; s++) a5[s] = src[v][c + (s - 2) * st];
        recon5_vjp<SCHEME>(a5, glo, ghi, g);
      } else {  // WENO-Z, MP5: dual numbers through the forward code
        typedef Dual<5> D5;
        D5 s5[5];
        for (int s = 0; s < 5; s++) s5[s] = D5::seed(src[v][c + (s - 2) * st], s);
        D5 l, h;
        recon5<SCHEME>(s5, l, h);
        for (int s = 0; s < 5; s++) g[s] = l.d[s] * glo + h.d[s] * ghi;
      }
      for (int s = 0; s < 5; s++)
        if (g[s] != 0.0) atomicAdd(&dst[v][c + (s - 2) * st], g[s]);
    }
  }
}

// u^i = W v^i at every cell: lambda_v += (du/dv)^T lambda_u.
__global__ void ka_uvel(Blk b, Ws w, AdjWs a) {
  const long count = (long)b.N[0] * b.N[1] * b.N[2];
  ALOOP(t, count) {
    int i, j, k;
    decode(t, 0, b.N[0], 0, b.N[1], 0, i, j, k);
    const long c = alin(b, i, j, k);
    const double lu[3] = {a.lu[c], a.lu[b.V + c], a.lu[2 * b.V + c]};
    if (lu[0] == 0.0 && lu[1] == 0.0 && lu[2] == 0.0) continue;
    double g6[6];
    for (int q = 0; q < 6; q++) g6[q] = w.cg[(CG_G + q) * b.V + c];
    typedef Dual<3> D3;
    const D3 v[3] = {D3::seed(a.P.f[2][c], 0), D3::seed(a.P.f[3][c], 1), D3::seed(a.P.f[4][c], 2)};
    const D3 W = 1.0 / sqrt(1.0 - contract_sym(g6, v, v));
    for (int r = 0; r < 3; r++) {
      double acc = 0.0;
      for (int q = 0; q < 3; q++) acc += (W * v[q]).d[r] * lu[q];
      a.lP[(2 + r) * b.V + c] += acc;
    }
  }
}

// Transpose of one ghost sweep along AX: every ghost entry hands its adjoint to the owned entries it was
// copied or extrapolated from, then becomes zero.  Sweeps are transposed in the reverse order z, y, x.
template <int AX>
__device__ __forceinline__ void ka_ghost(Blk b, double* const* f, const int* cell_like, const int* linear, int nf) {
  constexpr int A1 = (AX + 1) % 3, A2 = (AX + 2) % 3;
  const int g = b.g, n = b.n[AX], Nn = b.N[AX];
  const long m1 = b.N[A1] + 1, m2 = b.N[A2] + 1;
  const int slots = 2 * g + 1;
  const long st = astr(b, AX);
  const long count = slots * m1 * m2;
  ALOOP(t, count) {
    int q, q1, q2;
    unflatten3(t, (unsigned)slots, (unsigned)m1, q, q1, q2);
    const int i = (q < g) ? q : Nn - 2 * g + q;
    int pp[3];
    pp[AX] = 0;
    pp[A1] = q1;
    pp[A2] = q2;
    const long base = alin(b, pp[0], pp[1], pp[2]);
    for (int fi = 0; fi < nf; fi++) {
      const bool cl = (cell_like[fi] >> AX) & 1;
      const int lo = g;
      const int hi = (cl || b.bc[AX] == 0) ? g + n - 1 : g + n;
      if (i >= lo && i <= hi) continue;
      double* aa = f[fi] + base;
      const double lam = aa[i * st];
      if (lam == 0.0) continue;
      aa[i * st] = 0.0;
      if (b.bc[AX] == 0) {
        const int src = lo + (((i - lo) % n) + n) % n;
        atomicAdd(&aa[src * st], lam);
      } else {
        const int e0 = (i < lo) ? lo : hi;
        if (linear[fi] && hi > lo) {
          const int e1 = (i < lo) ? lo + 1 : hi - 1;
          const double kk = (double)(i < lo ? lo - i : i - hi);
          atomicAdd(&aa[e0 * st], (1.0 + kk) * lam);
          atomicAdd(&aa[e1 * st], -kk * lam);
        } else {
          atomicAdd(&aa[e0 * st], lam);
        }
      }
    }
  }
}

// Recovery by the implicit-function theorem at the root: prim2con(P, B) = U, so with Jp = d prim2con / dP and
// Jb = d prim2con / dB (dual numbers through prim->cons), lambda_U += Jp^-T lambda_P and lambda_B -= Jb^T
// Jp^-T lambda_P.  Interior cells; atmosphere cells (flag 2 or -1) pass nothing.
__global__ void ka_c2p(Blk b, Ws w, AdjWs a, double gamma, double gfac) {
  const long count = (long)b.n[0] * b.n[1] * b.n[2];
  ALOOP(t, count) {
    int i, j, k;
    decode(t, b.g, b.n[0], b.g, b.n[1], b.g, i, j, k);
    const long c = alin(b, i, j, k);
    double lp[5];
    bool any = false;
    for (int r = 0; r < 5; r++) {
      lp[r] = a.lP[r * b.V + c];
      any = any || lp[r] != 0.0;
    }
    if (!any || a.flags[c] == 2 || a.flags[c] == -1) continue;
    Geo m;
    load_geo(b, w.cg, c, m);
    typedef Dual<8> D8;
    const D8 rho = D8::seed(a.P.f[0][c], 0), press = D8::seed(a.P.f[1][c], 1);
    const D8 v[3] = {D8::seed(a.P.f[2][c], 2), D8::seed(a.P.f[3][c], 3), D8::seed(a.P.f[4][c], 4)};
    const D8 B[3] = {D8::seed(w.bc[c], 5), D8::seed(w.bc[b.V + c], 6), D8::seed(w.bc[2 * b.V + c], 7)};
    const D8 W = 1.0 / sqrt(1.0 - contract_sym(m.g, v, v));
    const D8 u[3] = {W * v[0], W * v[1], W * v[2]};
    SideOutT<D8> o;
    face_side<D8, false>(m, 1.0 / m.alp, m.alp * sqrt(m.gu[0]), 0, rho, press, u, B, gamma, gfac, o);
    // solve Jp^T x = lambda_P (5x5, partial pivoting); Jp[row q][col r] = dU_q / dP_r
    double M[5][6];
    for (int r = 0; r < 5; r++) {
      for (int q = 0; q < 5; q++) M[r][q] = o.U[q].d[r];
      M[r][5] = lp[r];
    }
    for (int col = 0; col < 5; col++) {
      int piv = col;
      for (int r = col + 1; r < 5; r++)
        if (::fabs(M[r][col]) > ::fabs(M[piv][col])) piv = r;
      if (piv != col)
        for (int q = 0; q < 6; q++) {
          const double tmp = M[col][q];
          M[col][q] = M[piv][q];
          M[piv][q] = tmp;
        }
      const double inv = 1.0 / M[col][col];
      for (int r = col + 1; r < 5; r++) {
        const double f = M[r][col] * inv;
        for (int q = col; q < 6; q++) M[r][q] -= f * M[col][q];
      }
    }
    double x[5];
    for (int r = 4; r >= 0; r--) {
      double acc = M[r][5];
      for (int q = r + 1; q < 5; q++) acc -= M[r][q] * x[q];
      x[r] = acc / M[r][r];
    }
    for (int q = 0; q < 5; q++) a.lY[q * b.V + c] += x[q];
    for (int r = 0; r < 3; r++) {
      double acc = 0.0;
      for (int q = 0; q < 5; q++) acc += o.U[q].d[5 + r] * x[q];
      a.lBc[r * b.V + c] -= acc;
    }
  }
}

// Centre field B^d(c) = (B~^d(c) + B~^d(c + e_d)) / (2 sqrt(g_c)): each face gathers its two cells.
__global__ void ka_bcentre(Blk b, Ws w, AdjWs a) {
  const long count = b.V;
  ALOOP(t, count) {
    int p[3];
    decode(t, 0, b.N[0] + 1, 0, b.N[1] + 1, 0, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    for (int d = 0; d < 3; d++) {
      double acc = 0.0;
      // cell c (if it exists) and cell c - e_d (if it exists)
      bool cell_c = p[0] < b.N[0] && p[1] < b.N[1] && p[2] < b.N[2];
      if (cell_c) acc += 0.5 * a.lBc[d * b.V + c] / w.cg[CG_SQG * b.V + c];
      int q[3] = {p[0], p[1], p[2]};
      q[d] -= 1;
      bool cell_m = q[d] >= 0 && q[0] < b.N[0] && q[1] < b.N[1] && q[2] < b.N[2];
      if (cell_m) {
        const long cm = c - astr(b, d);
        acc += 0.5 * a.lBc[d * b.V + cm] / w.cg[CG_SQG * b.V + cm];
      }
      if (acc != 0.0) a.lBf[d * b.V + c] += acc;
    }
  }
}

// B~ = curl A on faces (transposed): each edge gathers the faces that difference it.
__global__ void ka_curl(Blk b, AdjWs a) {
  const long count = b.V;
  ALOOP(t, count) {
    int p[3];
    decode(t, 0, b.N[0] + 1, 0, b.N[1] + 1, 0, p[0], p[1], p[2]);
    const long c = alin(b, p[0], p[1], p[2]);
    const double* bx = a.lBf;
    const double* by = a.lBf + b.V;
    const double* bz = a.lBf + 2 * b.V;
    // validity of a face entry: x-faces need j < N1, k < N2; y-faces i < N0, k < N2; z-faces i < N0, j < N1
    auto fx = [&](int i, int j, int k) {
      return (i >= 0 && j >= 0 && k >= 0 && i <= b.N[0] && j < b.N[1] && k < b.N[2]) ? bx[alin(b, i, j, k)] : 0.0;
    };
    auto fy = [&](int i, int j, int k) {
      return (i >= 0 && j >= 0 && k >= 0 && i < b.N[0] && j <= b.N[1] && k < b.N[2]) ? by[alin(b, i, j, k)] : 0.0;
    };
    auto fz = [&](int i, int j, int k) {
      return (i >= 0 && j >= 0 && k >= 0 && i < b.N[0] && j < b.N[1] && k <= b.N[2]) ? bz[alin(b, i, j, k)] : 0.0;
    };
    const int i = p[0], j = p[1], k = p[2];
    // bx(c) = (Az(c+sy) - Az(c)) idy - (Ay(c+sz) - Ay(c)) idz
    // by(c) = (Ax(c+sz) - Ax(c)) idz - (Az(c+1) - Az(c)) idx
    // bz(c) = (Ay(c+1) - Ay(c)) idx - (Ax(c+sy) - Ax(c)) idy
    const double lAx = (fy(i, j, k - 1) - fy(i, j, k)) * b.idx[2] - (fz(i, j - 1, k) - fz(i, j, k)) * b.idx[1];
    const double lAy = (fz(i - 1, j, k) - fz(i, j, k)) * b.idx[0] - (fx(i, j, k - 1) - fx(i, j, k)) * b.idx[2];
    const double lAz = (fx(i, j - 1, k) - fx(i, j, k)) * b.idx[1] - (fy(i - 1, j, k) - fy(i, j, k)) * b.idx[0];
    a.lY[5 * b.V + c] += lAx;
    a.lY[6 * b.V + c] += lAy;
    a.lY[7 * b.V + c] += lAz;
  }
}

struct GhostArgs {
  double* f[9];
  int cl[9];
  int lin[9];
};

template <int AX>
__global__ void ka_ghost_k(Blk b, GhostArgs g, int nf) {
  ka_ghost<AX>(b, g.f, g.cl, g.lin, nf);
}

void launch_ghost_adjoint(const Blk& b, const AdjGhost& ag, int nf, cudaStream_t s) {
  GhostArgs g;
  for (int f = 0; f < nf; f++) {
    g.f[f] = ag.f[f];
    g.cl[f] = ag.cl[f];
    g.lin[f] = ag.lin[f];
  }
  const int T = 128;
  const int slots = 2 * b.g + 1;
  ka_ghost_k<2><<<agrid((long)slots * (b.N[0] + 1) * (b.N[1] + 1), T), T, 0, s>>>(b, g, nf);
  ka_ghost_k<1><<<agrid((long)slots * (b.N[2] + 1) * (b.N[0] + 1), T), T, 0, s>>>(b, g, nf);
  ka_ghost_k<0><<<agrid((long)slots * (b.N[1] + 1) * (b.N[2] + 1), T), T, 0, s>>>(b, g, nf);
}

// field q of a pointer set, chosen with constant indices (a runtime index into a kernel parameter struct makes
// the compiler copy the whole struct to local memory in every thread)
template <class FS, int NF>
__device__ __forceinline__ double* field_at(const FS& x, int q) {
  double* p = x.f[0];
#pragma unroll
  for (int r = 1; r < NF; r++)
    if (q == r) p = x.f[r];
  return p;
}

// elementwise helpers of the RK4 adjoint (grid y = the field)
__global__ void ka_axpby9(Blk b, double alpha, F9 x, double beta, F9 y) {
  const double* __restrict__ xf = field_at<F9, 9>(x, blockIdx.y);
  double* __restrict__ yf = field_at<F9, 9>(y, blockIdx.y);
  ALOOP(c, b.V) yf[c] = alpha * xf[c] + beta * yf[c];
}

// Keeps the independent entries: g..g+n-1 along cell-like axes and along periodic axes (where the vertex index
// g+n is the periodic image of g), g..g+n along vertex-like axes with copy BCs.
__global__ void ka_mask_owned9(Blk b, F9 x) {
  const int f = blockIdx.y;
  const int clf = f < 5 ? 7 : (f == 5 ? 1 : (f == 6 ? 2 : (f == 7 ? 4 : 0)));  // bit d: cell-like along d
  int hi[3];
  for (int d = 0; d < 3; d++) hi[d] = (((clf >> d) & 1) || b.bc[d] == 0) ? b.g + b.n[d] - 1 : b.g + b.n[d];
  double* __restrict__ xf = field_at<F9, 9>(x, f);
  ALOOP(c, b.V) {
    int p[3];
    decode(c, 0, b.N[0] + 1, 0, b.N[1] + 1, 0, p[0], p[1], p[2]);
    bool own = true;
    for (int d = 0; d < 3; d++) own = own && p[d] >= b.g && p[d] <= hi[d];
    if (!own) xf[c] = 0.0;
  }
}

cudaError_t launch_axpby9(const Blk& b, double alpha, const F9& x, double beta, const F9& y, cudaStream_t s) {
  ka_axpby9<<<dim3(agrid(b.V, 256), 9), 256, 0, s>>>(b, alpha, x, beta, y);
  return cudaGetLastError();
}

cudaError_t launch_mask_owned9(const Blk& b, const F9& x, cudaStream_t s) {
  ka_mask_owned9<<<dim3(agrid(b.V, 256), 9), 256, 0, s>>>(b, x);
  return cudaGetLastError();
}

// Initial data: U_hydro = prim2con(P, B) at the interior cells (Eq. cons), B the centre field of curl A.
// lamP = (dU/dP)^T lamU, lambda_B = (dU/dB)^T lamU, both from dual numbers through prim->cons.
__global__ void ka_prim2con(Blk b, Ws w, AdjWs a, F9 lamU, F5 lamP, double gamma, double gfac) {
  const long count = (long)b.n[0] * b.n[1] * b.n[2];
  ALOOP(t, count) {
    int i, j, k;
    decode(t, b.g, b.n[0], b.g, b.n[1], b.g, i, j, k);
    const long c = alin(b, i, j, k);
    Geo m;
    load_geo(b, w.cg, c, m);
    typedef Dual<8> D8;
    const D8 rho = D8::seed(a.P.f[0][c], 0), press = D8::seed(a.P.f[1][c], 1);
    const D8 v[3] = {D8::seed(a.P.f[2][c], 2), D8::seed(a.P.f[3][c], 3), D8::seed(a.P.f[4][c], 4)};
    const D8 B[3] = {D8::seed(w.bc[c], 5), D8::seed(w.bc[b.V + c], 6), D8::seed(w.bc[2 * b.V + c], 7)};
    const D8 W = 1.0 / sqrt(1.0 - contract_sym(m.g, v, v));
    const D8 u[3] = {W * v[0], W * v[1], W * v[2]};
    SideOutT<D8> o;
    face_side<D8, false>(m, 1.0 / m.alp, m.alp * sqrt(m.gu[0]), 0, rho, press, u, B, gamma, gfac, o);
    double g8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 5; q++) {
      const double l = lamU.f[q][c];
      for (int r = 0; r < 8; r++) g8[r] += o.U[q].d[r] * l;
    }
    for (int r = 0; r < 5; r++) lamP.f[r][c] = g8[r];
    for (int r = 0; r < 3; r++) a.lBc[r * b.V + c] = g8[5 + r];
  }
}

__global__ void ka_zero5(Blk b, F5 x) {  // grid y = the field
  double* __restrict__ xf = field_at<F5, 5>(x, blockIdx.y);
  ALOOP(c, b.V) xf[c] = 0.0;
}

// the workspace as the kept intermediates of one stage see it
static Ws kept_ws(const StageArgs& sa, const AdjWs& a) {
  Ws w = sa.w;
  w.bf = a.kbf;
  w.bc = a.kbc;
  w.uvel = a.kuvel;
  w.face = a.kface;
  return w;
}

cudaError_t launch_prim2con_adjoint(const StageArgs& sa, const AdjWs& a, const F9& lamU, const F5& lamP,
                                    cudaStream_t s) {
  const Blk& b = sa.b;
  const int T = 128;
  const Ws w = kept_ws(sa, a);
  cudaError_t e = launch_ghost_state(b, a.Y, s);
  if (e == cudaSuccess) e = launch_bfield(b, w, a.Y, s);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(a.lY_base, 0, (size_t)ADJ_ACC_FIELDS * b.V * sizeof(double), s);
  ka_zero5<<<dim3(agrid(b.V, 256), 5), 256, 0, s>>>(b, lamP);
  ka_prim2con<<<agrid((long)b.n[0] * b.n[1] * b.n[2], T), T, 0, s>>>(b, w, a, lamU, lamP, sa.gamma, sa.gfac);
  ka_bcentre<<<agrid(b.V, T), T, 0, s>>>(b, w, a);
  ka_curl<<<agrid(b.V, T), T, 0, s>>>(b, a);
  F9 ly;
  for (int v = 0; v < 9; v++) ly.f[v] = a.lY + v * b.V;
  AdjGhost g;
  const int cl[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};
  for (int f = 0; f < 9; f++) {
    g.f[f] = ly.f[f];
    g.cl[f] = cl[f];
    g.lin[f] = (f >= 5 && f <= 7);
  }
  launch_ghost_adjoint(b, g, 9, s);
  // the potentials' own adjoints pass through unchanged: lY += lamU, then the hydro entries are cleared
  e = launch_axpby9(b, 1.0, lamU, 1.0, ly, s);
  if (e == cudaSuccess) e = launch_mask_owned9(b, ly, s);
  if (e != cudaSuccess) return e;
  for (int v = 0; v < 5; v++) cudaMemsetAsync(ly.f[v], 0, b.V * sizeof(double), s);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------------------------
// Orchestration of the VJP of the right-hand side at the state held in a.Y (ghost fill, recovery and the
// forward intermediates are recomputed here); mu on owned ranges in a.mu; result in a.lY (owned ranges).

template <int D>
static void adjoint_dir(const StageArgs& sa, const AdjWs& a, cudaStream_t s) {
  const Blk& b = sa.b;
  const int T = 128;
  Ws w = sa.w;
  w.rec = a.rec3[D];  // this direction's reconstruction, kept from the recompute
  const long fc = (long)b.N[0] * b.N[1] * b.N[2] / b.N[D] * (b.n[D] + 1);
  cudaMemsetAsync(a.lrec, 0, 2 * NREC * b.V * sizeof(double), s);
  if (sa.flux == 1 || sa.efield == 1)
    ka_faces<D, true><<<agrid(fc, T), T, 0, s>>>(b, w, a, sa.gamma, sa.gfac, sa.flux == 1, sa.efield == 1);
  else
    ka_faces<D, false><<<agrid(fc, T), T, 0, s>>>(b, w, a, sa.gamma, sa.gfac, 0, 0);
  const long rc = (long)b.N[0] * b.N[1] * b.N[2] / b.N[D] * (b.n[D] + 2);
  if (sa.recon == 0) ka_recon<D, 0><<<agrid(rc, T), T, 0, s>>>(b, w, a);
  else if (sa.recon == 1) ka_recon<D, 1><<<agrid(rc, T), T, 0, s>>>(b, w, a);
  else if (sa.recon == 3) ka_recon<D, 3><<<agrid(rc, T), T, 0, s>>>(b, w, a);
  else ka_recon<D, 2><<<agrid(rc, T), T, 0, s>>>(b, w, a);
}

cudaError_t launch_adjoint_forward(const StageArgs& sa, const AdjWs& a, cudaStream_t s) {
  StageArgs k = sa;
  k.w = kept_ws(sa, a);
  const Blk& b = sa.b;
  cudaError_t e = launch_ghost_state(b, a.Y, s);
  if (e == cudaSuccess) e = launch_bfield(b, k.w, a.Y, s);
  if (e == cudaSuccess) e = launch_c2p(k, a.Y, a.P, a.flags, nullptr, s);
  if (e == cudaSuccess) e = launch_ghost_prims(b, a.P, s);
  if (e == cudaSuccess) e = launch_face_data(k, a.P, a.rec3, a.roots, s);
  return e;
}

cudaError_t launch_adjoint_reverse(const StageArgs& sa0, const AdjWs& a, double dt, cudaStream_t s) {
  StageArgs sa = sa0;
  sa.w = kept_ws(sa0, a);
  const Blk& b = sa.b;
  const int T = 128;
  // adjoint accumulators
  cudaMemsetAsync(a.lY_base, 0, (size_t)ADJ_ACC_FIELDS * b.V * sizeof(double), s);
  const int lorenz = (sa.gauge == 0);
  const double xi = sa.xi > 0.0 ? sa.xi : 1.5 / dt;
  for (int D = 0; D < 3; D++) {
    const long fc = (long)b.n[0] * b.n[1] * b.n[2] / b.n[D] * (b.n[D] + 1);
    ka_flux_div<<<agrid(fc, T), T, 0, s>>>(b, a, a.mu, D);
  }
  ka_sources<<<agrid((long)b.n[0] * b.n[1] * b.n[2], T), T, 0, s>>>(b, sa.w, a, a.P, a.mu, sa.gfac);
  const long vc = (long)(b.n[0] + 3) * (b.n[1] + 3) * (b.n[2] + 3);
  if (lorenz) ka_psi<<<agrid(vc, T), T, 0, s>>>(b, sa.w, a, a.mu, xi);
  ka_grad_ga<<<agrid(vc, T), T, 0, s>>>(b, a, a.mu);
  const long ec = (long)(b.n[0] + 1) * (b.n[1] + 1) * (b.n[2] + 1);
  ka_edges<0><<<agrid(ec, T), T, 0, s>>>(b, sa.w, a, a.mu, sa.efield == 1);
  ka_edges<1><<<agrid(ec, T), T, 0, s>>>(b, sa.w, a, a.mu, sa.efield == 1);
  ka_edges<2><<<agrid(ec, T), T, 0, s>>>(b, sa.w, a, a.mu, sa.efield == 1);
  ka_vertex<<<agrid(vc, T), T, 0, s>>>(b, sa.w, a, lorenz);
  ka_vertex_to_edges<<<agrid((long)(b.n[0] + 4) * (b.n[1] + 4) * (b.n[2] + 4), T), T, 0, s>>>(b, a);
  adjoint_dir<0>(sa, a, s);
  adjoint_dir<1>(sa, a, s);
  adjoint_dir<2>(sa, a, s);
  ka_uvel<<<agrid((long)b.N[0] * b.N[1] * b.N[2], T), T, 0, s>>>(b, sa.w, a);
  // primitive ghost fill, transposed (z, y, x)
  {
    AdjGhost g;
    for (int f = 0; f < 5; f++) {
      g.f[f] = a.lP + f * b.V;
      g.cl[f] = 7;
      g.lin[f] = 0;
    }
    launch_ghost_adjoint(b, g, 5, s);
  }
  ka_c2p<<<agrid((long)b.n[0] * b.n[1] * b.n[2], T), T, 0, s>>>(b, sa.w, a, sa.gamma, sa.gfac);
  ka_bcentre<<<agrid(b.V, T), T, 0, s>>>(b, sa.w, a);
  ka_curl<<<agrid(b.V, T), T, 0, s>>>(b, a);
  {
    AdjGhost g;
    const int cl[9] = {7, 7, 7, 7, 7, 1, 2, 4, 0};
    for (int f = 0; f < 9; f++) {
      g.f[f] = a.lY + f * b.V;
      g.cl[f] = cl[f];
      g.lin[f] = (f >= 5 && f <= 7);
    }
    launch_ghost_adjoint(b, g, 9, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_rhs_adjoint(const StageArgs& sa, const AdjWs& a, double dt, cudaStream_t s) {
  cudaError_t e = launch_adjoint_forward(sa, a, s);
  if (e == cudaSuccess) e = launch_adjoint_reverse(sa, a, dt, s);
  return e;
}

}  // namespace asterx
