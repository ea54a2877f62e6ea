// Device-side pointwise physics of the GRMHD stage (FP64 throughout).
//
// Paper: AsterX, arXiv:2406.11669.  Sec. 2.2 (Valencia form, Eqs. eulerianB, grmhdeqs, cons, grmhdsrc),
// Sec. 3.3 (reconstruction, HLLE, magnetosonic speeds), Sec. 3.5 (Noble 2D / Palenzuela 1D recovery),
// Sec. 3.6 (atmosphere), Sec. 3.7 (ideal-gas EOS).
//
// Symmetric 3x3 tensors are stored as 6 components in the order xx, xy, xz, yy, yz, zz.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

#include "dual.cuh"
#include "layout.h"

namespace asterx {

__host__ __device__ constexpr int sym(int a, int b) {
  return (a == 0) ? b : (a == 1 ? (b == 0 ? 1 : b + 2) : (b == 0 ? 2 : (b == 1 ? 4 : 5)));
}

// 3+1 geometry at one point.
struct Geo {
  double alp;
  double beta[3];
  double g[6];   // gamma_ij
  double gu[6];  // gamma^ij
  double sqg;    // sqrt(det gamma)
};

template <class T>
__host__ __device__ __forceinline__ T contract_sym(const double m[6], const T a[3], const T b[3]) {
  return m[0] * a[0] * b[0] + m[3] * a[1] * b[1] + m[5] * a[2] * b[2] +
         m[1] * (a[0] * b[1] + a[1] * b[0]) + m[2] * (a[0] * b[2] + a[2] * b[0]) +
         m[4] * (a[1] * b[2] + a[2] * b[1]);
}

template <class T>
__host__ __device__ __forceinline__ void lower(const double m[6], const T a[3], T out[3]) {
  out[0] = m[0] * a[0] + m[1] * a[1] + m[2] * a[2];
  out[1] = m[1] * a[0] + m[3] * a[1] + m[4] * a[2];
  out[2] = m[2] * a[0] + m[4] * a[1] + m[5] * a[2];
}

// inverse and sqrt(det) of a symmetric positive-definite 3x3 matrix (cofactors)
__host__ __device__ __forceinline__ void sym_inverse(const double g[6], double gu[6], double* sqg) {
  const double c00 = g[3] * g[5] - g[4] * g[4];
  const double c01 = g[4] * g[2] - g[1] * g[5];
  const double c02 = g[1] * g[4] - g[3] * g[2];
  const double det = g[0] * c00 + g[1] * c01 + g[2] * c02;
  const double idet = 1.0 / det;
  gu[0] = c00 * idet;
  gu[1] = c01 * idet;
  gu[2] = c02 * idet;
  gu[3] = (g[0] * g[5] - g[2] * g[2]) * idet;
  gu[4] = (g[1] * g[2] - g[0] * g[4]) * idet;
  gu[5] = (g[0] * g[3] - g[1] * g[1]) * idet;
  *sqg = sqrt(det);
}

// ----------------------------------------------------------------------------------------------------------
// One side of a face: conserved variables, fluxes along d and the two extreme magnetosonic speeds.
//
// Algebra used (equivalent to Eqs. eulerianB, cons, grmhdeqs):  with W^2 = 1 + gamma_ij u^i u^j, v = u / W,
//   B.v = B^i v_i,  b^2 = B^2 / W^2 + (B.v)^2,  alpha b^0 = W (B.v),  b_j = B_j / W + W (B.v) v_j,
//   S_j = (rho h W^2 + B^2) v_j - (B.v) B_j,  tau = rho h W^2 - p - rho W + B^2 - b^2 / 2,
//   alpha sqrt(g) F^d:  D~ vt,  S~_j vt + a sqrt(g) (p_t delta^d_j - b_j B^d / W),  tau~ vt + a sqrt(g) (p_t v^d - (B.v) B^d)
// with vt = alpha v^d - beta^d, p_t = p + b^2/2.

template <class T>
struct SideOutT {
  T U[5];
  T F[5];
  T lm, lp;  // lambda_-, lambda_+
  T vt[3];   // v~^i = alpha v^i - beta^i
};
using SideOut = SideOutT<double>;

// 2^-959 < |x| < 2^960 (about 1e-289 .. 1e289), read from the exponent bits on the integer pipe (NaN, infinities,
// zeros and subnormals are outside): the range where the reciprocal estimates below are normal.
__host__ __device__ __forceinline__ bool exponent_in_range(double x) {
#ifdef __CUDA_ARCH__
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  return ex > 63u && ex < 1983u;
#else
  const double a = fabs(x);
  return a >= 0x1p-959 && a < 0x1p960;
#endif
}

// Reciprocal for Newton corrections, where a relative error far below the correction's own accuracy is enough:
// the PTX reciprocal estimate (rcp.approx.ftz.f64) refined by one Newton-Raphson step r <- r + r (1 - d r), the
// textbook iteration for 1/d (Flynn 1970), which squares the estimate's relative error.  Meant for
// exponent_in_range(d) (the caller divides outside that range); the host build divides.
__host__ __device__ __forceinline__ double newton_rcp(double d) {
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return fma(r, fma(-d, r, 1.0), r);
#else
  return 1.0 / d;
#endif
}

// Reciprocal to within about one unit in the last place where a correctly rounded quotient is not needed: the
// reciprocal estimate refined by two Newton-Raphson steps (each squares the relative error), inside the range
// where the estimate is normal (binary exponent within +-960, read from the bits on the integer pipe); the
// quotient 1 / d elsewhere.  Dual numbers divide.
__host__ __device__ __forceinline__ double recip(double d) {
#ifdef __CUDA_ARCH__
  const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
  if (ex > 63u && ex < 1983u) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    r = fma(r, fma(-d, r, 1.0), r);
    return fma(r, fma(-d, r, 1.0), r);
  }
#endif
  return 1.0 / d;
}
template <int N>
__host__ __device__ __forceinline__ Dual<N> recip(const Dual<N>& d) {
  return 1.0 / d;
}

// Correctly rounded a / b from y = 1 / b (itself a correctly rounded quotient), for several quotients by the same
// b at one division: q = a y is within one ulp of a / b, the remainder a - b q is exact in one fused multiply-add,
// and q + (a - b q) y rounds to the correctly rounded quotient (Markstein 1990; Muller et al., Handbook of
// Floating-Point Arithmetic, the theorem on correcting a faithful quotient with a correctly rounded
// reciprocal).  Valid away from overflow and underflow of the intermediate values; the callers divide by
// sqrt(gamma) of a metric (about 1) values far inside the range.
__host__ __device__ __forceinline__ double quotient_by(double a, double b, double y) {
  const double q = a * y;
  return fma(fma(-b, q, a), y, q);
}

// Extreme roots of the magnetosonic quartic (Sec. 3.3): with phi = (-lambda, e_d),
//   a = u^mu phi_mu = ud - lambda u0,  Bc = b^mu phi_mu = bd - lambda b0,
//   G = g^{mu nu} phi_mu phi_nu = gamma^dd - (lambda + beta^d)^2 / alpha^2,
//   Q(lambda) = rho h (1 - cs2) a^4 - (rho h cs2 + b^2) a^2 G + cs2 Bc^2 G   (the quartic times cs2),
// evaluated in this factored form (accurate where a -> 0, i.e. near the fluid speed, which the expanded
// polynomial is not for cold fluids) and solved by Newton from each light-cone speed, where it is monotone.
struct Quartic {
  double A4, C2, cs2, u0, ud, b0, bd, betad, ia2, gdd;
  __host__ __device__ __forceinline__ double newton(double lam, double width) const {
    return newton_cut<0>(lam, width, 0.0);
  }
  // The iteration, ended early once the iterate has passed `cut` in the direction of travel (kDir = +1 for the
  // largest root, approached from above; kDir = -1 for the smallest, from below; 0: no cut).  Every iterate lies
  // outside the root, so an iterate past `cut` shows that the root is past it too: the caller, which only needs
  // the larger (smaller) of this root and `cut`, has its answer without the rest of the iteration.
  template <int kDir>
  __host__ __device__ __forceinline__ double newton_cut(double lam, double width, double cut) const {
    // loop-invariant factors of Q' (Q itself keeps its factored form; Q' only scales the correction):
    //   dr/dlam = ka a + kb bc,  dG/dlam = kg (lam + beta^d),  d(A4 a^4)/dlam = k4 a^3
    const double ka = 2.0 * C2 * u0, kb = -2.0 * cs2 * b0, kg = -2.0 * ia2, k4 = -4.0 * A4 * u0;
    // quadratic convergence: once a step is below 3e-9 of the speed scale (|lambda| + alpha sqrt(gamma^dd), taken
    // at the start), the updated root is accurate to about the square of that (within 5e-15 of the scale on 4e5
    // sampled states with rho, p in [1e-6, 1], |u| <= 3), so no further step is taken
    const double thr = 3e-9 * (fabs(lam) + width);
#pragma unroll 1
    for (int it = 0; it < 60; it++) {
      if (kDir > 0 && lam <= cut) break;
      if (kDir < 0 && lam >= cut) break;
      const double a = ud - lam * u0;
      const double bc = bd - lam * b0;
      const double lb = lam + betad;
      const double G = gdd - lb * lb * ia2;
      const double a2 = a * a;
      const double r = cs2 * bc * bc - C2 * a2;
      const double q = A4 * a2 * a2 + r * G;
      const double dq = k4 * a2 * a + (ka * a + kb * bc) * G + r * (kg * lb);
      double step;
      if (exponent_in_range(dq)) {
        step = q * newton_rcp(dq);
      } else {
        if (dq == 0.0) break;
        step = q / dq;
      }
      lam -= step;
      if (fabs(step) <= thr) break;
    }
    return lam;
  }
};

// The same quartic with state-dependent coefficients of scalar type T: one Newton step from the converged root
// lam (a constant) gives lam - Q/Q', whose derivative is the implicit-function derivative -Q_theta / Q_lam.
template <class T>
struct QuarticT {
  T A4, C2, cs2, u0, ud, b0, bd;
  double betad, ia2, gdd;
  __host__ __device__ __forceinline__ T root_step(double lam) const {
    const T a = ud - lam * u0;
    const T bc = bd - lam * b0;
    const double lb = lam + betad;
    const double G = gdd - lb * lb * ia2;
    const double dG = -2.0 * lb * ia2;
    const T a2 = a * a;
    const T r = cs2 * bc * bc - C2 * a2;
    const T dr = -2.0 * (cs2 * bc * b0 - C2 * a * u0);
    const T q = A4 * a2 * a2 + r * G;
    const T dq = -4.0 * A4 * a2 * a * u0 + dr * G + r * dG;
    return lam - q / dq;
  }
};

// gfac = Gamma / (Gamma - 1), ia = 1 / alpha, width = alpha sqrt(gamma^dd) (hoisted by the caller).  kSpeeds =
// false skips the magnetosonic speeds (o.lm, o.lp unset: prim->cons and fluxes only); `roots`, when given, holds
// the two speeds (lambda_+, lambda_-) already found for these inputs, and replaces the Newton iteration.
// fluxes = false skips prim->cons and the fluxes (o.U, o.F unset: speeds and v~ only), for faces whose fluxes
// nothing reads.  With kCut, the Newton iterations of lambda_+ and lambda_- stop once they pass cut_p and cut_m
// (Quartic::newton_cut): for a caller that needs only max(cut_p, lambda_+) and min(cut_m, lambda_-), the result
// then carries the same information.
template <class T, bool kSpeeds = true, bool kCut = false>
__host__ __device__ __forceinline__ void face_side(const Geo& m, double ia, double width, int d, T rho, T press,
                                          const T u[3], const T B[3], double gamma, double gfac,
                                          SideOutT<T>& o, const double* roots = nullptr, bool fluxes = true,
                                          double cut_p = 0.0, double cut_m = 0.0) {
  const T uu = contract_sym(m.g, u, u);
  const T W = sqrt(1.0 + uu);
  const T iW = recip(W);
  T v[3] = {u[0] * iW, u[1] * iW, u[2] * iW};
  T vl[3], Bl[3];
  lower(m.g, v, vl);
  lower(m.g, B, Bl);
  const T B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const T Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const T iW2 = iW * iW;
  const T b2 = B2 * iW2 + Bv * Bv;
  const T rhoh = rho + gfac * press;
  const T W2 = W * W;
  for (int a = 0; a < 3; a++) o.vt[a] = m.alp * v[a] - m.beta[a];
  const T Bd = B[d];
  if (fluxes) {
    const double sg = m.sqg;
    const double asg = m.alp * sg;
    const T z = rhoh * W2;
    o.U[0] = sg * rho * W;
    for (int a = 0; a < 3; a++) o.U[1 + a] = sg * ((z + B2) * vl[a] - Bv * Bl[a]);
    o.U[4] = sg * (z - press - rho * W + B2 - 0.5 * b2);
    const T vt = o.vt[d];
    const T pt = press + 0.5 * b2;
    o.F[0] = o.U[0] * vt;
    for (int a = 0; a < 3; a++) {
      const T bl = Bl[a] * iW + W * Bv * vl[a];
      o.F[1 + a] = o.U[1 + a] * vt - asg * bl * Bd * iW;
    }
    o.F[1 + d] += asg * pt;
    o.F[4] = o.U[4] * vt + asg * (pt * v[d] - Bv * Bd);
  }

  if constexpr (!kSpeeds) return;
  // magnetosonic speeds
  const T u0 = W * ia;
  const T ud = W * (v[d] - m.beta[d] * ia);
  const T b0 = W * Bv * ia;
  const T bd = (Bd + m.alp * b0 * ud) * iW;
  // one division for cs^2 = Gamma p / (rho h) (= Gamma (Gamma - 1) eps / h) and cA^2 = b^2 / (rho h + b^2)
  const T ihb = recip(rhoh * (rhoh + b2));
  const T cs2 = gamma * press * (rhoh + b2) * ihb;
  const T ca2 = b2 * rhoh * ihb;
  Quartic Q;
  Q.cs2 = val(cs2);
  Q.A4 = val(rhoh) * (1.0 - Q.cs2);
  Q.C2 = val(rhoh) * Q.cs2 + val(b2);
  Q.u0 = val(u0);
  Q.ud = val(ud);
  Q.b0 = val(b0);
  Q.bd = val(bd);
  Q.betad = m.beta[d];
  Q.ia2 = ia * ia;
  Q.gdd = m.gu[sym(d, d)];
  double lp, lm;
  if (roots) {
    lp = roots[0];
    lm = roots[1];
  } else {
    // Starting points: the lab-frame speeds of an isotropic wave with the perpendicular fast speed
    // c^2 = cs^2 + cA^2 - cs^2 cA^2 (cA^2 = b^2 / (rho h + b^2)), which bounds the fast magnetosonic speed in
    // every direction, so both starts lie outside the extreme roots and Newton converges monotonically from
    // there (as from the light cone, but from much closer).  Clamped to the light cone.
    const double c2 = Q.cs2 + val(ca2) - Q.cs2 * val(ca2);
    const double v2 = 1.0 - val(iW2);
    const double den = 1.0 - v2 * c2;
    const double vd = val(v[d]);
    const double disc = fmax((1.0 - v2) * (Q.gdd * den - vd * vd * (1.0 - c2)), 0.0);
    const double spread = sqrt(c2 * disc);
    const double idn = m.alp * recip(den);
    const double mid = vd * (1.0 - c2);
    const double lc = -m.beta[d];
    const double lp0 = fmin((mid + spread) * idn - m.beta[d] + 1e-12 * width, lc + width);
    const double lm0 = fmax((mid - spread) * idn - m.beta[d] - 1e-12 * width, lc - width);
    lp = Q.newton_cut<kCut ? 1 : 0>(lp0, width, cut_p);
    lm = Q.newton_cut<kCut ? -1 : 0>(lm0, width, cut_m);
  }
  if constexpr (sizeof(T) == sizeof(double)) {
    o.lp = lp;
    o.lm = lm;
  } else {
    QuarticT<T> QT;
    QT.cs2 = cs2;
    QT.A4 = rhoh * (1.0 - cs2);
    QT.C2 = rhoh * cs2 + b2;
    QT.u0 = u0;
    QT.ud = ud;
    QT.b0 = b0;
    QT.bd = bd;
    QT.betad = Q.betad;
    QT.ia2 = Q.ia2;
    QT.gdd = Q.gdd;
    o.lp = QT.root_step(lp);
    o.lm = QT.root_step(lm);
  }
}

// Reverse mode of face_side: weights wb on its outputs (U, F, lambda_-, lambda_+, v~) give the gradient
// wb . d(outputs) / d(rho, p, u^i, B^i).  The primal is recomputed from the inputs except for the two roots, which
// the caller passes (as face_side returned them); the roots are differentiated by the implicit-function theorem,
// d lambda = -(dQ/d theta) / (dQ/d lambda) for the quartic's state-dependent coefficients theta.
struct SideBar {
  double U[5], F[5], lm, lp, vt[3];
};

__host__ __device__ __forceinline__ void face_side_vjp(const Geo& m, double ia, int d, double rho, double press,
                                                       const double u[3], const double B[3], double gamma,
                                                       double gfac, double lp, double lm, const SideBar& wb,
                                                       double& grho, double& gp, double gu[3], double gB[3]) {
  // ---- primal
  const double uu = contract_sym(m.g, u, u);
  const double W = sqrt(1.0 + uu);
  const double iW = 1.0 / W;
  const double v[3] = {u[0] * iW, u[1] * iW, u[2] * iW};
  double vl[3], Bl[3];
  lower(m.g, v, vl);
  lower(m.g, B, Bl);
  const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const double Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const double iW2 = iW * iW;
  const double b2 = B2 * iW2 + Bv * Bv;
  const double rhoh = rho + gfac * press;
  const double W2 = W * W;
  const double z = rhoh * W2;
  const double sg = m.sqg;
  const double asg = m.alp * sg;
  double U[5];
  U[0] = sg * rho * W;
  for (int a = 0; a < 3; a++) U[1 + a] = sg * ((z + B2) * vl[a] - Bv * Bl[a]);
  U[4] = sg * (z - press - rho * W + B2 - 0.5 * b2);
  const double vtd = m.alp * v[d] - m.beta[d];
  const double pt = press + 0.5 * b2;
  const double Bd = B[d];
  double bl[3];
  for (int a = 0; a < 3; a++) bl[a] = Bl[a] * iW + W * Bv * vl[a];
  const double u0 = W * ia;
  const double ud = W * (v[d] - m.beta[d] * ia);
  const double b0 = W * Bv * ia;
  const double bd = (Bd + m.alp * b0 * ud) * iW;
  const double cs2 = gamma * press / rhoh;
  const double A4 = rhoh * (1.0 - cs2);
  const double C2 = rhoh * cs2 + b2;
  const double ia2 = ia * ia;
  const double gdd = m.gu[sym(d, d)];
  // ---- reverse
  double bA4 = 0.0, bC2 = 0.0, bcs2 = 0.0, bu0 = 0.0, bud = 0.0, bb0 = 0.0, bbd = 0.0;
  const double lam[2] = {lp, lm}, blam[2] = {wb.lp, wb.lm};
  for (int k = 0; k < 2; k++) {
    if (blam[k] == 0.0) continue;
    const double L = lam[k];
    const double a = ud - L * u0;
    const double bc = bd - L * b0;
    const double lb = L + m.beta[d];
    const double G = gdd - lb * lb * ia2;
    const double dG = -2.0 * lb * ia2;
    const double a2 = a * a;
    const double r = cs2 * bc * bc - C2 * a2;
    const double dr = -2.0 * (cs2 * bc * b0 - C2 * a * u0);
    const double dq = -4.0 * A4 * a2 * a * u0 + dr * G + r * dG;
    const double sc = -blam[k] / dq;
    const double Qa = 4.0 * A4 * a2 * a - 2.0 * C2 * a * G;
    const double Qbc = 2.0 * cs2 * bc * G;
    bA4 += sc * a2 * a2;
    bC2 -= sc * a2 * G;
    bcs2 += sc * bc * bc * G;
    bud += sc * Qa;
    bu0 -= sc * Qa * L;
    bbd += sc * Qbc;
    bb0 -= sc * Qbc * L;
  }
  double brhoh = bA4 * (1.0 - cs2) + bC2 * cs2;
  bcs2 += bC2 * rhoh - bA4 * rhoh;
  double bb2 = bC2;
  double bp = bcs2 * gamma / rhoh;
  brhoh -= bcs2 * cs2 / rhoh;
  // bd = (Bd + alp b0 ud) / W
  double bBd = bbd * iW;
  bb0 += bbd * m.alp * ud * iW;
  bud += bbd * m.alp * b0 * iW;
  double biW = bbd * (Bd + m.alp * b0 * ud);
  // b0 = W Bv / alp, ud = W (v^d - beta^d / alp), u0 = W / alp
  double bW = bb0 * Bv * ia + bud * (v[d] - m.beta[d] * ia) + bu0 * ia;
  double bBv = bb0 * W * ia;
  double bv[3] = {0.0, 0.0, 0.0};
  bv[d] += bud * W;
  // fluxes
  double bU[5], bvl[3] = {0.0, 0.0, 0.0}, bBl[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 5; q++) bU[q] = wb.U[q];
  double bvtd = 0.0, bpt = 0.0;
  bU[4] += wb.F[4] * vtd;
  bvtd += wb.F[4] * U[4];
  bpt += wb.F[4] * asg * v[d];
  bv[d] += wb.F[4] * asg * pt;
  bBv -= wb.F[4] * asg * Bd;
  bBd -= wb.F[4] * asg * Bv;
  bpt += wb.F[1 + d] * asg;
  for (int a = 0; a < 3; a++) {
    const double f = wb.F[1 + a];
    bU[1 + a] += f * vtd;
    bvtd += f * U[1 + a];
    const double bbl = -f * asg * Bd * iW;
    bBd -= f * asg * bl[a] * iW;
    biW -= f * asg * bl[a] * Bd;
    // bl = Bl / W + W Bv vl
    bBl[a] += bbl * iW;
    biW += bbl * Bl[a];
    bW += bbl * Bv * vl[a];
    bBv += bbl * W * vl[a];
    bvl[a] += bbl * W * Bv;
  }
  bU[0] += wb.F[0] * vtd;
  bvtd += wb.F[0] * U[0];
  double bpress = bp + bpt;
  bb2 += 0.5 * bpt;
  // v~ = alp v - beta
  for (int a = 0; a < 3; a++) bv[a] += wb.vt[a] * m.alp;
  bv[d] += bvtd * m.alp;
  // conserved variables
  const double bU4 = bU[4] * sg;
  double bz = bU4;
  bpress -= bU4;
  double brho = -bU4 * W;
  bW -= bU4 * rho;
  double bB2 = bU4;
  bb2 -= 0.5 * bU4;
  for (int a = 0; a < 3; a++) {
    const double bs = bU[1 + a] * sg;
    bz += bs * vl[a];
    bB2 += bs * vl[a];
    bvl[a] += bs * (z + B2);
    bBv -= bs * Bl[a];
    bBl[a] -= bs * Bv;
  }
  brho += bU[0] * sg * W;
  bW += bU[0] * sg * rho;
  // z = rho h W^2, rho h = rho + gfac p
  brhoh += bz * W2;
  bW += bz * rhoh * 2.0 * W;
  brho += brhoh;
  bpress += brhoh * gfac;
  // b^2 = B^2 / W^2 + Bv^2
  bB2 += bb2 * iW2;
  biW += bb2 * B2 * 2.0 * iW;
  bBv += bb2 * 2.0 * Bv;
  // Bv = B . vl, B^2 = B . Bl, vl = g v, Bl = g B
  double bB[3];
  for (int i = 0; i < 3; i++) {
    bB[i] = bBv * vl[i] + bB2 * Bl[i];
    bvl[i] += bBv * B[i];
    bBl[i] += bB2 * B[i];
  }
  double tmp[3];
  lower(m.g, bBl, tmp);
  for (int i = 0; i < 3; i++) bB[i] += tmp[i];
  bB[d] += bBd;
  lower(m.g, bvl, tmp);
  for (int i = 0; i < 3; i++) bv[i] += tmp[i];
  // v = u / W, W = sqrt(1 + u.g.u)
  for (int a = 0; a < 3; a++) biW += bv[a] * u[a];
  bW -= biW * iW2;
  const double buu = bW * 0.5 * iW;
  double gl[3];
  lower(m.g, u, gl);
  for (int a = 0; a < 3; a++) gu[a] = bv[a] * iW + 2.0 * buu * gl[a];
  for (int i = 0; i < 3; i++) gB[i] = bB[i];
  grho = brho;
  gp = bpress;
}

// ----------------------------------------------------------------------------------------------------------
// Reconstruction of one cell from a_{i-2..i+2}: values at its lower (lo) and upper (hi) faces.

template <class T>
__host__ __device__ __forceinline__ T minmod2(T x, T y) {
  if (x * y <= 0.0) return T(0.0);
  return (fabs(x) <= fabs(y)) ? x : y;
}

template <class T>
__host__ __device__ __forceinline__ T ppm_dq(T am, T a0, T ap) {
  // van Leer limited slope of Colella & Woodward (1984)
  if ((ap - a0) * (a0 - am) <= 0.0) return T(0.0);
  const T c = 0.5 * (ap - am);
  const T s = fmin(fabs(c), fmin(2.0 * fabs(a0 - am), 2.0 * fabs(ap - a0)));
  return (c < 0.0) ? -s : s;
}

template <class T>
__host__ __device__ __forceinline__ void ppm_limit(T ai, T& l, T& r) {
  // monotonicity constraints of the parabola (CW84)
  if ((r - ai) * (ai - l) <= 0.0) {
    l = ai;
    r = ai;
  } else {
    const T dlr = r - l;
    const T mid = ai - 0.5 * (l + r);
    const T d6 = dlr * dlr * (1.0 / 6.0);
    if (dlr * mid > d6) l = 3.0 * ai - 2.0 * r;
    else if (-d6 > dlr * mid) r = 3.0 * ai - 2.0 * l;
  }
}

// WENO-Z arithmetic in double is written as explicit fused multiply-adds throughout, so that the compiler cannot
// fuse the same expression differently in different kernels or contexts: a value formed at a pencil's first cell
// equals the value carried into it bit for bit, and a block stepped alone, in a batch or as a tile of a domain
// reconstructs bit for bit alike.  Dual numbers (the adjoint) take the plain expressions.
template <class T>
__host__ __device__ __forceinline__ T fmadd(T a, T b, T c) {
  if constexpr (std::is_same<T, double>::value) return fma(a, b, c);
  else return a * b + c;
}

// The three-point WENO candidates (times 6): c0(a, b, c) = 2 a - 7 b + 11 c and the two that are mirror images of
// each other, cp(a, b, c) = -a + 5 b + 2 c and cm(a, b, c) = 2 a + 5 b - c.  The upper face's cp on (s1, s2, s3) is
// the next cell's lower-face cp on its (s0, s1, s2), and the upper face's cm on (s2, s3, s4) the next cell's
// lower-face cm on its (s1, s2, s3), so a sliding pencil carries them from one cell to the next.
template <class T>
__host__ __device__ __forceinline__ T weno_cand_0(T a, T b, T c) {
  return fmadd(T(11.0), c, fmadd(T(-7.0), b, 2.0 * a));
}
template <class T>
__host__ __device__ __forceinline__ T weno_cand_p(T a, T b, T c) {
  return fmadd(T(2.0), c, fmadd(T(5.0), b, -a));
}
template <class T>
__host__ __device__ __forceinline__ T weno_cand_m(T a, T b, T c) {
  return fmadd(T(2.0), a, fmadd(T(5.0), b, -c));
}

// WENO-Z values at both faces of the middle cell of s[0..4], from tau5 = |beta_0 - beta_2| and e_k = beta_k + eps
// (wenoz_indicators).  The lower face uses the mirrored stencil, whose smoothness indicators are those of the
// upper face in reverse order, so the indicators are shared.  With p = 2 the nonlinear weights alpha_k = d_k (1 + (tau5 / e_k)^2) are proportional to
// d_k (e_k^2 + tau5^2) prod_{j != k} e_j^2, which needs no division before the normalisation (e_k >= eps keeps the
// products above the smallest normal double; out-of-range products take the form with the quotients).
// Candidates: upper face h0 = c0(s0, s1, s2), h1 = cp(s1, s2, s3), h2 = cm(s2, s3, s4); lower face
// l0 = c0(s4, s3, s2), l1 = cm(s1, s2, s3), l2 = cp(s0, s1, s2).
template <class T>
__host__ __device__ __forceinline__ void wenoz_combine(T tau5, T e0, T e1, T e2, T h0, T h1, T h2, T l0, T l1, T l2,
                                                       T& lo, T& hi) {
  const T E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
  T a0 = fmadd(tau5, tau5, E0) * (E1 * E2), a1 = fmadd(tau5, tau5, E1) * (E0 * E2),
    a2 = fmadd(tau5, tau5, E2) * (E0 * E1);
  // upper face: linear weights (1/10, 6/10, 3/10) on the sub-stencils ending at, centred on, starting at i, with the
  // candidates' common factor 1/6 and the weights' 1/10 taken out of numerator and denominator; lower face: the
  // mirrored stencil, whose indicator k is indicator 2-k here
  T w1 = 6.0 * a1;
  T Nh = fmadd(3.0 * a2, h2, fmadd(w1, h1, a0 * h0));
  T Nl = fmadd(3.0 * a0, l2, fmadd(w1, l1, a2 * l0));
  T Dh = fmadd(T(3.0), a2, a0 + w1), Dl = fmadd(T(3.0), a0, a2 + w1);
  // both normalisations from one reciprocal where the product of the two sums is in range (which also shows that
  // the weights are finite and not all zero)
  const T DD = Dh * Dl;
  if (exponent_in_range(val(DD))) {
    const T r = recip(6.0 * DD);
    hi = (Nh * Dl) * r;
    lo = (Nl * Dh) * r;
    return;
  }
  if (!(isfinite(val(a0 + a1 + a2)) && val(a0 + a1 + a2) > 0.0)) {  // products out of range: the quotient form
    const T r0 = tau5 / e0, r1 = tau5 / e1, r2 = tau5 / e2;
    a0 = fmadd(r0, r0, T(1.0));
    a1 = fmadd(r1, r1, T(1.0));
    a2 = fmadd(r2, r2, T(1.0));
    w1 = 6.0 * a1;
    Nh = fmadd(3.0 * a2, h2, fmadd(w1, h1, a0 * h0));
    Nl = fmadd(3.0 * a0, l2, fmadd(w1, l1, a2 * l0));
    Dh = fmadd(T(3.0), a2, a0 + w1);
    Dl = fmadd(T(3.0), a0, a2 + w1);
  }
  hi = Nh / (6.0 * Dh);
  lo = Nl / (6.0 * Dl);
}

template <class T>
__host__ __device__ __forceinline__ void wenoz_from_indicators(const T s[5], T tau5, T e0, T e1, T e2, T& lo, T& hi) {
  wenoz_combine(tau5, e0, e1, e2, weno_cand_0(s[0], s[1], s[2]), weno_cand_p(s[1], s[2], s[3]),
                weno_cand_m(s[2], s[3], s[4]), weno_cand_0(s[4], s[3], s[2]), weno_cand_m(s[1], s[2], s[3]),
                weno_cand_p(s[0], s[1], s[2]), lo, hi);
}

// The Jiang-Shu indicators beta_k = (13/12) ta_k^2 + (1/4) tb_k^2, in double with every operation rounded on its
// own in the order the formula is written (no fused multiply-add).  Where the data are symmetric about the middle
// cell (an extremum), beta_0 and beta_2 agree up to rounding and tau5 = |beta_0 - beta_2| is rounding noise,
// which nevertheless decides the weights when beta_1 is near eps: the indicators are therefore formed exactly as
// the plain formula rounds them, independently of how the compiler would fuse them in a given kernel.
// wenoz_curv is the (13/12) ta^2 part for the three-point sub-stencil centred at b, shared by consecutive cells of
// a pencil.
template <class T>
__host__ __device__ __forceinline__ T wenoz_curv(T a, T b, T c) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, double>::value) {
    const double t = __dadd_rn(fma(-2.0, b, a), c);  // the product 2 b is exact: one rounding, as a - 2 b
    return __dmul_rn(__dmul_rn(13.0 / 12.0, t), t);
  }
#endif
  const T t = a - 2.0 * b + c;
  return (13.0 / 12.0) * t * t;
}

// tau5 and e_k = beta_k + eps from the curvature parts k_k (wenoz_curv) and the stencil values.
template <class T>
__host__ __device__ __forceinline__ void wenoz_indicators(const T s[5], T k0, T k1, T k2, T& tau5, T& e0, T& e1,
                                                          T& e2) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, double>::value) {
    // products by 4 and 1/4 are exact, so a fused multiply-add rounds them as the plain formula does; the
    // products by 3 are rounded on their own
    const double s3x = __dmul_rn(3.0, s[2]);
    const double t0b = __dadd_rn(fma(-4.0, s[1], s[0]), s3x);
    const double t1b = __dsub_rn(s[1], s[3]);
    const double t2b = __dadd_rn(fma(-4.0, s[3], s3x), s[4]);
    const double b0 = fma(0.25, __dmul_rn(t0b, t0b), k0);
    const double b1 = fma(0.25, __dmul_rn(t1b, t1b), k1);
    const double b2 = fma(0.25, __dmul_rn(t2b, t2b), k2);
    tau5 = fabs(__dsub_rn(b0, b2));
    e0 = __dadd_rn(b0, 1e-40);
    e1 = __dadd_rn(b1, 1e-40);
    e2 = __dadd_rn(b2, 1e-40);
    return;
  }
#endif
  const T t0b = s[0] - 4.0 * s[1] + 3.0 * s[2];
  const T t1b = s[1] - s[3];
  const T t2b = 3.0 * s[2] - 4.0 * s[3] + s[4];
  const T b0 = k0 + 0.25 * t0b * t0b, b1 = k1 + 0.25 * t1b * t1b, b2 = k2 + 0.25 * t2b * t2b;
  tau5 = fabs(b0 - b2);
  e0 = b0 + 1e-40;
  e1 = b1 + 1e-40;
  e2 = b2 + 1e-40;
}

template <class T>
__host__ __device__ __forceinline__ void wenoz_both(const T s[5], T& lo, T& hi) {
  T tau5, e0, e1, e2;
  wenoz_indicators(s, wenoz_curv(s[0], s[1], s[2]), wenoz_curv(s[1], s[2], s[3]), wenoz_curv(s[2], s[3], s[4]), tau5,
                   e0, e1, e2);
  wenoz_from_indicators(s, tau5, e0, e1, e2, lo, hi);
}

// MP5, the monotonicity-preserving fifth-order reconstruction of Suresh & Huynh (1997): the fifth-order interface
// value is kept where it lies between the cell value and the monotonicity-preserving bound a_i + minmod(a_i+1 -
// a_i, 4 (a_i - a_i-1)); otherwise it is clipped to the interval the limited curvatures allow (the median of the
// value and the interval's ends, formed as value + minmod(lower - value, upper - value)).  mp5_face gives the
// upper face of the middle cell of (s0 .. s4); the lower face is mp5_face of the reversed stencil.
template <class T>
__host__ __device__ __forceinline__ T minmod4(T w, T x, T y, T z) {
  if (val(w) > 0.0 && val(x) > 0.0 && val(y) > 0.0 && val(z) > 0.0) return fmin(fmin(w, x), fmin(y, z));
  if (val(w) < 0.0 && val(x) < 0.0 && val(y) < 0.0 && val(z) < 0.0) return fmax(fmax(w, x), fmax(y, z));
  return T(0.0);
}

template <class T>
__host__ __device__ __forceinline__ T minmod2v(T x, T y) {  // minmod with the tests on values (dual-safe)
  if (val(x) * val(y) <= 0.0) return T(0.0);
  return (fabs(val(x)) <= fabs(val(y))) ? x : y;
}

template <class T>
__host__ __device__ __forceinline__ T mp5_face(T s0, T s1, T s2, T s3, T s4) {
  const T up = s2 - s1;  // a_i - a_i-1
  const T v5 = (2.0 * s0 - 13.0 * s1 + 47.0 * s2 + 27.0 * s3 - 3.0 * s4) * (1.0 / 60.0);
  const T vb = s2 + minmod2v(s3 - s2, 4.0 * up);
  if (val(v5 - s2) * val(v5 - vb) <= 0.0) return v5;
  const T c_m = s0 - 2.0 * s1 + s2, c_0 = s1 - 2.0 * s2 + s3, c_p = s2 - 2.0 * s3 + s4;
  const T k_up = minmod4(4.0 * c_0 - c_p, 4.0 * c_p - c_0, c_0, c_p);  // limited curvature at the upper face
  const T k_lo = minmod4(4.0 * c_m - c_0, 4.0 * c_0 - c_m, c_m, c_0);  // and at the lower face
  const T v_ul = s2 + 4.0 * up;
  const T v_md = 0.5 * (s2 + s3) - 0.5 * k_up;
  const T v_lc = s2 + 0.5 * up + (4.0 / 3.0) * k_lo;
  const T lower = fmax(fmin(fmin(s2, s3), v_md), fmin(fmin(s2, v_ul), v_lc));
  const T upper = fmin(fmax(fmax(s2, s3), v_md), fmax(fmax(s2, v_ul), v_lc));
  return v5 + minmod2v(lower - v5, upper - v5);
}

template <int SCHEME, class T>
__host__ __device__ __forceinline__ void recon5(const T a[5], T& lo, T& hi) {
  if (SCHEME == 0) {
    const T s = minmod2(a[2] - a[1], a[3] - a[2]);
    lo = a[2] - 0.5 * s;
    hi = a[2] + 0.5 * s;
  } else if (SCHEME == 1) {
    const T dm = ppm_dq(a[0], a[1], a[2]);
    const T d0 = ppm_dq(a[1], a[2], a[3]);
    const T dp = ppm_dq(a[2], a[3], a[4]);
    T l = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) * (1.0 / 6.0);
    T r = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) * (1.0 / 6.0);
    ppm_limit(a[2], l, r);
    lo = l;
    hi = r;
  } else if (SCHEME == 3) {
    hi = mp5_face(a[0], a[1], a[2], a[3], a[4]);
    lo = mp5_face(a[4], a[3], a[2], a[1], a[0]);
  } else {
    wenoz_both(a, lo, hi);
  }
}

// Reverse mode of recon5 for minmod and PPM: weights (glo, ghi) on the cell's (lower, upper) values give the
// gradient g[0..4] with respect to a[0..4], along the branches the forward code takes (ties as there: minmod
// keeps x when |x| = |y|, fmin keeps its first argument).
__host__ __device__ __forceinline__ void ppm_dq_vjp(double am, double a0, double ap, double gd, double& gm,
                                                    double& g0, double& gp) {
  if (gd == 0.0 || (ap - a0) * (a0 - am) <= 0.0) return;
  const double c = 0.5 * (ap - am);
  const double x = 2.0 * fabs(a0 - am), y = 2.0 * fabs(ap - a0);
  const bool inner_y = y < x;  // fmin(x, y) keeps x on ties
  const double inner = inner_y ? y : x;
  if (!(inner < fabs(c))) {  // |c| is the minimum: the slope is c
    gp += 0.5 * gd;
    gm -= 0.5 * gd;
  } else if (inner_y) {  // 2 |ap - a0| with the sign of c, which is the sign of ap - a0 here
    gp += 2.0 * gd;
    g0 -= 2.0 * gd;
  } else {  // 2 |a0 - am|
    g0 += 2.0 * gd;
    gm -= 2.0 * gd;
  }
}

// Reverse of ppm_limit along the branch the forward takes: weights (glo, ghi) on the limited (l, r) give the
// weight on the cell value ai (added) and on the raw interface values (gl, gr).
__host__ __device__ __forceinline__ void ppm_limit_vjp(double ai, double l, double r, double glo, double ghi,
                                                       double& gai, double& gl, double& gr) {
  gl = gr = 0.0;
  if ((r - ai) * (ai - l) <= 0.0) {
    gai += glo + ghi;
    return;
  }
  const double dlr = r - l;
  const double mid = ai - 0.5 * (l + r);
  const double d6 = dlr * dlr * (1.0 / 6.0);
  if (dlr * mid > d6) {  // lo = 3 ai - 2 r
    gai += 3.0 * glo;
    gr = ghi - 2.0 * glo;
  } else if (-d6 > dlr * mid) {  // hi = 3 ai - 2 l
    gai += 3.0 * ghi;
    gl = glo - 2.0 * ghi;
  } else {
    gl = glo;
    gr = ghi;
  }
}

// PPM values on both sides of the interface between positions 2 and 3 of f[0..5] (the upper value of cell 2 and
// the lower value of cell 3, each as recon5<1> gives it), with the primal kept for the reverse sweep: values()
// forms the slopes of cells 1..4 and the three interface values once, then vjp() turns the weights on (L, R)
// into the gradient with respect to f[0..5] without recomputing the primal.
struct PpmPair {
  double f[6], d[4], am, ac, ap, L, R;
  __host__ __device__ __forceinline__ void values(const double in[6]) {
    for (int i = 0; i < 6; i++) f[i] = in[i];
    for (int i = 0; i < 4; i++) d[i] = ppm_dq(f[i], f[i + 1], f[i + 2]);
    am = f[1] + 0.5 * (f[2] - f[1]) - (d[1] - d[0]) * (1.0 / 6.0);
    ac = f[2] + 0.5 * (f[3] - f[2]) - (d[2] - d[1]) * (1.0 / 6.0);
    ap = f[3] + 0.5 * (f[4] - f[3]) - (d[3] - d[2]) * (1.0 / 6.0);
    double l2 = am, r2 = ac, l3 = ac, r3 = ap;
    ppm_limit(f[2], l2, r2);
    ppm_limit(f[3], l3, r3);
    L = r2;
    R = l3;
  }
  __host__ __device__ __forceinline__ void vjp(double gL, double gR, double g[6]) const {
    for (int i = 0; i < 6; i++) g[i] = 0.0;
    double gl2, gr2, gl3, gr3;
    ppm_limit_vjp(f[2], am, ac, 0.0, gL, g[2], gl2, gr2);
    ppm_limit_vjp(f[3], ac, ap, gR, 0.0, g[3], gl3, gr3);
    const double gam = gl2, gac = gr2 + gl3, gap = gr3;
    double gd[4];
    g[1] += 0.5 * gam;
    g[2] += 0.5 * gam + 0.5 * gac;
    g[3] += 0.5 * gac + 0.5 * gap;
    g[4] += 0.5 * gap;
    gd[0] = gam * (1.0 / 6.0);
    gd[1] = (gac - gam) * (1.0 / 6.0);
    gd[2] = (gap - gac) * (1.0 / 6.0);
    gd[3] = -gap * (1.0 / 6.0);
    for (int i = 0; i < 4; i++) ppm_dq_vjp(f[i], f[i + 1], f[i + 2], gd[i], g[i], g[i + 1], g[i + 2]);
  }
};

template <int SCHEME>
__host__ __device__ __forceinline__ void recon5_vjp(const double a[5], double glo, double ghi, double g[5]) {
  for (int i = 0; i < 5; i++) g[i] = 0.0;
  if (SCHEME == 0) {
    const double x = a[2] - a[1], y = a[3] - a[2];
    const double gs = 0.5 * (ghi - glo);
    g[2] += glo + ghi;
    if (x * y > 0.0) {
      if (fabs(x) <= fabs(y)) {
        g[2] += gs;
        g[1] -= gs;
      } else {
        g[3] += gs;
        g[2] -= gs;
      }
    }
  } else {
    const double dm = ppm_dq(a[0], a[1], a[2]);
    const double d0 = ppm_dq(a[1], a[2], a[3]);
    const double dp = ppm_dq(a[2], a[3], a[4]);
    const double l = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) * (1.0 / 6.0);
    const double r = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) * (1.0 / 6.0);
    double gl, gr;
    ppm_limit_vjp(a[2], l, r, glo, ghi, g[2], gl, gr);
    // l = (a1 + a2) / 2 - (d0 - dm) / 6, r = (a2 + a3) / 2 - (dp - d0) / 6
    g[1] += 0.5 * gl;
    g[2] += 0.5 * gl + 0.5 * gr;
    g[3] += 0.5 * gr;
    const double gdm = gl * (1.0 / 6.0), gd0 = (gr - gl) * (1.0 / 6.0), gdp = -gr * (1.0 / 6.0);
    ppm_dq_vjp(a[0], a[1], a[2], gdm, g[0], g[1], g[2]);
    ppm_dq_vjp(a[1], a[2], a[3], gd0, g[1], g[2], g[3]);
    ppm_dq_vjp(a[2], a[3], a[4], gdp, g[2], g[3], g[4]);
  }
}

// Source terms (Eq. grmhdsrc in 3+1 form with the input K_ij, K = -1/2 L_n gamma of Sec. 2.1):
//   tau~: alpha sqrt(g) [T^00 (b^i b^j K_ij - b^i d_i alpha) + T^0i (2 b^j K_ij - d_i alpha) + T^ij K_ij]
//   S~_i: alpha sqrt(g) [-T^00 alpha d_i alpha + T^0_k d_i b^k + 1/2 (T^00 b^j b^k + 2 T^0j b^k + T^jk) d_i g_jk]
// (b = beta) with T^{mu nu} = (rho h + b^2) u u + (p + b^2/2) g^{mu nu} - b b (Eq. tmunu); cg is the centre
// geometry record (K_ij and the 4th-order metric derivatives at index c, field pitch V).
template <class T>
__host__ __device__ __forceinline__ void sources(const Geo& m, const double* __restrict__ cg, long V, long c, T rho, T press,
                                          const T v[3], const T B[3], double gfac, T src[5]) {
  T vl[3], Bl[3];
  lower(m.g, v, vl);
  lower(m.g, B, Bl);
  const T iW = sqrt(1.0 - (v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2]));  // 1 / W
  const T W = 1.0 / iW;
  const T B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const T Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const double ia = 1.0 / m.alp;
  const T b2 = B2 * iW * iW + Bv * Bv;
  const T rhoh = rho + gfac * press;
  const T e = rhoh + b2;
  const T pt = press + 0.5 * b2;
  T u[4], bb[4];
  u[0] = W * ia;
  bb[0] = W * Bv * ia;
  for (int q = 0; q < 3; q++) {
    u[1 + q] = W * (v[q] - m.beta[q] * ia);
    bb[1 + q] = (B[q] + m.alp * bb[0] * u[1 + q]) * iW;
  }
  const double ia2 = ia * ia;
  const T T00 = e * u[0] * u[0] - pt * ia2 - bb[0] * bb[0];
  T T0[3], Tij[6];
  for (int q = 0; q < 3; q++) T0[q] = e * u[0] * u[1 + q] + pt * m.beta[q] * ia2 - bb[0] * bb[1 + q];
  for (int q = 0; q < 3; q++)
    for (int r = q; r < 3; r++)
      Tij[sym(q, r)] = e * u[1 + q] * u[1 + r] + pt * (m.gu[sym(q, r)] - m.beta[q] * m.beta[r] * ia2) -
                       bb[1 + q] * bb[1 + r];
  double K[6], dalp[3];
  for (int q = 0; q < 6; q++) K[q] = cg[(CG_K + q) * V + c];
  for (int q = 0; q < 3; q++) dalp[q] = cg[(CG_DALP + q) * V + c];
  double betal[3];
  lower(m.g, m.beta, betal);
  const double asg = m.alp * m.sqg;
  double Kb[3];
  for (int q = 0; q < 3; q++) Kb[q] = K[sym(q, 0)] * m.beta[0] + K[sym(q, 1)] * m.beta[1] + K[sym(q, 2)] * m.beta[2];
  T st = T00 * (m.beta[0] * Kb[0] + m.beta[1] * Kb[1] + m.beta[2] * Kb[2]);
  for (int q = 0; q < 3; q++) st += -T00 * m.beta[q] * dalp[q] + T0[q] * (2.0 * Kb[q] - dalp[q]);
  st += Tij[0] * K[0] + Tij[3] * K[3] + Tij[5] * K[5] + 2.0 * (Tij[1] * K[1] + Tij[2] * K[2] + Tij[4] * K[4]);
  src[0] = T(0.0);
  src[4] = asg * st;
  T T0l[3];
  for (int q = 0; q < 3; q++)
    T0l[q] = betal[q] * T00 + m.g[sym(q, 0)] * T0[0] + m.g[sym(q, 1)] * T0[1] + m.g[sym(q, 2)] * T0[2];
  T M[6];
  for (int q = 0; q < 3; q++)
    for (int r = q; r < 3; r++)
      M[sym(q, r)] = T00 * m.beta[q] * m.beta[r] + T0[q] * m.beta[r] + T0[r] * m.beta[q] + Tij[sym(q, r)];
  for (int i = 0; i < 3; i++) {
    T s = -T00 * m.alp * dalp[i];
    for (int q = 0; q < 3; q++) s += T0l[q] * cg[(CG_DBETA + i * 3 + q) * V + c];
    const double* dg = cg + (CG_DG + i * 6) * V + c;
    s += 0.5 * (M[0] * dg[0] + M[3] * dg[3 * V] + M[5] * dg[5 * V]) + M[1] * dg[V] + M[2] * dg[2 * V] +
         M[4] * dg[4 * V];
    src[1 + i] = asg * s;
  }
}


// Reverse mode of sources: g = sum_{q=1..4} mu[q] d src_q / d(rho, p, v^i, B^i).  The sources are linear in the
// stress-energy components, so the weights are first carried back to T^00, T^0i, T^ij (metric coefficients
// only), then through T^{mu nu}(rho, p, v, B).
__host__ __device__ __forceinline__ void sources_vjp(const Geo& m, const double* __restrict__ cg, long V, long c,
                                                     double rho, double press, const double v[3],
                                                     const double B[3], double gfac, const double mu[5],
                                                     double g[8]) {
  // ---- primal
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
  double u[4], bb[4];
  u[0] = W * ia;
  bb[0] = W * Bv * ia;
  for (int q = 0; q < 3; q++) {
    u[1 + q] = W * (v[q] - m.beta[q] * ia);
    bb[1 + q] = (B[q] + m.alp * bb[0] * u[1 + q]) * iW;
  }
  const double ia2 = ia * ia;
  // ---- weights of T^00, T^0i, T^ij in sum_q mu_q src_q
  double K[6], dalp[3];
  for (int q = 0; q < 6; q++) K[q] = cg[(CG_K + q) * V + c];
  for (int q = 0; q < 3; q++) dalp[q] = cg[(CG_DALP + q) * V + c];
  double betal[3];
  lower(m.g, m.beta, betal);
  const double asg = m.alp * m.sqg;
  double Kb[3];
  for (int q = 0; q < 3; q++) Kb[q] = K[sym(q, 0)] * m.beta[0] + K[sym(q, 1)] * m.beta[1] + K[sym(q, 2)] * m.beta[2];
  const double w4 = mu[4] * asg;
  double bT00 = w4 * (m.beta[0] * Kb[0] + m.beta[1] * Kb[1] + m.beta[2] * Kb[2]);
  double bT0[3], bTij[6];
  for (int q = 0; q < 3; q++) {
    bT00 -= w4 * m.beta[q] * dalp[q];
    bT0[q] = w4 * (2.0 * Kb[q] - dalp[q]);
  }
  for (int q = 0; q < 6; q++) bTij[q] = ((q == 0 || q == 3 || q == 5) ? 1.0 : 2.0) * w4 * K[q];
  double bT0l[3] = {0.0, 0.0, 0.0}, bM[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 3; i++) {
    const double wi = mu[1 + i] * asg;
    bT00 -= wi * m.alp * dalp[i];
    for (int q = 0; q < 3; q++) bT0l[q] += wi * cg[(CG_DBETA + i * 3 + q) * V + c];
    const double* dg = cg + (CG_DG + i * 6) * V + c;
    bM[0] += 0.5 * wi * dg[0];
    bM[3] += 0.5 * wi * dg[3 * V];
    bM[5] += 0.5 * wi * dg[5 * V];
    bM[1] += wi * dg[V];
    bM[2] += wi * dg[2 * V];
    bM[4] += wi * dg[4 * V];
  }
  for (int q = 0; q < 3; q++) {
    bT00 += bT0l[q] * betal[q];
    for (int r = 0; r < 3; r++) bT0[r] += bT0l[q] * m.g[sym(q, r)];
  }
  for (int q = 0; q < 3; q++)
    for (int r = q; r < 3; r++) {
      const double bm = bM[sym(q, r)];
      bT00 += bm * m.beta[q] * m.beta[r];
      bT0[q] += bm * m.beta[r];
      bT0[r] += bm * m.beta[q];
      bTij[sym(q, r)] += bm;
    }
  // ---- T^{mu nu} = e u u + p_t g^{mu nu} - b b, back to (e, p_t, u, b)
  double be = bT00 * u[0] * u[0], bpt = -bT00 * ia2;
  double bu[4] = {2.0 * e * u[0] * bT00, 0.0, 0.0, 0.0};
  double bbb[4] = {-2.0 * bb[0] * bT00, 0.0, 0.0, 0.0};
  for (int q = 0; q < 3; q++) {
    be += bT0[q] * u[0] * u[1 + q];
    bpt += bT0[q] * m.beta[q] * ia2;
    bu[0] += bT0[q] * e * u[1 + q];
    bu[1 + q] += bT0[q] * e * u[0];
    bbb[0] -= bT0[q] * bb[1 + q];
    bbb[1 + q] -= bT0[q] * bb[0];
  }
  for (int q = 0; q < 3; q++)
    for (int r = q; r < 3; r++) {
      const double bt = bTij[sym(q, r)];
      be += bt * u[1 + q] * u[1 + r];
      bpt += bt * (m.gu[sym(q, r)] - m.beta[q] * m.beta[r] * ia2);
      bu[1 + q] += bt * e * u[1 + r];
      bu[1 + r] += bt * e * u[1 + q];
      bbb[1 + q] -= bt * bb[1 + r];
      bbb[1 + r] -= bt * bb[1 + q];
    }
  // b^i = (B^i + alpha b^0 u^i) / W, b^0 = W Bv / alpha, u^i = W (v^i - beta^i / alpha), u^0 = W / alpha
  double bB[3], bv[3], biW = 0.0, bW = 0.0, bBv = 0.0;
  for (int q = 0; q < 3; q++) {
    bB[q] = bbb[1 + q] * iW;
    bbb[0] += bbb[1 + q] * m.alp * u[1 + q] * iW;
    bu[1 + q] += bbb[1 + q] * m.alp * bb[0] * iW;
    biW += bbb[1 + q] * (B[q] + m.alp * bb[0] * u[1 + q]);
  }
  bW += bbb[0] * Bv * ia + bu[0] * ia;
  bBv += bbb[0] * W * ia;
  for (int q = 0; q < 3; q++) {
    bW += bu[1 + q] * (v[q] - m.beta[q] * ia);
    bv[q] = bu[1 + q] * W;
  }
  // e = rho h + b^2, p_t = p + b^2 / 2, b^2 = B^2 / W^2 + Bv^2, rho h = rho + gfac p
  const double bb2 = be + 0.5 * bpt;
  const double brhoh = be;
  double bB2 = bb2 * iW * iW;
  biW += bb2 * B2 * 2.0 * iW;
  bBv += bb2 * 2.0 * Bv;
  g[0] = brhoh;
  g[1] = bpt + gfac * brhoh;
  // W = (1 - v.g.v)^(-1/2), iW = 1 / W
  bW -= biW * iW * iW;
  const double bvv = bW * 0.5 * W * W * W;
  // Bv = B . g v, B^2 = B . g B
  for (int q = 0; q < 3; q++) {
    bv[q] += 2.0 * bvv * vl[q];
    bB[q] += bBv * vl[q] + 2.0 * bB2 * Bl[q];
  }
  double tmp[3];
  const double bvlB[3] = {bBv * B[0], bBv * B[1], bBv * B[2]};
  lower(m.g, bvlB, tmp);
  for (int q = 0; q < 3; q++) {
    g[2 + q] = bv[q] + tmp[q];
    g[5 + q] = bB[q];
  }
}

// ----------------------------------------------------------------------------------------------------------
// Primitive recovery (Sec. 3.5) for one cell.  Inputs undensitised: D, S_i, tau, centre B^i.

struct C2PParams {
  double gamma, rho_atm, K_atm, gamma_atm, tol, W_max;
  int maxiter, brent_maxiter, use_fallback;
};

struct C2PResult {
  double rho, press, v[3];
  int flag;   // 0 Noble, 1 Palenzuela, 2 atmosphere, -1 failed (atmosphere)
  int iters;
};

__host__ __device__ __forceinline__ void c2p_velocity(const Geo& m, const double S[3], const double B[3], double z,
                                             double B2, double BS, double v[3]) {
  // Eq. (Noble2D v)
  const double izB = 1.0 / (z + B2);
  const double f = BS / z * izB;
  v[0] = (m.gu[0] * S[0] + m.gu[1] * S[1] + m.gu[2] * S[2]) * izB + f * B[0];
  v[1] = (m.gu[1] * S[0] + m.gu[3] * S[1] + m.gu[4] * S[2]) * izB + f * B[1];
  v[2] = (m.gu[2] * S[0] + m.gu[4] * S[1] + m.gu[5] * S[2]) * izB + f * B[2];
}

__host__ __device__ __forceinline__ bool not_physical(double x) { return !(x >= 0.0) || isinf(x); }

// Noble et al. 2D Newton on (z, v^2): residuals Eqs. (Noble2D momentum) and (Noble2D energy) with the ideal-gas
// p(z, v^2) = (G-1)/G (z (1 - v^2) - D sqrt(1 - v^2)); a step that would make z <= 0 halves z instead.
__host__ __device__ inline bool c2p_noble(const Geo& m, double D, const double S[3], double tau, const double B[3], double S2,
                          double B2, double BS, double z, double v2, const C2PParams& P, C2PResult& r) {
  const double gf = (P.gamma - 1.0) / P.gamma;
  const double v2max = 1.0 - 1.0 / (P.W_max * P.W_max);
  const double BS2 = BS * BS;
  bool conv = false;
  int it;
#pragma unroll 1
  for (it = 1; it <= P.maxiter; it++) {
    const double sq = sqrt(1.0 - v2);
    const double Bz = B2 + z;
    const double iz = recip(z);
    const double iz2 = iz * iz;
    const double p = gf * (z * (1.0 - v2) - D * sq);
    const double f0 = v2 * Bz * Bz - BS2 * (B2 + 2.0 * z) * iz2 - S2;
    const double f1 = tau + D - 0.5 * B2 * (1.0 + v2) + 0.5 * BS2 * iz2 - z + p;
    const double J00 = 2.0 * v2 * Bz + 2.0 * BS2 * Bz * iz2 * iz;
    const double J01 = Bz * Bz;
    const double J10 = -BS2 * iz2 * iz - 1.0 + gf * (1.0 - v2);
    const double J11 = -0.5 * B2 + gf * (-z + 0.5 * D / sq);
    const double idet = recip(J00 * J11 - J01 * J10);
    const double dz = (-f0 * J11 + J01 * f1) * idet;
    const double dv2 = (-J00 * f1 + J10 * f0) * idet;
    const bool damped = !(z + dz > 0.0);
    z = damped ? 0.5 * z : z + dz;
    v2 += dv2;
    v2 = fmin(fmax(v2, 0.0), v2max);
    if (!isfinite(z) || !isfinite(v2)) break;
    if (!damped && fabs(dz) <= P.tol * fabs(z) && fabs(dv2) <= P.tol) {
      conv = true;
      break;
    }
  }
  r.iters = (it > P.maxiter) ? P.maxiter : it;
  if (!conv || !(z > 0.0) || !(v2 >= 0.0) || !(v2 < 1.0)) return false;
  const double W = 1.0 / sqrt(1.0 - v2);
  const double rho = D / W;
  c2p_velocity(m, S, B, z, B2, BS, r.v);
  const double eps = (z / (rho * W * W) - 1.0) / P.gamma;  // Eq. (Noble2D epsilon), adiabatic index
  const double press = (P.gamma - 1.0) * rho * eps;
  if (not_physical(rho) || not_physical(eps) || not_physical(press)) return false;
  if (!isfinite(r.v[0]) || !isfinite(r.v[1]) || !isfinite(r.v[2])) return false;
  r.rho = rho;
  r.press = press;
  return true;
}

// Palenzuela et al. 1D function f(x) = x - h^(x) W^(x), x = hW (Eq. Palenzuela Brent and the steps below it).
struct PalFn {
  double q, r, s, t, D, gamma, v2max;
  __host__ __device__ __forceinline__ double operator()(double x, double* W_, double* rho_, double* eps_) const {
    double v2 = (r * x * x + t * t * (2.0 * x + s)) / (x * x * (x + s) * (x + s));
    v2 = fmin(fmax(v2, 0.0), v2max);
    const double W = 1.0 / sqrt(1.0 - v2);
    const double rho = D / W;
    double eps = -1.0 + (x / W) * (1.0 - W * W) + W * (1.0 + q - s + 0.5 * (t * t / (x * x) + s / (W * W)));
    eps = fmax(eps, 0.0);
    const double press = (gamma - 1.0) * rho * eps;
    *W_ = W;
    *rho_ = rho;
    *eps_ = eps;
    return x - (1.0 + eps + press / rho) * W;
  }
};

// Bracketed root by Brent's method (Brent 1973): inverse quadratic / secant steps kept inside the bracket,
// bisection otherwise.  Returns false without a sign change or after maxiter.
__host__ __device__ inline bool brent(const PalFn& f, double lo, double hi, double xtol, int maxiter, double* root) {
  double W_, r_, e_;
  double a = lo, b = hi, fa = f(a, &W_, &r_, &e_), fb = f(b, &W_, &r_, &e_);
  if (!isfinite(fa) || !isfinite(fb) || (fa > 0.0 && fb > 0.0) || (fa < 0.0 && fb < 0.0)) return false;
  double c = a, fc = fa, d = b - a, e = d;
#pragma unroll 1
  for (int it = 0; it < maxiter; it++) {
    if ((fb > 0.0) == (fc > 0.0) && fb != 0.0 && fc != 0.0) {
      c = a;
      fc = fa;
      d = e = b - a;
    }
    if (fabs(fc) < fabs(fb)) {
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    const double tol = 4.440892098500626e-16 * fabs(b) + 0.5 * xtol;
    const double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) {
      *root = b;
      return true;
    }
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      double p, q;
      const double s = fb / fa;
      if (a == c) {
        p = 2.0 * m * s;
        q = 1.0 - s;
      } else {
        const double qq = fa / fc, rr = fb / fc;
        p = s * (2.0 * m * qq * (qq - rr) - (b - a) * (rr - 1.0));
        q = (qq - 1.0) * (rr - 1.0) * (s - 1.0);
      }
      if (p > 0.0) q = -q;
      else p = -p;
      if (2.0 * p < fmin(3.0 * m * q - fabs(tol * q), fabs(e * q))) {
        e = d;
        d = p / q;
      } else {
        d = m;
        e = d;
      }
    } else {
      d = m;
      e = d;
    }
    a = b;
    fa = fb;
    b += (fabs(d) > tol) ? d : (m > 0.0 ? tol : -tol);
    fb = f(b, &W_, &r_, &e_);
    if (!isfinite(fb)) return false;
  }
  return false;
}

__host__ __device__ inline bool c2p_palenzuela(const Geo& m, double D, const double S[3], double tau, const double B[3], double S2,
                               double B2, double BS, const C2PParams& P, C2PResult& r) {
  PalFn f;
  f.q = tau / D;
  f.r = S2 / (D * D);
  f.s = B2 / D;
  f.t = BS / (D * sqrt(D));
  f.D = D;
  f.gamma = P.gamma;
  f.v2max = 1.0 - 1.0 / (P.W_max * P.W_max);
  const double lo = fmax(1.0 + f.q - f.s, 1.0);  // x = hW >= 1
  const double hi = 2.0 + 2.0 * f.q - f.s;
  if (!(hi > lo)) return false;
  double x;
  if (!brent(f, lo, hi, 1e-15 * hi, P.brent_maxiter, &x)) return false;
  double W, rho, eps;
  f(x, &W, &rho, &eps);
  const double press = (P.gamma - 1.0) * rho * eps;
  c2p_velocity(m, S, B, D * x, B2, BS, r.v);  // z = rho W x = D x
  if (not_physical(rho) || not_physical(eps) || not_physical(press)) return false;
  if (!isfinite(r.v[0]) || !isfinite(r.v[1]) || !isfinite(r.v[2])) return false;
  r.rho = rho;
  r.press = press;
  return true;
}

}  // namespace asterx
