// CPU oracle for the GRMHD method-of-lines RK stage of AsterX (arXiv:2406.11669).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 reference that the CUDA path is checked
// against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
// shares no code, header or table with the CUDA library (paper_2406_11669_gb300/csrc) and the product path
// never calls it.
//
// Style: every step is written out literally in the order the paper states it, per cell / per face /
// per edge, with temporaries in full-size arrays and no fusion, hoisting or blocking.  The physics and the
// stage's grid steps are templated on the scalar type R: R = double for results, a flop-counting type for the
// algorithmic counts, and a one-direction dual number for Jacobian-vector products of the stage operator.
// Citations name the paper's sections and equation labels.
//
// Readings of the paper that this file takes (all listed in the repository's design notes):
//  * Densitised evolution (Eq. fluxconseqs): U = sqrt(gamma) (D, S_j, tau); fluxes are alpha sqrt(gamma) F^i.
//  * E = -v~ x B~ (induction, Eq. inductioneq) and dA/dt = -E - grad G_A (Eq. Ainductioneqs); the
//    second line of Eq. recastedAvec carries the opposite sign of the v x B term and is not followed.
//  * Source terms in 3+1 form with the input K_ij; equal to Eq. grmhdsrc for a static metric.
//  * Ideal-gas eps recovery of Eq. Noble2D epsilon uses the adiabatic index Gamma (printed "1/gamma").
//  * Palenzuela eps-hat uses t^2/x^2 (the derivation from Eq. Noble2D energy; printed "t^2/x").
//  * Palenzuela lower bracket raised to max(1 + q - s, 1) because x = hW >= 1.
//  * The atmosphere criterion is the one of Sec. 3.6 only: D~ < sqrt(gamma) rho_atm, tested before recovery.
//  * Wave speeds: extreme roots of the magnetosonic quartic, multiplied through by c_s^2, found by Newton
//    from the light-cone speeds; G = gamma^dd - (lambda + beta^d)^2 / alpha^2.
//  * Reconstructed variables: rho, p, W v^i and the transverse cell-centre B (undensitised).
//  * 4th-order Lagrange interpolation of the vertex metric; near the edge of the padded array the 4-point
//    stencil is shifted inward (still 4th order).
//  * UCT face->edge reconstruction is PPM (Sec. 3.4 (ii)); a_+-(edge) = max over the two adjacent faces.
//  * Copy (Neumann) BCs copy the nearest owned value, except the edge potential A_i, which is extrapolated
//    linearly along the boundary normal.

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace asterx_oracle {

// ------------------------------------------------------------------------------------------------------
// Flop-counting scalar.  + - * / sqrt each count one flop; divisions and square roots are also counted apart.
// A value is either data (derived from the evolved state) or a constant (a literal, a parameter, or derived from
// the frozen metric alone): operations whose operands are all constants are not counted, because a frozen
// metric's arithmetic is done once, not every stage.  Fc(x) makes a constant; fc_data(x) a data value.

struct Flops {
  unsigned long long add = 0, mul = 0, div = 0, sqrt = 0;
};
static Flops g_flops;
static unsigned long long flops_total(const Flops& f) { return f.add + f.mul + f.div + f.sqrt; }
// Flops spent inside the wave-speed Newton loops (flop-counting scalar only), and the phase boundaries of the
// right-hand side (set by the flop-count entry; null otherwise).
static unsigned long long g_speed_loop_flops = 0;
static Flops* g_rhs_marks = nullptr;
// Flops of steps that this literal oracle repeats where an implementation does them once (flop-counting scalar
// only): u = W v per cell (formed for each of the three directions), the per-cell reconstruction (formed for
// both faces of every cell), the PPM interfaces of the edge fields (formed for both edges that share a face
// value); and the face solves themselves.
static unsigned long long g_cellvar_flops = 0, g_recon_flops = 0, g_facesolve_flops = 0, g_edge_ppm_flops = 0;

struct Fc {
  double v;
  bool k;  // constant
  Fc() : v(0.0), k(true) {}
  Fc(double x) : v(x), k(true) {}
  Fc(double x, bool constant) : v(x), k(constant) {}
};
inline Fc fc_data(double x) { return Fc(x, false); }
inline Fc operator+(Fc a, Fc b) { if (!(a.k && b.k)) g_flops.add++; return Fc(a.v + b.v, a.k && b.k); }
inline Fc operator-(Fc a, Fc b) { if (!(a.k && b.k)) g_flops.add++; return Fc(a.v - b.v, a.k && b.k); }
inline Fc operator*(Fc a, Fc b) { if (!(a.k && b.k)) g_flops.mul++; return Fc(a.v * b.v, a.k && b.k); }
inline Fc operator/(Fc a, Fc b) { if (!(a.k && b.k)) g_flops.div++; return Fc(a.v / b.v, a.k && b.k); }
inline Fc operator-(Fc a) { return Fc(-a.v, a.k); }
inline Fc& operator+=(Fc& a, Fc b) { a = a + b; return a; }
inline Fc& operator-=(Fc& a, Fc b) { a = a - b; return a; }
inline Fc& operator*=(Fc& a, Fc b) { a = a * b; return a; }
inline bool operator<(Fc a, Fc b) { return a.v < b.v; }
inline bool operator>(Fc a, Fc b) { return a.v > b.v; }
inline bool operator<=(Fc a, Fc b) { return a.v <= b.v; }
inline bool operator>=(Fc a, Fc b) { return a.v >= b.v; }
inline bool operator==(Fc a, Fc b) { return a.v == b.v; }
inline bool operator!=(Fc a, Fc b) { return a.v != b.v; }
inline Fc sqrt(Fc a) { if (!a.k) g_flops.sqrt++; return Fc(std::sqrt(a.v), a.k); }
inline Fc fabs(Fc a) { return Fc(std::fabs(a.v), a.k); }
inline double val(Fc a) { return a.v; }
inline double val(double a) { return a; }
inline bool finite(double a) { return std::isfinite(a); }
inline bool finite(Fc a) { return std::isfinite(a.v); }

// Adds the flops counted while it lives to *acc (flop-counting scalar only; a no-op for other scalars).
template <class R> struct FlopScope {
  unsigned long long* acc;
  unsigned long long t0;
  explicit FlopScope(unsigned long long* a) : acc(a), t0(std::is_same<R, Fc>::value ? flops_total(g_flops) : 0) {}
  ~FlopScope() {
    if (std::is_same<R, Fc>::value) *acc += flops_total(g_flops) - t0;
  }
};

// Forward-mode dual number with one direction: value v and directional derivative d.  Comparisons act on the
// value, so a branch contributes the derivative of the branch taken.
struct Dual1 {
  double v, d;
  Dual1() : v(0.0), d(0.0) {}
  Dual1(double x) : v(x), d(0.0) {}
  Dual1(double x, double dx) : v(x), d(dx) {}
};
inline Dual1 operator+(Dual1 a, Dual1 b) { return Dual1(a.v + b.v, a.d + b.d); }
inline Dual1 operator-(Dual1 a, Dual1 b) { return Dual1(a.v - b.v, a.d - b.d); }
inline Dual1 operator*(Dual1 a, Dual1 b) { return Dual1(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual1 operator/(Dual1 a, Dual1 b) {
  const double q = a.v / b.v;
  return Dual1(q, (a.d - q * b.d) / b.v);
}
inline Dual1 operator-(Dual1 a) { return Dual1(-a.v, -a.d); }
inline Dual1& operator+=(Dual1& a, Dual1 b) { a = a + b; return a; }
inline Dual1& operator-=(Dual1& a, Dual1 b) { a = a - b; return a; }
inline Dual1& operator*=(Dual1& a, Dual1 b) { a = a * b; return a; }
inline bool operator<(Dual1 a, Dual1 b) { return a.v < b.v; }
inline bool operator>(Dual1 a, Dual1 b) { return a.v > b.v; }
inline bool operator<=(Dual1 a, Dual1 b) { return a.v <= b.v; }
inline bool operator>=(Dual1 a, Dual1 b) { return a.v >= b.v; }
inline bool operator==(Dual1 a, Dual1 b) { return a.v == b.v; }
inline bool operator!=(Dual1 a, Dual1 b) { return a.v != b.v; }
inline Dual1 sqrt(Dual1 a) {
  const double r = std::sqrt(a.v);
  return Dual1(r, a.d / (2.0 * r));
}
inline Dual1 fabs(Dual1 a) { return (a.v < 0.0) ? -a : a; }
inline double val(Dual1 a) { return a.v; }
inline bool finite(Dual1 a) { return std::isfinite(a.v); }
using std::fabs;
using std::sqrt;

// The per-cell, per-face and per-edge loops of the grid steps run on OpenMP threads over (k, j) pencils (every
// iteration writes its own entries; counters are reduced).  The flop-counting scalar keeps one global tally, so
// loops instantiated with it stay on one thread.  oracle_set_threads() sets the thread count.
template <class R> constexpr bool parallel_ok() { return !std::is_same<R, Fc>::value; }
#define ORACLE_PRAGMA(x) _Pragma(#x)
#define ORACLE_PAR(R) ORACLE_PRAGMA(omp parallel for collapse(2) schedule(static) if (parallel_ok<R>()))
#define ORACLE_PAR_REDUCE(R, red) \
  ORACLE_PRAGMA(omp parallel for collapse(2) schedule(static) if (parallel_ok<R>()) red)

template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }
template <class R> inline R rmin(R a, R b) { return (b < a) ? b : a; }

// ------------------------------------------------------------------------------------------------------
// ABI structs (mirrored by ctypes in oracle/__init__.py)

struct OParams {
  double gamma;       // ideal-gas adiabatic index (Sec. 3.7)
  double rho_atm;     // atmosphere density floor (Sec. 3.6)
  double K_atm;       // atmosphere polytrope constant
  double gamma_atm;   // atmosphere polytrope exponent
  double c2p_tol;     // Noble Newton tolerance
  int c2p_maxiter;
  int brent_maxiter;
  double W_max;       // Lorentz-factor cap used on failure paths of the recovery
  int recon;          // 0 minmod, 1 PPM, 2 WENO-Z, 3 MP5
  int gauge;          // 0 generalised Lorenz, 1 algebraic
  double xi_lorenz;   // Lorenz damping; 0 => 1.5/dt
  int use_fallback;   // Palenzuela fallback on/off
  int flux;           // 0 HLLE (Eq. HLLEfluxes), 1 Lax-Friedrichs (Eq. LxFfluxes)
  int efield;         // 0 upwind constrained transport (Eq. eq3.20), 1 flux constrained transport
};

struct OBlock {
  int n[3];
  int g;
  double x0[3];
  double dx[3];
  int bc[3];  // 0 periodic, 1 copy
};

struct OStats {
  unsigned long long n_noble, n_fallback, n_atm, n_failed, iters;
};

enum { RECON_MINMOD = 0, RECON_PPM = 1, RECON_WENOZ = 2, RECON_MP5 = 3 };
enum { FLUX_HLLE = 0, FLUX_LXF = 1 };
enum { EFIELD_UCT = 0, EFIELD_FCT = 1 };
enum { BC_PERIODIC = 0, BC_COPY = 1 };
enum { GAUGE_LORENZ = 0, GAUGE_ALGEBRAIC = 1 };

// ------------------------------------------------------------------------------------------------------
// Grid indexing: every field spans the vertex-index box [0, N]^3, N = n + 2g, x fastest.

struct Grid {
  int n[3], g, N[3];
  long s[3];
  double dx[3];
  int bc[3];
  explicit Grid(const OBlock& b) {
    g = b.g;
    for (int d = 0; d < 3; d++) {
      n[d] = b.n[d];
      N[d] = b.n[d] + 2 * b.g;
      dx[d] = b.dx[d];
      bc[d] = b.bc[d];
    }
    s[0] = 1;
    s[1] = N[0] + 1;
    s[2] = (long)(N[0] + 1) * (N[1] + 1);
  }
  long size() const { return (long)(N[0] + 1) * (N[1] + 1) * (N[2] + 1); }
  long at(int i, int j, int k) const { return i + s[1] * j + s[2] * k; }
  long at(const int p[3]) const { return at(p[0], p[1], p[2]); }
};

typedef std::vector<double> Field;

// ------------------------------------------------------------------------------------------------------
// 3+1 metric at a point (Sec. 2.1, Eq. lineelement): lapse, shift, 3-metric, its inverse and determinant.

template <class R> struct Metric3 {
  R alp, beta[3], g[3][3], K[3][3];
  R gu[3][3], sqrtg;
};

template <class R> void metric_complete(Metric3<R>& m) {
  // determinant and inverse by cofactors
  R c00 = m.g[1][1] * m.g[2][2] - m.g[1][2] * m.g[2][1];
  R c01 = m.g[1][2] * m.g[2][0] - m.g[1][0] * m.g[2][2];
  R c02 = m.g[1][0] * m.g[2][1] - m.g[1][1] * m.g[2][0];
  R det = m.g[0][0] * c00 + m.g[0][1] * c01 + m.g[0][2] * c02;
  R c11 = m.g[0][0] * m.g[2][2] - m.g[0][2] * m.g[2][0];
  R c12 = m.g[0][1] * m.g[2][0] - m.g[0][0] * m.g[2][1];
  R c22 = m.g[0][0] * m.g[1][1] - m.g[0][1] * m.g[1][0];
  m.gu[0][0] = c00 / det;
  m.gu[0][1] = c01 / det;
  m.gu[0][2] = c02 / det;
  m.gu[1][0] = m.gu[0][1];
  m.gu[1][1] = c11 / det;
  m.gu[1][2] = c12 / det;
  m.gu[2][0] = m.gu[0][2];
  m.gu[2][1] = m.gu[1][2];
  m.gu[2][2] = c22 / det;
  m.sqrtg = sqrt(det);
}

// The 16 vertex fields, in ABI order: alp, beta^x,y,z, g_xx,xy,xz,yy,yz,zz, K_xx,xy,xz,yy,yz,zz.
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

struct VertexMetric {
  const double* f[16];
};

// 4-point Lagrange weights for the midpoint between nodes p and p+1 of the node set s..s+3 (Sec. 3.2: the
// vertex metric is interpolated to centres and faces at 4th order).  Near the end of the padded array the
// stencil start s is shifted so that all four nodes exist.
static void lagrange_mid(int p, int Nv, int* start, double w[4]) {
  int s = p - 1;
  if (s < 0) s = 0;
  if (s > Nv - 3) s = Nv - 3;
  const double t = (p - s) + 0.5;  // target position in node units
  for (int a = 0; a < 4; a++) {
    double num = 1.0, den = 1.0;
    for (int b = 0; b < 4; b++) {
      if (b == a) continue;
      num *= (t - b);
      den *= (double)(a - b);
    }
    w[a] = num / den;
  }
  *start = s;
}

// Staggered 4th-order first derivative at the midpoint p+1/2 from nodes p-1..p+2:
// (f(p-1) - 27 f(p) + 27 f(p+1) - f(p+2)) / (24 h).
static const double DER4[4] = {1.0 / 24.0, -27.0 / 24.0, 27.0 / 24.0, -1.0 / 24.0};

// Interpolate the vertex metric to a point that is at vertex index along axes where half[d] == 0 and at the
// midpoint p+1/2 along axes where half[d] == 1.  If dflag >= 0, the axis dflag (which must be a half axis)
// takes the staggered derivative stencil instead, and the result is d/dx^dflag of the field.  The sums run
// x innermost, then y, then z, each term a fused multiply-add (one rounding).
static double vertex_interp(const Grid& G, const double* f, const int p[3], const int half[3], int dflag) {
  int st[3];
  double w[3][4];
  int cnt[3];
  for (int d = 0; d < 3; d++) {
    if (!half[d]) {
      st[d] = p[d];
      cnt[d] = 1;
      w[d][0] = 1.0;
    } else if (d == dflag) {
      st[d] = p[d] - 1;
      cnt[d] = 4;
      for (int a = 0; a < 4; a++) w[d][a] = DER4[a] / G.dx[d];
    } else {
      lagrange_mid(p[d], G.N[d], &st[d], w[d]);
      cnt[d] = 4;
    }
  }
  double acc = 0.0;
  for (int c = 0; c < cnt[2]; c++) {
    double accy = 0.0;
    for (int b = 0; b < cnt[1]; b++) {
      double accx = 0.0;
      for (int a = 0; a < cnt[0]; a++) accx = std::fma(w[0][a], f[G.at(st[0] + a, st[1] + b, st[2] + c)], accx);
      accy = std::fma(w[1][b], accx, accy);
    }
    acc = std::fma(w[2][c], accy, acc);
  }
  return acc;
}

static Metric3<double> metric_at(const Grid& G, const VertexMetric& vm, const int p[3], const int half[3]) {
  Metric3<double> m;
  m.alp = vertex_interp(G, vm.f[0], p, half, -1);
  for (int a = 0; a < 3; a++) m.beta[a] = vertex_interp(G, vm.f[1 + a], p, half, -1);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      m.g[a][b] = vertex_interp(G, vm.f[4 + SYM[a][b]], p, half, -1);
      m.K[a][b] = vertex_interp(G, vm.f[10 + SYM[a][b]], p, half, -1);
    }
  metric_complete(m);
  return m;
}

static Metric3<double> metric_at_centre(const Grid& G, const VertexMetric& vm, int i, int j, int k) {
  const int p[3] = {i, j, k};
  const int half[3] = {1, 1, 1};
  return metric_at(G, vm, p, half);
}

static Metric3<double> metric_at_face(const Grid& G, const VertexMetric& vm, int d, int i, int j, int k) {
  const int p[3] = {i, j, k};
  int half[3] = {1, 1, 1};
  half[d] = 0;
  return metric_at(G, vm, p, half);
}

static Metric3<double> metric_at_vertex(const Grid& G, const VertexMetric& vm, int i, int j, int k) {
  const int p[3] = {i, j, k};
  const int half[3] = {0, 0, 0};
  return metric_at(G, vm, p, half);
}

// The frozen metric (and, below, its derivatives) as scalars R: they carry no derivative.
template <class R> Metric3<R> lift(const Metric3<double>& m) {
  Metric3<R> r;
  r.alp = R(m.alp);
  r.sqrtg = R(m.sqrtg);
  for (int a = 0; a < 3; a++) {
    r.beta[a] = R(m.beta[a]);
    for (int b = 0; b < 3; b++) {
      r.g[a][b] = R(m.g[a][b]);
      r.K[a][b] = R(m.K[a][b]);
      r.gu[a][b] = R(m.gu[a][b]);
    }
  }
  return r;
}

// ------------------------------------------------------------------------------------------------------
// Primitive -> conserved map and fluxes (Sec. 2.2, Eqs. eulerianB, grmhdeqs, cons).

template <class R> struct Prim {
  R rho, press, eps, vel[3], B[3];  // v^i Eulerian, B^i undensitised Eulerian
};

template <class R> struct Cons {
  R D, S[3], tau;  // densitised by sqrt(gamma)
};

// Comoving-frame quantities of a primitive state (Eq. eulerianB and the covariant b_i below Eq. Noble2D z).
template <class R> struct Comoving {
  R W, vlow[3], h, Blow[3], B2, Bv, b0, bup[3], blow[3], b2, u0, uup[3];
};

template <class R> Comoving<R> comoving(const Metric3<R>& m, const Prim<R>& P) {
  Comoving<R> c;
  R v2 = R(0.0);
  for (int a = 0; a < 3; a++) {
    c.vlow[a] = m.g[a][0] * P.vel[0] + m.g[a][1] * P.vel[1] + m.g[a][2] * P.vel[2];
  }
  for (int a = 0; a < 3; a++) v2 += P.vel[a] * c.vlow[a];
  c.W = R(1.0) / sqrt(R(1.0) - v2);
  c.h = R(1.0) + P.eps + P.press / P.rho;
  c.B2 = R(0.0);
  c.Bv = R(0.0);
  for (int a = 0; a < 3; a++) {
    c.Blow[a] = m.g[a][0] * P.B[0] + m.g[a][1] * P.B[1] + m.g[a][2] * P.B[2];
  }
  for (int a = 0; a < 3; a++) {
    c.B2 += P.B[a] * c.Blow[a];
    c.Bv += P.B[a] * c.vlow[a];
  }
  c.u0 = c.W / m.alp;
  for (int a = 0; a < 3; a++) c.uup[a] = c.W * (P.vel[a] - m.beta[a] / m.alp);
  c.b0 = c.W * c.Bv / m.alp;
  for (int a = 0; a < 3; a++) c.bup[a] = (P.B[a] + m.alp * c.b0 * c.uup[a]) / c.W;
  for (int a = 0; a < 3; a++) c.blow[a] = c.Blow[a] / c.W + m.alp * c.b0 * c.vlow[a];
  c.b2 = (c.B2 + m.alp * m.alp * c.b0 * c.b0) / (c.W * c.W);
  return c;
}

template <class R> Cons<R> prim2con(const Metric3<R>& m, const Prim<R>& P, const Comoving<R>& c) {
  Cons<R> U;
  const R rhohb = P.rho * c.h + c.b2;
  U.D = m.sqrtg * (P.rho * c.W);
  for (int a = 0; a < 3; a++)
    U.S[a] = m.sqrtg * (rhohb * c.W * c.W * c.vlow[a] - m.alp * c.b0 * c.blow[a]);
  U.tau = m.sqrtg * (rhohb * c.W * c.W - (P.press + R(0.5) * c.b2) - m.alp * m.alp * c.b0 * c.b0 - P.rho * c.W);
  return U;
}

// alpha sqrt(gamma) F^d for the five hydro variables (Eq. grmhdeqs), with v~^d = alpha v^d - beta^d.
template <class R> void flux(const Metric3<R>& m, const Prim<R>& P, const Comoving<R>& c, const Cons<R>& U, int d,
                             R F[5]) {
  const R vt = m.alp * P.vel[d] - m.beta[d];
  const R asg = m.alp * m.sqrtg;
  const R ptot = P.press + R(0.5) * c.b2;
  F[0] = U.D * vt;
  for (int a = 0; a < 3; a++) {
    F[1 + a] = U.S[a] * vt - asg * c.blow[a] * P.B[d] / c.W;
    if (a == d) F[1 + a] = F[1 + a] + asg * ptot;
  }
  F[4] = U.tau * vt + asg * ptot * P.vel[d] - asg * m.alp * c.b0 * P.B[d] / c.W;
}

// ------------------------------------------------------------------------------------------------------
// Fast magnetosonic speeds along d (Sec. 3.3: extreme roots of the quartic, refs. therein).
// With phi_mu = (-lambda, delta^d_mu): a = u.phi, Bc = b.phi, G = g^{mu nu} phi phi = gamma^dd - (lambda +
// beta^d)^2/alpha^2.  The quartic  rho h (1/cs2 - 1) a^4 - (rho h + b^2/cs2) a^2 G + Bc^2 G = 0  is used
// multiplied by cs2 (same roots, finite for cs2 = 0).  Newton from each light-cone speed converges
// monotonically to the outermost root on that side.

template <class R> struct Quartic {
  R e, cs2, b2, u0, ud, b0, bd, alp, betad, gdd;
  R eval(R lam, R* dq) const {
    const R a = ud - lam * u0;
    const R Bc = bd - lam * b0;
    const R lb = lam + betad;
    const R G = gdd - lb * lb / (alp * alp);
    const R dG = R(-2.0) * lb / (alp * alp);
    const R c4 = e * (R(1.0) - cs2);
    const R c2 = e * cs2 + b2;
    const R a2 = a * a;
    const R q = c4 * a2 * a2 - c2 * a2 * G + cs2 * Bc * Bc * G;
    *dq = R(4.0) * c4 * a2 * a * (-u0) - c2 * (R(2.0) * a * (-u0) * G + a2 * dG) +
          cs2 * (R(2.0) * Bc * (-b0) * G + Bc * Bc * dG);
    return q;
  }
};

template <class R> void wave_speeds(const Metric3<R>& m, const Prim<R>& P, const Comoving<R>& c, double gamma, int d,
                                    R* lam_minus, R* lam_plus, int* iters) {
  Quartic<R> Q;
  Q.e = P.rho * c.h;
  Q.cs2 = R(gamma * (gamma - 1.0)) * P.eps / c.h;  // ideal gas: cs^2 = Gamma (Gamma-1) eps / h
  Q.b2 = c.b2;
  Q.u0 = c.u0;
  Q.ud = c.uup[d];
  Q.b0 = c.b0;
  Q.bd = c.bup[d];
  Q.alp = m.alp;
  Q.betad = m.beta[d];
  Q.gdd = m.gu[d][d];
  const R width = m.alp * sqrt(m.gu[d][d]);
  int it_total = 0;
  const Flops loop0 = g_flops;
  for (int side = 0; side < 2; side++) {
    const R sgn = (side == 0) ? R(1.0) : R(-1.0);
    R lam = -m.beta[d] + sgn * width;  // light-cone speed on this side
    for (int it = 0; it < 60; it++) {
      R dq;
      R q = Q.eval(lam, &dq);
      it_total++;
      if (dq == R(0.0)) break;
      const R step = q / dq;
      lam = lam - step;
      if (fabs(step) <= R(1e-13) * (fabs(lam) + width)) break;
    }
    if (side == 0) *lam_plus = lam;
    else *lam_minus = lam;
  }
  if (std::is_same<R, Fc>::value) g_speed_loop_flops += flops_total(g_flops) - flops_total(loop0);
  if (iters) *iters = it_total;
}

// ------------------------------------------------------------------------------------------------------
// Reconstruction (Sec. 3.3, ReconX): per cell, the values at its lower (aL) and upper (aR) faces from the
// five cell averages a[0..4] = a_{i-2..i+2}.

template <class R> R minmod(R x, R y) {
  if (x * y <= R(0.0)) return R(0.0);
  return (fabs(x) <= fabs(y)) ? x : y;
}

template <class R> void recon_minmod(const R a[5], R* aL, R* aR) {
  const R slope = minmod(a[2] - a[1], a[3] - a[2]);
  *aL = a[2] - R(0.5) * slope;
  *aR = a[2] + R(0.5) * slope;
}

// Colella & Woodward (1984) PPM without flattening or steepening: van-Leer limited slopes, the 4th-order
// interface value, then the monotonicity constraints on the parabola of the cell.
template <class R> R ppm_slope(R am, R a0, R ap) {
  if ((ap - a0) * (a0 - am) <= R(0.0)) return R(0.0);
  const R c = R(0.5) * (ap - am);
  R s = rmin(fabs(c), rmin(R(2.0) * fabs(a0 - am), R(2.0) * fabs(ap - a0)));
  return (c < R(0.0)) ? -s : s;
}

template <class R> void recon_ppm(const R a[5], R* aL, R* aR) {
  const R dm = ppm_slope(a[0], a[1], a[2]);
  const R d0 = ppm_slope(a[1], a[2], a[3]);
  const R dp = ppm_slope(a[2], a[3], a[4]);
  R l = a[1] + R(0.5) * (a[2] - a[1]) - (d0 - dm) / R(6.0);  // a_{i-1/2}
  R r = a[2] + R(0.5) * (a[3] - a[2]) - (dp - d0) / R(6.0);  // a_{i+1/2}
  const R ai = a[2];
  if ((r - ai) * (ai - l) <= R(0.0)) {
    l = ai;
    r = ai;
  } else {
    const R dlr = r - l;
    const R mid = ai - R(0.5) * (l + r);
    if (dlr * mid > dlr * dlr / R(6.0)) {
      l = R(3.0) * ai - R(2.0) * r;
    } else if (-(dlr * dlr) / R(6.0) > dlr * mid) {
      r = R(3.0) * ai - R(2.0) * l;
    }
  }
  *aL = l;
  *aR = r;
}

// WENO-Z (Borges et al. 2008), fifth order, epsilon = 1e-40, power p = 2.  Value at the upper face of the
// middle cell of s[0..4]; the lower face is the same formula on the mirrored stencil.
template <class R> R wenoz_upper(R s0, R s1, R s2, R s3, R s4) {
  const R q0 = (R(2.0) * s0 - R(7.0) * s1 + R(11.0) * s2) / R(6.0);
  const R q1 = (-s1 + R(5.0) * s2 + R(2.0) * s3) / R(6.0);
  const R q2 = (R(2.0) * s2 + R(5.0) * s3 - s4) / R(6.0);
  const R t0a = s0 - R(2.0) * s1 + s2, t0b = s0 - R(4.0) * s1 + R(3.0) * s2;
  const R t1a = s1 - R(2.0) * s2 + s3, t1b = s1 - s3;
  const R t2a = s2 - R(2.0) * s3 + s4, t2b = R(3.0) * s2 - R(4.0) * s3 + s4;
  const R b0 = R(13.0 / 12.0) * t0a * t0a + R(0.25) * t0b * t0b;
  const R b1 = R(13.0 / 12.0) * t1a * t1a + R(0.25) * t1b * t1b;
  const R b2 = R(13.0 / 12.0) * t2a * t2a + R(0.25) * t2b * t2b;
  const R tau5 = fabs(b0 - b2);
  const R eps = R(1e-40);
  const R r0 = tau5 / (b0 + eps), r1 = tau5 / (b1 + eps), r2 = tau5 / (b2 + eps);
  const R w0 = R(0.1) * (R(1.0) + r0 * r0);
  const R w1 = R(0.6) * (R(1.0) + r1 * r1);
  const R w2 = R(0.3) * (R(1.0) + r2 * r2);
  return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

template <class R> void recon_wenoz(const R a[5], R* aL, R* aR) {
  *aR = wenoz_upper(a[0], a[1], a[2], a[3], a[4]);
  *aL = wenoz_upper(a[4], a[3], a[2], a[1], a[0]);
}

// MP5 (Suresh & Huynh 1997, the monotonicity-preserving fifth-order scheme; Sec. 3.3 lists it among the
// reconstruction methods): the fifth-order interface value from the five averages, kept where it lies between
// the cell value and the monotonicity-preserving bound a_i + minmod(a_{i+1} - a_i, alpha (a_i - a_{i-1}))
// (alpha = 4); elsewhere moved to the nearer end of the interval the curvature-based bounds allow (the
// median of the value and the interval's ends).  Value at the upper face of the middle cell of s[0..4]; the
// lower face is the same formula on the mirrored stencil.
template <class R> R minmod4(R w, R x, R y, R z) {
  const R zero = R(0.0);
  if (w > zero && x > zero && y > zero && z > zero) return rmin(rmin(w, x), rmin(y, z));
  if (w < zero && x < zero && y < zero && z < zero) return rmax(rmax(w, x), rmax(y, z));
  return zero;
}

template <class R> R median3(R x, R lo, R hi) {  // the median of x, lo, hi for lo <= hi: x clipped to [lo, hi]
  return x + minmod(lo - x, hi - x);
}

template <class R> R mp5_upper(R s0, R s1, R s2, R s3, R s4) {
  const R alpha = R(4.0);
  const R v_or = (R(2.0) * s0 - R(13.0) * s1 + R(47.0) * s2 + R(27.0) * s3 - R(3.0) * s4) / R(60.0);
  const R v_mp = s2 + minmod(s3 - s2, alpha * (s2 - s1));
  if ((v_or - s2) * (v_or - v_mp) <= R(0.0)) return v_or;
  // second differences at cells i-1, i, i+1 and the limited curvatures at the faces i-1/2, i+1/2
  const R dm = s0 - R(2.0) * s1 + s2;
  const R d0 = s1 - R(2.0) * s2 + s3;
  const R dp = s2 - R(2.0) * s3 + s4;
  const R dM4p = minmod4(R(4.0) * d0 - dp, R(4.0) * dp - d0, d0, dp);
  const R dM4m = minmod4(R(4.0) * dm - d0, R(4.0) * d0 - dm, dm, d0);
  const R v_ul = s2 + alpha * (s2 - s1);
  const R v_av = R(0.5) * (s2 + s3);
  const R v_md = v_av - R(0.5) * dM4p;
  const R v_lc = s2 + R(0.5) * (s2 - s1) + R(4.0 / 3.0) * dM4m;
  const R v_min = rmax(rmin(rmin(s2, s3), v_md), rmin(rmin(s2, v_ul), v_lc));
  const R v_max = rmin(rmax(rmax(s2, s3), v_md), rmax(rmax(s2, v_ul), v_lc));
  return median3(v_or, v_min, v_max);
}

template <class R> void recon_mp5(const R a[5], R* aL, R* aR) {
  *aR = mp5_upper(a[0], a[1], a[2], a[3], a[4]);
  *aL = mp5_upper(a[4], a[3], a[2], a[1], a[0]);
}

template <class R> void recon_cell(int scheme, const R a[5], R* aL, R* aR) {
  if (scheme == RECON_MINMOD) recon_minmod(a, aL, aR);
  else if (scheme == RECON_PPM) recon_ppm(a, aL, aR);
  else if (scheme == RECON_MP5) recon_mp5(a, aL, aR);
  else recon_wenoz(a, aL, aR);
}

// ------------------------------------------------------------------------------------------------------
// HLLE (Eq. HLLEfluxes): c_max = max(0, c+_l, c+_r), c_min = -min(0, c-_l, c-_r).

template <class R> void hlle(const R FL[5], const R FR[5], const R UL[5], const R UR[5], R cmax, R cmin, R out[5]) {
  const R den = cmax + cmin;
  for (int v = 0; v < 5; v++) {
    if (den > R(0.0))
      out[v] = (cmin * FR[v] + cmax * FL[v] - cmax * cmin * (UR[v] - UL[v])) / den;
    else
      out[v] = R(0.5) * (FL[v] + FR[v]);
  }
}

// Lax-Friedrichs (Eq. LxFfluxes): the average of the two fluxes minus c_wave / 2 times the jump of the conserved
// variables, c_wave = max(c_max, c_min).
template <class R> void lxf(const R FL[5], const R FR[5], const R UL[5], const R UR[5], R cmax, R cmin, R out[5]) {
  const R cw = rmax(cmax, cmin);
  for (int v = 0; v < 5; v++) out[v] = R(0.5) * (FR[v] + FL[v] - cw * (UR[v] - UL[v]));
}

// ------------------------------------------------------------------------------------------------------
// Face solve: from the reconstructed left/right states and the face metric, the HLLE (or Lax-Friedrichs) flux of
// the 5 hydro variables, the data that upwind constrained transport needs at this face (Eq. uct1, uct2), and
// for flux constrained transport the same solver's fluxes of the induction equation (Eq. inductioneq):
// along d the flux of B~^a (a != d) is v~^d B~^a - v~^a B~^d.

template <class R> struct FaceInputT {
  R rho[2], press[2], u[2][3], Bt[2][3];  // side 0 = left, 1 = right; u = W v; Bt: transverse B only
  R Bn;                                    // densitised normal field at the face (staggered)
};
typedef FaceInputT<double> FaceInput;

template <class R> struct FaceOut {
  R F[5];
  R vbar[3];  // upwind v~ components (the normal one unused)
  R Fb[3];    // induction fluxes along d of the densitised B~^a, a != d (the normal one unused)
  R cmax, cmin;
  int iters;
};

template <class R, class In>
FaceOut<R> face_solve(const Metric3<R>& m, const In& in, double gamma, int d, int solver = FLUX_HLLE,
                      bool induction = false) {
  FaceOut<R> out;
  R U[2][5], F[2][5], lp[2], lm[2], vt[2][3], Bt[2][3];
  out.iters = 0;
  for (int s = 0; s < 2; s++) {
    Prim<R> P;
    P.rho = R(in.rho[s]);
    P.press = R(in.press[s]);
    P.eps = P.press / (R(gamma - 1.0) * P.rho);  // ideal gas (Sec. 3.7)
    // W from u^i = W v^i: W^2 = 1 + gamma_ij u^i u^j
    R uu = R(0.0);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) uu += m.g[a][b] * R(in.u[s][a]) * R(in.u[s][b]);
    const R W = sqrt(R(1.0) + uu);
    for (int a = 0; a < 3; a++) P.vel[a] = R(in.u[s][a]) / W;
    for (int a = 0; a < 3; a++) P.B[a] = (a == d) ? R(in.Bn) / m.sqrtg : R(in.Bt[s][a]);
    Comoving<R> c = comoving(m, P);
    Cons<R> Us = prim2con(m, P, c);
    flux(m, P, c, Us, d, F[s]);
    U[s][0] = Us.D;
    U[s][1] = Us.S[0];
    U[s][2] = Us.S[1];
    U[s][3] = Us.S[2];
    U[s][4] = Us.tau;
    int it = 0;
    wave_speeds(m, P, c, gamma, d, &lm[s], &lp[s], &it);
    out.iters += it;
    for (int a = 0; a < 3; a++) vt[s][a] = m.alp * P.vel[a] - m.beta[a];
    for (int a = 0; a < 3; a++) Bt[s][a] = (a == d) ? R(in.Bn) : m.sqrtg * P.B[a];
  }
  out.cmax = rmax(R(0.0), rmax(lp[0], lp[1]));
  out.cmin = -rmin(R(0.0), rmin(lm[0], lm[1]));
  if (solver == FLUX_LXF) lxf(F[0], F[1], U[0], U[1], out.cmax, out.cmin, out.F);
  else hlle(F[0], F[1], U[0], U[1], out.cmax, out.cmin, out.F);
  // induction fluxes of the transverse B~ with the same solver (one-component forms of the above), when the
  // electric field is formed from them
  for (int a = 0; a < 3; a++) {
    if (a == d || !induction) {
      out.Fb[a] = R(0.0);
      continue;
    }
    R fl[5] = {vt[0][d] * Bt[0][a] - vt[0][a] * Bt[0][d], R(0.0), R(0.0), R(0.0), R(0.0)};
    R fr[5] = {vt[1][d] * Bt[1][a] - vt[1][a] * Bt[1][d], R(0.0), R(0.0), R(0.0), R(0.0)};
    R ul[5] = {Bt[0][a], R(0.0), R(0.0), R(0.0), R(0.0)};
    R ur[5] = {Bt[1][a], R(0.0), R(0.0), R(0.0), R(0.0)};
    R o5[5];
    if (solver == FLUX_LXF) lxf(fl, fr, ul, ur, out.cmax, out.cmin, o5);
    else hlle(fl, fr, ul, ur, out.cmax, out.cmin, o5);
    out.Fb[a] = o5[0];
  }
  const R den = out.cmax + out.cmin;
  for (int a = 0; a < 3; a++) {
    if (a == d) {
      out.vbar[a] = R(0.0);
    } else if (den > R(0.0)) {
      out.vbar[a] = (out.cmax * vt[0][a] + out.cmin * vt[1][a]) / den;
    } else {
      out.vbar[a] = R(0.5) * (vt[0][a] + vt[1][a]);
    }
  }
  return out;
}

// ------------------------------------------------------------------------------------------------------
// Primitive recovery (Sec. 3.5): Noble 2D Newton on (z, v^2), Palenzuela 1D Brent on x = hW, atmosphere.

struct C2POut {
  double rho, press, vel[3];
  int flag;   // 0 Noble, 1 Palenzuela, 2 atmosphere, -1 both failed (atmosphere applied)
  int iters;  // Noble iterations
  bool reset; // conserved variables must be reset to the atmosphere
};

struct C2PIn {
  double Dtilde;         // densitised D~ = sqrt(gamma) D, for the atmosphere test
  double D, S[3], tau;   // undensitised
  double B[3];           // undensitised centre field
  double guess_rho, guess_press, guess_vel[3];
};

// Noble et al. 2006 residuals, Eqs. (Noble2D momentum) and (Noble2D energy), with the ideal-gas pressure
// p(z, v^2) = (Gamma-1)/Gamma (z (1 - v^2) - D sqrt(1 - v^2)) that follows from z = rho h W^2, h = 1 + Gamma eps.
template <class R> void noble_residual(R z, R v2, R D, R tau, R S2, R B2, R BS, double gamma, R f[2], R J[2][2]) {
  const R gf = R((gamma - 1.0) / gamma);
  const R sq = sqrt(R(1.0) - v2);
  const R p = gf * (z * (R(1.0) - v2) - D * sq);
  const R dp_dz = gf * (R(1.0) - v2);
  const R dp_dv2 = gf * (-z + R(0.5) * D / sq);
  const R Bz = B2 + z;
  f[0] = v2 * Bz * Bz - BS * BS * (B2 + R(2.0) * z) / (z * z) - S2;
  f[1] = tau + D - R(0.5) * B2 * (R(1.0) + v2) + BS * BS / (R(2.0) * z * z) - z + p;
  J[0][0] = R(2.0) * v2 * Bz + R(2.0) * BS * BS * Bz / (z * z * z);
  J[0][1] = Bz * Bz;
  J[1][0] = -BS * BS / (z * z * z) - R(1.0) + dp_dz;
  J[1][1] = R(-0.5) * B2 + dp_dv2;
}

// A state-derived input of the recovery as a scalar of type R (a data value for the flop-counting scalar).
template <class R> inline R datum(double x) { return R(x); }
template <> inline Fc datum<Fc>(double x) { return fc_data(x); }

// velocity from Eq. (Noble2D v): v^i = gamma^ij S_j / (z + B^2) + (B^j S_j) B^i / (z (z + B^2))
template <class R>
static void noble_velocity(const Metric3<R>& m, const C2PIn& in, R z, R B2, R BS, R v[3]) {
  for (int a = 0; a < 3; a++) {
    R Su = m.gu[a][0] * datum<R>(in.S[0]) + m.gu[a][1] * datum<R>(in.S[1]) + m.gu[a][2] * datum<R>(in.S[2]);
    v[a] = Su / (z + B2) + BS * datum<R>(in.B[a]) / (z * (z + B2));
  }
}

template <class R> static bool bad(R x) { return !finite(x) || x < R(0.0); }

// x^(3/2); the flop-counting scalar counts it as one product and one square root
static double pow15(double x) { return std::pow(x, 1.5); }
static Fc pow15(Fc x) {
  g_flops.mul++;
  g_flops.sqrt++;
  return Fc(std::pow(x.v, 1.5));
}

// The recovery is templated on the scalar for the algorithmic flop count; the inputs (C2PIn) and results
// (C2POut) are plain doubles, and every branch is decided on values.
template <class R>
static bool c2p_noble(const Metric3<R>& m, const C2PIn& in, const OParams& P, R S2, R B2, R BS, C2POut* out) {
  const double gamma = P.gamma;
  const double v2max = 1.0 - 1.0 / (P.W_max * P.W_max);
  // initial guess from the previous primitives
  R gv2 = R(0.0);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) gv2 += m.g[a][b] * datum<R>(in.guess_vel[a]) * datum<R>(in.guess_vel[b]);
  if (!(gv2 >= R(0.0))) gv2 = R(0.0);
  if (gv2 > R(v2max)) gv2 = R(v2max);
  const R gW = R(1.0) / sqrt(R(1.0) - gv2);
  const R geps = datum<R>(in.guess_press) / (R(gamma - 1.0) * datum<R>(in.guess_rho));
  const R gh = R(1.0) + geps + datum<R>(in.guess_press) / datum<R>(in.guess_rho);
  R z = datum<R>(in.guess_rho) * gh * gW * gW;
  R v2 = gv2;
  if (!(z > R(0.0)) || !finite(z)) return false;
  bool conv = false;
  int it;
  for (it = 1; it <= P.c2p_maxiter; it++) {
    R f[2], J[2][2];
    noble_residual<R>(z, v2, datum<R>(in.D), datum<R>(in.tau), S2, B2, BS, gamma, f, J);
    const R det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const R dz = (-f[0] * J[1][1] + J[0][1] * f[1]) / det;
    const R dv2 = (-J[0][0] * f[1] + J[1][0] * f[0]) / det;
    // damped step: a step that would make z non-positive halves z instead (z = rho h W^2 > 0)
    const bool damped = !(z + dz > R(0.0));
    z = damped ? R(0.5) * z : z + dz;
    v2 += dv2;
    if (v2 < R(0.0)) v2 = R(0.0);
    if (v2 > R(v2max)) v2 = R(v2max);
    if (!finite(z) || !finite(v2)) break;
    if (!damped && fabs(dz) <= R(P.c2p_tol) * fabs(z) && fabs(dv2) <= R(P.c2p_tol)) {
      conv = true;
      break;
    }
  }
  out->iters = (it > P.c2p_maxiter) ? P.c2p_maxiter : it;
  if (!conv || !(z > R(0.0)) || !(v2 >= R(0.0)) || !(v2 < R(1.0))) return false;
  const R W = R(1.0) / sqrt(R(1.0) - v2);
  const R rho = datum<R>(in.D) / W;
  R v[3];
  noble_velocity<R>(m, in, z, B2, BS, v);
  const R eps = (z / (rho * W * W) - R(1.0)) / R(gamma);  // Eq. (Noble2D epsilon) with the adiabatic index
  const R press = R(gamma - 1.0) * rho * eps;
  if (bad(rho) || bad(eps) || bad(press)) return false;
  for (int a = 0; a < 3; a++)
    if (!finite(v[a])) return false;
  out->rho = val(rho);
  out->press = val(press);
  for (int a = 0; a < 3; a++) out->vel[a] = val(v[a]);
  return true;
}

// Palenzuela et al. 2015 function f(x) = x - h^ W^ (Eq. Palenzuela Brent), with W^, rho^, eps^ from x.
template <class R> struct PalenzuelaFn {
  R q, r, s, t, D;
  double gamma, v2max;
  R W, rho, eps, press;
  R operator()(R x) {
    R v2 = (r * x * x + t * t * (R(2.0) * x + s)) / (x * x * (x + s) * (x + s));
    if (v2 > R(v2max)) v2 = R(v2max);
    if (v2 < R(0.0)) v2 = R(0.0);
    W = R(1.0) / sqrt(R(1.0) - v2);
    rho = D / W;
    eps = R(-1.0) + (x / W) * (R(1.0) - W * W) + W * (R(1.0) + q - s + R(0.5) * (t * t / (x * x) + s / (W * W)));
    if (eps < R(0.0)) eps = R(0.0);
    press = R(gamma - 1.0) * rho * eps;
    const R h = R(1.0) + eps + press / rho;
    return x - h * W;
  }
};

// Brent's method (Brent 1973, "Algorithms for Minimization without Derivatives", ch. 4): keep a bracket
// [b, c] with a sign change, b the best iterate; try inverse quadratic interpolation (or the secant when only
// two points are distinct) and fall back to bisection whenever the interpolated step is not safely inside
// the bracket or does not shrink fast enough.
template <class R, class F> static bool brent_root(F& f, R lo, R hi, R xtol, int maxiter, R* root) {
  R a = lo, b = hi;
  R fa = f(a), fb = f(b);
  if (!finite(fa) || !finite(fb)) return false;
  if ((fa > R(0.0) && fb > R(0.0)) || (fa < R(0.0) && fb < R(0.0))) return false;
  R c = a, fc = fa;
  R step = b - a, prev_step = step;
  for (int it = 0; it < maxiter; it++) {
    if ((fb > R(0.0) && fc > R(0.0)) || (fb < R(0.0) && fc < R(0.0))) {
      c = a;  // re-establish the bracket [b, c]
      fc = fa;
      step = prev_step = b - a;
    }
    if (fabs(fc) < fabs(fb)) {  // make b the better end
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    const R tol = R(2.0 * 2.220446049250313e-16) * fabs(b) + R(0.5) * xtol;
    const R half = R(0.5) * (c - b);
    if (fabs(half) <= tol || fb == R(0.0)) {
      *root = b;
      return true;
    }
    bool bisect = true;
    if (fabs(prev_step) >= tol && fabs(fa) > fabs(fb)) {
      R num, den;
      const R sb = fb / fa;
      if (a == c) {  // secant through a, b
        num = R(2.0) * half * sb;
        den = R(1.0) - sb;
      } else {       // inverse quadratic interpolation through a, b, c
        const R qa = fa / fc, rb = fb / fc;
        num = sb * (R(2.0) * half * qa * (qa - rb) - (b - a) * (rb - R(1.0)));
        den = (qa - R(1.0)) * (rb - R(1.0)) * (sb - R(1.0));
      }
      if (num > R(0.0)) den = -den;
      else num = -num;
      const R lim1 = R(3.0) * half * den - fabs(tol * den);
      const R lim2 = fabs(prev_step * den);
      if (R(2.0) * num < (lim1 < lim2 ? lim1 : lim2)) {
        prev_step = step;
        step = num / den;
        bisect = false;
      }
    }
    if (bisect) {
      step = half;
      prev_step = step;
    }
    a = b;
    fa = fb;
    if (fabs(step) > tol) b += step;
    else b += (half > R(0.0) ? tol : -tol);
    fb = f(b);
    if (!finite(fb)) return false;
  }
  return false;
}

template <class R>
static bool c2p_palenzuela(const Metric3<R>& m, const C2PIn& in, const OParams& P, R S2, R B2, R BS,
                           C2POut* out) {
  PalenzuelaFn<R> f;
  const R D = datum<R>(in.D);
  f.q = datum<R>(in.tau) / D;
  f.r = S2 / (D * D);
  f.s = B2 / D;
  f.t = BS / pow15(D);
  f.D = D;
  f.gamma = P.gamma;
  f.v2max = 1.0 - 1.0 / (P.W_max * P.W_max);
  R lo = R(1.0) + f.q - f.s;
  if (lo < R(1.0)) lo = R(1.0);
  const R hi = R(2.0) + R(2.0) * f.q - f.s;
  if (!(hi > lo)) return false;
  R x;
  if (!brent_root<R>(f, lo, hi, R(1e-15) * hi, P.brent_maxiter, &x)) return false;
  f(x);  // primitives at the root
  const R z = D * x;  // z = rho W x (Eq. Noble2D z with x = hW)
  R v[3];
  noble_velocity<R>(m, in, z, B2, BS, v);
  if (bad(f.rho) || bad(f.eps) || bad(f.press)) return false;
  for (int a = 0; a < 3; a++)
    if (!finite(v[a])) return false;
  out->rho = val(f.rho);
  out->press = val(f.press);
  for (int a = 0; a < 3; a++) out->vel[a] = val(v[a]);
  return true;
}

// Atmosphere (Sec. 3.6): rho = rho_atm, polytropic p and eps, v = 0.
static void atmosphere(const OParams& P, C2POut* out) {
  out->rho = P.rho_atm;
  out->press = P.K_atm * std::pow(P.rho_atm, P.gamma_atm);
  out->vel[0] = out->vel[1] = out->vel[2] = 0.0;
  out->reset = true;
}

template <class R> static C2POut c2p_cell(const Metric3<R>& m, const C2PIn& in, const OParams& P) {
  C2POut out;
  out.flag = 0;
  out.iters = 0;
  out.reset = false;
  // atmosphere test on the densitised density before the recovery: D~ < sqrt(gamma) rho_atm
  if (!(datum<R>(in.Dtilde) >= m.sqrtg * R(P.rho_atm))) {
    atmosphere(P, &out);
    out.flag = 2;
    return out;
  }
  R S2 = R(0.0), B2 = R(0.0), BS = R(0.0);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      S2 += m.gu[a][b] * datum<R>(in.S[a]) * datum<R>(in.S[b]);
      B2 += m.g[a][b] * datum<R>(in.B[a]) * datum<R>(in.B[b]);
    }
  for (int a = 0; a < 3; a++) BS += datum<R>(in.B[a]) * datum<R>(in.S[a]);
  bool ok = c2p_noble<R>(m, in, P, S2, B2, BS, &out);
  if (ok) {
    out.flag = 0;
  } else if (P.use_fallback) {
    ok = c2p_palenzuela<R>(m, in, P, S2, B2, BS, &out);
    if (ok) out.flag = 1;
  }
  if (!ok) {
    atmosphere(P, &out);
    out.flag = -1;
  }
  return out;
}

// ------------------------------------------------------------------------------------------------------
// Ghost zones (Sec. 3.8): periodic wrap, or copy of the nearest owned value (linear extrapolation for A).

// stagger: 1 if the quantity is cell-like along `axis`, 0 if vertex-like.
template <class R> static void fill_axis(const Grid& G, R* f, int axis, int cell_like, bool linear) {
  const int n = G.n[axis], g = G.g, Nn = G.N[axis];
  const int lo = g;
  const int hi = (cell_like || G.bc[axis] == BC_PERIODIC) ? g + n - 1 : g + n;  // owned index range [lo, hi]
  const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
  for (int q2 = 0; q2 <= G.N[a2]; q2++)
    for (int q1 = 0; q1 <= G.N[a1]; q1++)
      for (int i = 0; i <= Nn; i++) {
        if (i >= lo && i <= hi) continue;
        int p[3];
        p[axis] = i;
        p[a1] = q1;
        p[a2] = q2;
        R v;
        if (G.bc[axis] == BC_PERIODIC) {
          int src = lo + (((i - lo) % n) + n) % n;  // periodic image inside the owned range
          int q[3] = {p[0], p[1], p[2]};
          q[axis] = src;
          v = f[G.at(q)];
        } else {
          int e0 = (i < lo) ? lo : hi;
          int e1 = (i < lo) ? lo + 1 : hi - 1;
          int q0[3] = {p[0], p[1], p[2]}, q1v[3] = {p[0], p[1], p[2]};
          q0[axis] = e0;
          q1v[axis] = e1;
          if (linear && hi > lo) {  // linear extrapolation needs two owned layers; one layer copies
            const R f0 = f[G.at(q0)], f1 = f[G.at(q1v)];
            v = f0 + R((double)(i < lo ? lo - i : i - hi)) * (f0 - f1);
          } else {
            v = f[G.at(q0)];
          }
        }
        f[G.at(p)] = v;
      }
}

// cell_like[field][axis] for D, Sx, Sy, Sz, tau, Ax, Ay, Az, Psi
static const int STATE_CELL_LIKE[9][3] = {{1, 1, 1}, {1, 1, 1}, {1, 1, 1}, {1, 1, 1}, {1, 1, 1},
                                          {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 0, 0}};

template <class R> static void ghost_fill_state(const Grid& G, R* const U[9]) {
  for (int axis = 0; axis < 3; axis++)
    for (int v = 0; v < 9; v++) fill_axis(G, U[v], axis, STATE_CELL_LIKE[v][axis], v >= 5 && v <= 7);
}

template <class R> static void ghost_fill_prims(const Grid& G, R* const P[5]) {
  for (int axis = 0; axis < 3; axis++)
    for (int v = 0; v < 5; v++) fill_axis(G, P[v], axis, 1, false);
}

// ------------------------------------------------------------------------------------------------------
// Magnetic field from the vector potential (Sec. 3.4, Eq. BEulerian): B~^i = [ijk] d_j A_k on faces, by
// second-order differences of the edge values.  Cell-centre B^i = (B~^i_- + B~^i_+) / (2 sqrt(gamma_c)).

template <class R>
static void face_B(const Grid& G, const R* Ax, const R* Ay, const R* Az, std::vector<R> Bf[3]) {
  for (int d = 0; d < 3; d++) Bf[d].assign(G.size(), R(0.0));
  const double ix = 1.0 / G.dx[0], iy = 1.0 / G.dx[1], iz = 1.0 / G.dx[2];
  ORACLE_PAR(R)
  for (int k = 0; k <= G.N[2]; k++)
    for (int j = 0; j <= G.N[1]; j++)
      for (int i = 0; i <= G.N[0]; i++) {
        const long c = G.at(i, j, k);
        if (j < G.N[1] && k < G.N[2])  // x-face (i, j+1/2, k+1/2)
          Bf[0][c] = (Az[G.at(i, j + 1, k)] - Az[c]) * R(iy) - (Ay[G.at(i, j, k + 1)] - Ay[c]) * R(iz);
        if (i < G.N[0] && k < G.N[2])  // y-face (i+1/2, j, k+1/2)
          Bf[1][c] = (Ax[G.at(i, j, k + 1)] - Ax[c]) * R(iz) - (Az[G.at(i + 1, j, k)] - Az[c]) * R(ix);
        if (i < G.N[0] && j < G.N[1])  // z-face (i+1/2, j+1/2, k)
          Bf[2][c] = (Ay[G.at(i + 1, j, k)] - Ay[c]) * R(ix) - (Ax[G.at(i, j + 1, k)] - Ax[c]) * R(iy);
      }
}

template <class R>
static void centre_B(const Grid& G, const VertexMetric& vm, const std::vector<R> Bf[3], std::vector<R> Bc[3]) {
  for (int d = 0; d < 3; d++) Bc[d].assign(G.size(), R(0.0));
  ORACLE_PAR(R)
  for (int k = 0; k < G.N[2]; k++)
    for (int j = 0; j < G.N[1]; j++)
      for (int i = 0; i < G.N[0]; i++) {
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        const long c = G.at(i, j, k);
        for (int d = 0; d < 3; d++) {
          const long c1 = c + G.s[d];
          Bc[d][c] = R(0.5) * (Bf[d][c] + Bf[d][c1]) / R(m.sqrtg);
        }
      }
}

// ------------------------------------------------------------------------------------------------------
// Source terms (Eq. grmhdsrc, written in 3+1 form with the input K_ij; K = -1/2 L_n gamma, Sec. 2.1):
//   tau~ : alpha sqrt(g) [T^00 (b^i b^j K_ij - b^i d_i alpha) + T^0i (2 b^j K_ij - d_i alpha) + T^ij K_ij]
//   S~_i : alpha sqrt(g) [-T^00 alpha d_i alpha + T^0_k d_i beta^k + 1/2 (T^00 b^j b^k + 2 T^0j b^k + T^jk) d_i g_jk]
// (b = beta here), with T^{mu nu} of Eq. tmunu.

template <class R> struct MetricDeriv {
  R dalp[3], dbeta[3][3], dg[3][3][3];  // d_i alpha, d_i beta^j, d_i gamma_jk
};

template <class R> void source_terms(const Metric3<R>& m, const MetricDeriv<R>& dm, const Prim<R>& P, R src[5]) {
  Comoving<R> c = comoving(m, P);
  const R a2 = m.alp * m.alp;
  R guu[4][4];  // inverse 4-metric
  guu[0][0] = R(-1.0) / a2;
  for (int i = 0; i < 3; i++) {
    guu[0][i + 1] = m.beta[i] / a2;
    guu[i + 1][0] = guu[0][i + 1];
    for (int j = 0; j < 3; j++) guu[i + 1][j + 1] = m.gu[i][j] - m.beta[i] * m.beta[j] / a2;
  }
  R u[4], b[4];
  u[0] = c.u0;
  b[0] = c.b0;
  for (int i = 0; i < 3; i++) {
    u[i + 1] = c.uup[i];
    b[i + 1] = c.bup[i];
  }
  const R rhohb = P.rho * c.h + c.b2;
  const R ptot = P.press + R(0.5) * c.b2;
  R T[4][4];
  for (int mu = 0; mu < 4; mu++)
    for (int nu = 0; nu < 4; nu++) T[mu][nu] = rhohb * u[mu] * u[nu] + ptot * guu[mu][nu] - b[mu] * b[nu];
  R betalow[3];
  for (int k = 0; k < 3; k++) betalow[k] = m.g[k][0] * m.beta[0] + m.g[k][1] * m.beta[1] + m.g[k][2] * m.beta[2];
  R T0low[3];  // T^0_k = g_k0 T^00 + g_kj T^0j
  for (int k = 0; k < 3; k++) {
    T0low[k] = betalow[k] * T[0][0];
    for (int j = 0; j < 3; j++) T0low[k] += m.g[k][j] * T[0][j + 1];
  }
  const R asg = m.alp * m.sqrtg;
  // energy
  R st = R(0.0);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) st += T[0][0] * m.beta[i] * m.beta[j] * m.K[i][j];
  for (int i = 0; i < 3; i++) st -= T[0][0] * m.beta[i] * dm.dalp[i];
  for (int i = 0; i < 3; i++) {
    R bk = R(0.0);
    for (int j = 0; j < 3; j++) bk += R(2.0) * m.beta[j] * m.K[i][j];
    st += T[0][i + 1] * (bk - dm.dalp[i]);
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) st += T[i + 1][j + 1] * m.K[i][j];
  src[0] = R(0.0);
  src[4] = asg * st;
  // momentum
  for (int i = 0; i < 3; i++) {
    R s = -T[0][0] * m.alp * dm.dalp[i];
    for (int k = 0; k < 3; k++) s += T0low[k] * dm.dbeta[i][k];
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++)
        s += R(0.5) * (T[0][0] * m.beta[j] * m.beta[k] + R(2.0) * T[0][j + 1] * m.beta[k] + T[j + 1][k + 1]) *
             dm.dg[i][j][k];
    src[1 + i] = asg * s;
  }
}

static MetricDeriv<double> metric_deriv_at_centre(const Grid& G, const VertexMetric& vm, int i, int j, int k) {
  MetricDeriv<double> dm;
  const int p[3] = {i, j, k};
  const int half[3] = {1, 1, 1};
  for (int d = 0; d < 3; d++) {
    dm.dalp[d] = vertex_interp(G, vm.f[0], p, half, d);
    for (int a = 0; a < 3; a++) dm.dbeta[d][a] = vertex_interp(G, vm.f[1 + a], p, half, d);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) dm.dg[d][a][b] = vertex_interp(G, vm.f[4 + SYM[a][b]], p, half, d);
  }
  return dm;
}

template <class R> MetricDeriv<R> lift_deriv(const MetricDeriv<double>& d) {
  MetricDeriv<R> r;
  for (int a = 0; a < 3; a++) {
    r.dalp[a] = R(d.dalp[a]);
    for (int b = 0; b < 3; b++) {
      r.dbeta[a][b] = R(d.dbeta[a][b]);
      for (int c = 0; c < 3; c++) r.dg[a][b][c] = R(d.dg[a][b][c]);
    }
  }
  return r;
}

// ------------------------------------------------------------------------------------------------------
// The right-hand side of one stage (Sec. 3.12 workflow: reconstruct, Riemann solve, sources; Sec. 3.4 for
// the potentials).  Inputs: state with ghosts filled and primitives with ghosts filled.

struct RhsStats {
  unsigned long long speed_iters, faces;
};

template <class R> struct FaceDataT {
  std::vector<R> F[5], vbar[3], Fb[3], cmax, cmin;
};

template <class R>
static void compute_faces(const Grid& G, const VertexMetric& vm, const OParams& P, R* const prim[5],
                          const std::vector<R> Bf[3], const std::vector<R> Bc[3], int d, FaceDataT<R>& fd,
                          RhsStats* st) {
  for (int v = 0; v < 5; v++) fd.F[v].assign(G.size(), R(0.0));
  for (int v = 0; v < 3; v++) fd.vbar[v].assign(G.size(), R(0.0));
  for (int v = 0; v < 3; v++) fd.Fb[v].assign(G.size(), R(0.0));
  fd.cmax.assign(G.size(), R(0.0));
  fd.cmin.assign(G.size(), R(0.0));
  // reconstructed variables at every cell: rho, p, u^x, u^y, u^z (u = W v) and the centre B
  std::vector<R> cellvar[8];
  for (int v = 0; v < 8; v++) cellvar[v].assign(G.size(), R(0.0));
  {
  FlopScope<R> scope(&g_cellvar_flops);
  ORACLE_PAR(R)
  for (int k = 0; k < G.N[2]; k++)
    for (int j = 0; j < G.N[1]; j++)
      for (int i = 0; i < G.N[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        R v2 = R(0.0);
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) v2 += R(m.g[a][b]) * prim[2 + a][c] * prim[2 + b][c];
        const R W = R(1.0) / sqrt(R(1.0) - v2);
        cellvar[0][c] = prim[0][c];
        cellvar[1][c] = prim[1][c];
        for (int a = 0; a < 3; a++) cellvar[2 + a][c] = W * prim[2 + a][c];
        for (int a = 0; a < 3; a++) cellvar[5 + a][c] = Bc[a][c];
      }
  }
  const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
  unsigned long long n_iters = 0, n_faces = 0;
  ORACLE_PAR_REDUCE(R, reduction(+ : n_iters, n_faces))
  for (int q2 = 0; q2 < G.N[a2]; q2++)
    for (int q1 = 0; q1 < G.N[a1]; q1++)
      for (int f = G.g; f <= G.g + G.n[d]; f++) {
        int p[3];
        p[d] = f;
        p[a1] = q1;
        p[a2] = q2;
        const long fc = G.at(p);
        FaceInputT<R> in;
        {
        FlopScope<R> recon_scope(&g_recon_flops);
        for (int s = 0; s < 2; s++) {
          // left state: upper face value of cell f-1; right state: lower face value of cell f
          const int cell = f - 1 + s;
          R stencil[8][5];
          for (int t = 0; t < 5; t++) {
            int q[3] = {p[0], p[1], p[2]};
            q[d] = cell - 2 + t;
            const long cc = G.at(q);
            for (int v = 0; v < 8; v++) stencil[v][t] = cellvar[v][cc];
          }
          R rec[8];
          for (int v = 0; v < 8; v++) {
            if (v >= 5 && v - 5 == d) {
              rec[v] = R(0.0);  // normal B is the staggered face value, not reconstructed
              continue;
            }
            R aL, aR;
            recon_cell<R>(P.recon, stencil[v], &aL, &aR);
            rec[v] = (s == 0) ? aR : aL;
          }
          in.rho[s] = rec[0];
          in.press[s] = rec[1];
          for (int a = 0; a < 3; a++) in.u[s][a] = rec[2 + a];
          for (int a = 0; a < 3; a++) in.Bt[s][a] = rec[5 + a];
        }
        }
        in.Bn = Bf[d][fc];
        const Metric3<R> m = lift<R>(metric_at_face(G, vm, d, p[0], p[1], p[2]));
        FaceOut<R> o;
        {
          FlopScope<R> solve_scope(&g_facesolve_flops);
          o = face_solve<R>(m, in, P.gamma, d, P.flux, P.efield == EFIELD_FCT);
        }
        for (int v = 0; v < 5; v++) fd.F[v][fc] = o.F[v];
        for (int a = 0; a < 3; a++) fd.vbar[a][fc] = o.vbar[a];
        for (int a = 0; a < 3; a++) fd.Fb[a][fc] = o.Fb[a];
        fd.cmax[fc] = o.cmax;
        fd.cmin[fc] = o.cmin;
        n_iters += o.iters;
        n_faces++;
      }
  if (st) {
    st->speed_iters += n_iters;
    st->faces += n_faces;
  }
}

// PPM value at the interface between stencil positions 2 and 3 of f[0..5]: left = upper value of cell 2
// (stencil 0..4), right = lower value of cell 3 (stencil 1..5).
template <class T> static void ppm_interface(const T f[6], T* L, T* R) {
  T aL, aR;
  recon_ppm<T>(f, &aL, &aR);
  *L = aR;
  recon_ppm<T>(f + 1, &aL, &aR);
  *R = aL;
}

template <class T> static T hll_edge(T ap, T am, T vL, T BL, T vR, T BR) {
  const T den = ap + am;
  if (den > T(0.0)) return (ap * vL * BL + am * vR * BR - ap * am * (BR - BL)) / den;
  return T(0.5) * (vL * BL + vR * BR);
}

// Upwind constrained transport (Sec. 3.4, Eqs. uct1, uct2, eq3.20) for the edge along e at vertex-index
// position p, with (e, d1, d2) cyclic:  E_e = -HLL_d1(v^d1 B~^d2) + HLL_d2(v^d2 B~^d1), the products
// reconstructed (PPM) to the edge from the faces normal to d2 (resp. d1), and a^d_+- at the edge the maximum
// over the two d-faces sharing the edge.
template <class R>
static R uct_E(const Grid& G, const FaceDataT<R> fd[3], const std::vector<R> Bf[3], int e, const int p[3]) {
  const int d1 = (e + 1) % 3, d2 = (e + 2) % 3;
  R term[2];
  for (int t = 0; t < 2; t++) {
    const int dr = (t == 0) ? d1 : d2;    // direction of reconstruction / upwinding
    const int df = (t == 0) ? d2 : d1;    // normal of the faces that carry the data
    R vs[6], bs[6];
    for (int s = 0; s < 6; s++) {
      int q[3] = {p[0], p[1], p[2]};
      q[dr] = p[dr] - 3 + s;
      const long c = G.at(q);
      vs[s] = fd[df].vbar[dr][c];
      bs[s] = Bf[df][c];
    }
    R vL, vR, BL, BR;
    {
      FlopScope<R> scope(&g_edge_ppm_flops);
      ppm_interface(vs, &vL, &vR);
      ppm_interface(bs, &BL, &BR);
    }
    // speeds along dr: the two dr-faces sharing the edge are at p - e_df and p
    int q0[3] = {p[0], p[1], p[2]};
    q0[df] -= 1;
    const long c0 = G.at(q0), c1 = G.at(p);
    const R ap = rmax(fd[dr].cmax[c0], fd[dr].cmax[c1]);
    const R am = rmax(fd[dr].cmin[c0], fd[dr].cmin[c1]);
    term[t] = hll_edge(ap, am, vL, BL, vR, BR);
  }
  return -term[0] + term[1];
}

// Flux constrained transport (Sec. 3.4; Balsara & Spicer 1999): the electric field on the edge along e at
// vertex-index position p is the average of the induction fluxes on the four faces that share the edge.  With
// (e, d1, d2) cyclic and E = -v~ x B~, the flux along d1 of B~^d2 is -E_e and the flux along d2 of B~^d1 is +E_e;
// the d1-faces sharing the edge sit at p and p - e_d2, the d2-faces at p and p - e_d1.
template <class R> static R fct_E(const Grid& G, const FaceDataT<R> fd[3], int e, const int p[3]) {
  const int d1 = (e + 1) % 3, d2 = (e + 2) % 3;
  int q1[3] = {p[0], p[1], p[2]};
  q1[d2] -= 1;
  int q2[3] = {p[0], p[1], p[2]};
  q2[d1] -= 1;
  const R f1 = fd[d1].Fb[d2][G.at(p)] + fd[d1].Fb[d2][G.at(q1)];
  const R f2 = fd[d2].Fb[d1][G.at(p)] + fd[d2].Fb[d1][G.at(q2)];
  return R(0.25) * (f2 - f1);
}

struct RhsOut {
  double* const* dU;  // 9 fields (D, Sx, Sy, Sz, tau at cells; Ax, Ay, Az at edges; Psi at vertices)
};

template <class R>
static void rhs(const Grid& G, const VertexMetric& vm, const OParams& P, double dt, R* const U[9],
                R* const prim[5], R* const dU[9], RhsStats* st) {
  std::vector<R> Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  FaceDataT<R> fd[3];
  const bool marks = std::is_same<R, Fc>::value && g_rhs_marks;
  if (marks) g_rhs_marks[0] = g_flops;
  for (int d = 0; d < 3; d++) compute_faces(G, vm, P, prim, Bf, Bc, d, fd[d], st);
  if (marks) g_rhs_marks[1] = g_flops;
  const int g = G.g;
  // hydro: flux divergence plus sources at interior cells
  ORACLE_PAR(R)
  for (int k = g; k < g + G.n[2]; k++)
    for (int j = g; j < g + G.n[1]; j++)
      for (int i = g; i < g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        R r[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
        for (int d = 0; d < 3; d++) {
          const long c1 = c + G.s[d];
          for (int v = 0; v < 5; v++) r[v] -= (fd[d].F[v][c1] - fd[d].F[v][c]) / R(G.dx[d]);
        }
        const Metric3<R> m = lift<R>(metric_at_centre(G, vm, i, j, k));
        const MetricDeriv<R> dm = lift_deriv<R>(metric_deriv_at_centre(G, vm, i, j, k));
        Prim<R> pr;
        pr.rho = prim[0][c];
        pr.press = prim[1][c];
        pr.eps = pr.press / (R(P.gamma - 1.0) * pr.rho);
        for (int a = 0; a < 3; a++) {
          pr.vel[a] = prim[2 + a][c];
          pr.B[a] = Bc[a][c];
        }
        R src[5];
        source_terms<R>(m, dm, pr, src);
        for (int v = 0; v < 5; v++) dU[v][c] = r[v] + src[v];
      }
  if (marks) g_rhs_marks[2] = g_flops;
  // potentials: G_A and F_Psi at vertices, from the vertex average of the edge A_j (Sec. 3.4)
  std::vector<R> GA(G.size(), R(0.0)), FPsi[3];
  for (int d = 0; d < 3; d++) FPsi[d].assign(G.size(), R(0.0));
  const bool lorenz = (P.gauge == GAUGE_LORENZ);
  ORACLE_PAR(R)
  for (int k = 1; k <= G.N[2]; k++)
    for (int j = 1; j <= G.N[1]; j++)
      for (int i = 1; i <= G.N[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<R> m = lift<R>(metric_at_vertex(G, vm, i, j, k));
        R Av[3];
        for (int a = 0; a < 3; a++) Av[a] = R(0.5) * (U[5 + a][c - G.s[a]] + U[5 + a][c]);
        const R psi = U[8][c];
        R bA = R(0.0);
        for (int a = 0; a < 3; a++) bA += m.beta[a] * Av[a];
        GA[c] = lorenz ? (m.alp * psi / m.sqrtg - bA) : R(0.0);
        for (int a = 0; a < 3; a++) {
          R Aup = m.gu[a][0] * Av[0] + m.gu[a][1] * Av[1] + m.gu[a][2] * Av[2];
          FPsi[a][c] = m.alp * m.sqrtg * Aup - m.beta[a] * psi;
        }
      }
  if (marks) g_rhs_marks[3] = g_flops;
  // dA_e/dt = -E_e - d_e G_A on edges
  for (int e = 0; e < 3; e++) {
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
      lo[a] = g;
      hi[a] = (a == e) ? g + G.n[a] - 1 : g + G.n[a];
    }
    ORACLE_PAR(R)
    for (int k = lo[2]; k <= hi[2]; k++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          const int p[3] = {i, j, k};
          const long c = G.at(p);
          const R E = (P.efield == EFIELD_FCT) ? fct_E(G, fd, e, p) : uct_E(G, fd, Bf, e, p);
          const R dG = (GA[c + G.s[e]] - GA[c]) / R(G.dx[e]);
          dU[5 + e][c] = -E - dG;
        }
  }
  if (marks) g_rhs_marks[4] = g_flops;
  // dPsi/dt = -d_j F_Psi^j - xi alpha Psi at vertices (Eq. recastedScalarPot)
  const double xi = (P.xi_lorenz > 0.0) ? P.xi_lorenz : 1.5 / dt;
  ORACLE_PAR(R)
  for (int k = g; k <= g + G.n[2]; k++)
    for (int j = g; j <= g + G.n[1]; j++)
      for (int i = g; i <= g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        if (!lorenz) {
          dU[8][c] = R(0.0);
          continue;
        }
        R div = R(0.0);
        for (int a = 0; a < 3; a++) div += (FPsi[a][c + G.s[a]] - FPsi[a][c - G.s[a]]) / R(2.0 * G.dx[a]);
        dU[8][c] = -div - R(xi * vm.f[0][c]) * U[8][c];
      }
}

// ------------------------------------------------------------------------------------------------------
// Recovery over the interior cells of a block.

static void con2prim(const Grid& G, const VertexMetric& vm, const OParams& P, double* const U[9],
                     double* const prim[5], signed char* flags, OStats* stats) {
  Field Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  const int g = G.g;
  unsigned long long s_iters = 0, s_noble = 0, s_fb = 0, s_atm = 0, s_failed = 0;
  ORACLE_PAR_REDUCE(double, reduction(+ : s_iters, s_noble, s_fb, s_atm, s_failed))
  for (int k = g; k < g + G.n[2]; k++)
    for (int j = g; j < g + G.n[1]; j++)
      for (int i = g; i < g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        C2PIn in;
        in.Dtilde = U[0][c];
        in.D = U[0][c] / m.sqrtg;
        for (int a = 0; a < 3; a++) in.S[a] = U[1 + a][c] / m.sqrtg;
        in.tau = U[4][c] / m.sqrtg;
        for (int a = 0; a < 3; a++) in.B[a] = Bc[a][c];
        in.guess_rho = prim[0][c];
        in.guess_press = prim[1][c];
        for (int a = 0; a < 3; a++) in.guess_vel[a] = prim[2 + a][c];
        C2POut o = c2p_cell(m, in, P);
        prim[0][c] = o.rho;
        prim[1][c] = o.press;
        for (int a = 0; a < 3; a++) prim[2 + a][c] = o.vel[a];
        if (flags) flags[c] = (signed char)o.flag;
        s_iters += o.iters;
        if (o.flag == 0) s_noble++;
        else if (o.flag == 1) s_fb++;
        else if (o.flag == 2) s_atm++;
        else s_failed++;
        if (o.reset) {
          // conserved variables reset from the atmosphere primitives with B kept (Sec. 3.6)
          Prim<double> pr;
          pr.rho = o.rho;
          pr.press = o.press;
          pr.eps = o.press / ((P.gamma_atm - 1.0) * o.rho);
          for (int a = 0; a < 3; a++) {
            pr.vel[a] = 0.0;
            pr.B[a] = Bc[a][c];
          }
          Comoving<double> cm = comoving(m, pr);
          Cons<double> uc = prim2con(m, pr, cm);
          U[0][c] = uc.D;
          for (int a = 0; a < 3; a++) U[1 + a][c] = uc.S[a];
          U[4][c] = uc.tau;
        }
      }
  if (stats) {
    stats->iters += s_iters;
    stats->n_noble += s_noble;
    stats->n_fallback += s_fb;
    stats->n_atm += s_atm;
    stats->n_failed += s_failed;
  }
}

// Conserved variables at all cells from primitives (initial data, Sec. 3.12 and Eq. cons): B~ = curl A on
// faces, B at centres, then the pointwise map.  R = Dual1 carries a direction in (A, primitives) through it.
template <class R>
static void prim2con_fields(const Grid& G, const VertexMetric& vm, const OParams& P, const R* const A[3],
                            const R* const prim[5], R* const U[5]) {
  std::vector<R> Bf[3], Bc[3];
  face_B(G, A[0], A[1], A[2], Bf);
  centre_B(G, vm, Bf, Bc);
  ORACLE_PAR(R)
  for (int k = 0; k < G.N[2]; k++)
    for (int j = 0; j < G.N[1]; j++)
      for (int i = 0; i < G.N[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<R> m = lift<R>(metric_at_centre(G, vm, i, j, k));
        Prim<R> pr;
        pr.rho = prim[0][c];
        pr.press = prim[1][c];
        pr.eps = pr.press / (R(P.gamma - 1.0) * pr.rho);
        for (int a = 0; a < 3; a++) {
          pr.vel[a] = prim[2 + a][c];
          pr.B[a] = Bc[a][c];
        }
        Comoving<R> cm = comoving(m, pr);
        Cons<R> uc = prim2con(m, pr, cm);
        U[0][c] = uc.D;
        for (int a = 0; a < 3; a++) U[1 + a][c] = uc.S[a];
        U[4][c] = uc.tau;
      }
}

static void prim2con_grid(const Grid& G, const VertexMetric& vm, const OParams& P, double* const U[9],
                          double* const prim[5]) {
  const double* A[3] = {U[5], U[6], U[7]};
  prim2con_fields<double>(G, vm, P, A, prim, U);
}

// ------------------------------------------------------------------------------------------------------
// Classical RK4 stage (method of lines): k_s = L(U_s); U_{s+1} = U_n + c_{s+1} dt k_s, c = (1/2, 1/2, 1);
// U_acc accumulates b_s dt k_s, b = (1/6, 1/3, 1/3, 1/6); the last stage writes U_n + U_acc + dt/6 k_3.
// Stages 4 and 5 are the two stages of RK2, the explicit midpoint method: U_1 = U_n + dt/2 k(U_n), then
// U_{n+1} = U_n + dt k(U_1) (U_acc unused).
// Stage order (Sec. 3.12): ghost fill U_s, con2prim on the interior, ghost fill primitives, RHS, combine.

static void owned_range(const Grid& G, int v, int lo[3], int hi[3]) {
  for (int a = 0; a < 3; a++) {
    lo[a] = G.g;
    hi[a] = STATE_CELL_LIKE[v][a] ? G.g + G.n[a] - 1 : G.g + G.n[a];
  }
}

static void rk_stage(const Grid& G, const VertexMetric& vm, const OParams& P, int stage, double dt,
                     double* const Un[9], double* const Us[9], double* const Unext[9], double* const Uacc[9],
                     double* const prim[5], signed char* flags, OStats* stats, bool fill_ghosts = true) {
  if (fill_ghosts) ghost_fill_state(G, Us);
  con2prim(G, vm, P, Us, prim, flags, stats);
  if (fill_ghosts) ghost_fill_prims(G, prim);
  std::vector<Field> k(9, Field(G.size(), 0.0));
  double* kp[9];
  for (int v = 0; v < 9; v++) kp[v] = k[v].data();
  rhs(G, vm, P, dt, Us, prim, kp, nullptr);
  static const double cnext[3] = {0.5, 0.5, 1.0};
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  for (int v = 0; v < 9; v++) {
    int lo[3], hi[3];
    owned_range(G, v, lo, hi);
    ORACLE_PAR(double)
    for (int kk = lo[2]; kk <= hi[2]; kk++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          const long c = G.at(i, j, kk);
          const double kv = k[v][c];
          if (stage == 0) {
            Uacc[v][c] = bw[0] * dt * kv;
            Unext[v][c] = Un[v][c] + cnext[0] * dt * kv;
          } else if (stage < 3) {
            Uacc[v][c] = Uacc[v][c] + bw[stage] * dt * kv;
            Unext[v][c] = Un[v][c] + cnext[stage] * dt * kv;
          } else if (stage == 3) {
            Unext[v][c] = Un[v][c] + Uacc[v][c] + bw[3] * dt * kv;
          } else if (stage == 4) {  // RK2 (explicit midpoint), first stage
            Unext[v][c] = Un[v][c] + 0.5 * dt * kv;
          } else {  // RK2, second stage: the slope at the midpoint state
            Unext[v][c] = Un[v][c] + dt * kv;
          }
        }
  }
}

// ------------------------------------------------------------------------------------------------------
// Stress-energy tensor at vertices (Eq. tmunu; T_{mu nu} is stored at vertices, Sec. 3.1).  The cell-centred
// rest-mass density, pressure, u^i = W v^i (W from the cell's metric) and centre field B^i of the eight cells
// around a vertex are averaged to it; W, v^i and the comoving field follow from the vertex metric, T^{mu nu}
// is formed as in the source terms, and both indices are lowered with the 4-metric,
// T_{mu nu} = g_{mu a} g_{nu b} T^{ab}.  Components in the order tt, tx, ty, tz, xx, xy, xz, yy, yz, zz.

static void tmunu_vertices(const Grid& G, const VertexMetric& vm, const OParams& P, double* const U[9],
                           double* const prim[5], double* const Tout[10]) {
  std::vector<double> Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  const int g = G.g;
  for (int k = g; k <= g + G.n[2]; k++)
    for (int j = g; j <= g + G.n[1]; j++)
      for (int i = g; i <= g + G.n[0]; i++) {
        double rho = 0.0, press = 0.0, u[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
        for (int ck = k - 1; ck <= k; ck++)
          for (int cj = j - 1; cj <= j; cj++)
            for (int ci = i - 1; ci <= i; ci++) {
              const long c = G.at(ci, cj, ck);
              const Metric3<double> mc = metric_at_centre(G, vm, ci, cj, ck);
              double v2 = 0.0;
              for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) v2 += mc.g[a][b] * prim[2 + a][c] * prim[2 + b][c];
              const double Wc = 1.0 / std::sqrt(1.0 - v2);
              rho += prim[0][c];
              press += prim[1][c];
              for (int a = 0; a < 3; a++) {
                u[a] += Wc * prim[2 + a][c];
                B[a] += Bc[a][c];
              }
            }
        rho /= 8.0;
        press /= 8.0;
        for (int a = 0; a < 3; a++) {
          u[a] /= 8.0;
          B[a] /= 8.0;
        }
        const Metric3<double> m = metric_at_vertex(G, vm, i, j, k);
        double u2 = 0.0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) u2 += m.g[a][b] * u[a] * u[b];
        const double W = std::sqrt(1.0 + u2);
        Prim<double> pr;
        pr.rho = rho;
        pr.press = press;
        pr.eps = press / ((P.gamma - 1.0) * rho);
        for (int a = 0; a < 3; a++) {
          pr.vel[a] = u[a] / W;
          pr.B[a] = B[a];
        }
        const Comoving<double> cm = comoving(m, pr);
        double u4[4], b4[4];
        u4[0] = cm.u0;
        b4[0] = cm.b0;
        for (int a = 0; a < 3; a++) {
          u4[a + 1] = cm.uup[a];
          b4[a + 1] = cm.bup[a];
        }
        const double a2 = m.alp * m.alp;
        double guu[4][4], gdd[4][4];  // inverse and covariant 4-metric
        guu[0][0] = -1.0 / a2;
        double betalow[3];
        for (int a = 0; a < 3; a++) betalow[a] = m.g[a][0] * m.beta[0] + m.g[a][1] * m.beta[1] + m.g[a][2] * m.beta[2];
        gdd[0][0] = -a2 + betalow[0] * m.beta[0] + betalow[1] * m.beta[1] + betalow[2] * m.beta[2];
        for (int a = 0; a < 3; a++) {
          guu[0][a + 1] = guu[a + 1][0] = m.beta[a] / a2;
          gdd[0][a + 1] = gdd[a + 1][0] = betalow[a];
          for (int b = 0; b < 3; b++) {
            guu[a + 1][b + 1] = m.gu[a][b] - m.beta[a] * m.beta[b] / a2;
            gdd[a + 1][b + 1] = m.g[a][b];
          }
        }
        const double rhohb = pr.rho * cm.h + cm.b2;
        const double ptot = pr.press + 0.5 * cm.b2;
        double Tup[4][4];
        for (int mu = 0; mu < 4; mu++)
          for (int nu = 0; nu < 4; nu++) Tup[mu][nu] = rhohb * u4[mu] * u4[nu] + ptot * guu[mu][nu] - b4[mu] * b4[nu];
        static const int IDX[10][2] = {{0, 0}, {0, 1}, {0, 2}, {0, 3}, {1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};
        const long v = G.at(i, j, k);
        for (int q = 0; q < 10; q++) {
          const int mu = IDX[q][0], nu = IDX[q][1];
          double t = 0.0;
          for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) t += gdd[mu][a] * gdd[nu][b] * Tup[a][b];
          Tout[q][v] = t;
        }
      }
}

// ------------------------------------------------------------------------------------------------------
// Two refinement levels (the BoxInBox fixed refinement of Sec. 3; prolongation at the inner refinement boundary
// as the magnetic-rotor AMR test describes it): a fine block of half the spacing whose interior covers the
// coarse cells L .. L+m-1 along each axis (m = n_fine / 2).  The fine ghost layers are prolonged from the coarse
// level; after a step the coarse points under the fine interior are restricted from it.
//
// Prolongation, axis by axis in the order x, y, z: where the variable is cell-centred along the axis, third-order
// conservative: the parabola through three coarse cell averages averaged over the fine half,
// u_I -/+ (u_{I+1} - u_{I-1}) / 8, with the linear fallback u_I -/+ minmod(u_I - u_{I-1}, u_{I+1} - u_I) / 4
// for both halves where either parabola value would leave the range of the three averages (a discontinuity or
// an extremum; deciding per coarse cell keeps the halves' mean at u_I); where it is
// vertex-centred, a fine point on a coarse point copies it and a midpoint takes the cubic through four coarse
// points, (-u_{J-1} + 9 u_J + 9 u_{J+1} - u_{J+2}) / 16.  Restriction: the mean of the fine points covering a
// coarse point (two halves along a cell-centred axis, the coincident point along a vertex-centred one).

static int floor_div2(int f) { return (f >= 0) ? f / 2 : -((-f + 1) / 2); }

template <class Get> static double prolong_1d(bool cell, int f, const Get& get) {
  if (cell) {
    const int I = floor_div2(f);
    const bool right = (f - 2 * I) == 1;
    const double um = get(I - 1), u0 = get(I), up = get(I + 1);
    const double d = (up - um) / 8.0;
    const double lo = std::min(um, std::min(u0, up)), hi = std::max(um, std::max(u0, up));
    // the decision is the coarse cell's, for both halves, so that their mean stays u0
    if (u0 - d < lo || u0 - d > hi || u0 + d < lo || u0 + d > hi) {
      const double a = u0 - um, b = up - u0;
      const double s = (a * b <= 0.0) ? 0.0 : (std::fabs(a) <= std::fabs(b) ? a : b);
      return right ? u0 + 0.25 * s : u0 - 0.25 * s;
    }
    return right ? u0 + d : u0 - d;
  }
  if ((f & 1) == 0) return get(f / 2);
  const int J = floor_div2(f - 1);
  return (-get(J - 1) + 9.0 * get(J) + 9.0 * get(J + 1) - get(J + 2)) / 16.0;
}

// value at the fine point of interior-relative index fr (fine units) of a field with staggering cl from the
// coarse array uc (coarse interior-relative index of the box corner L)
static double prolong_point(const Grid& C, const double* uc, const int L[3], const int cl[3], const int fr[3]) {
  auto coarse = [&](int qx, int qy, int qz) { return uc[C.at(C.g + L[0] + qx, C.g + L[1] + qy, C.g + L[2] + qz)]; };
  auto along_z = [&](int qz) {
    auto along_y = [&](int qy) {
      auto along_x = [&](int qx) { return coarse(qx, qy, qz); };
      return prolong_1d(cl[0], fr[0], along_x);
    };
    return prolong_1d(cl[1], fr[1], along_y);
  };
  return prolong_1d(cl[2], fr[2], along_z);
}

static const int PRIM_CELL_LIKE[3] = {1, 1, 1};

// fills the fine block's ghost points (outside the owned ranges, copy-BC convention) of the 9 state fields and
// the 5 primitives; with all != 0 every point of the fine padded array
static void prolong_grid(const Grid& C, const Grid& F, const int L[3], double* const Uc[9], double* const Pc[5],
                         double* const Uf[9], double* const Pf[5], bool all) {
  for (int k = 0; k <= F.N[2]; k++)
    for (int j = 0; j <= F.N[1]; j++)
      for (int i = 0; i <= F.N[0]; i++) {
        const int p[3] = {i, j, k};
        const int fr[3] = {i - F.g, j - F.g, k - F.g};
        const long c = F.at(p);
        for (int v = 0; v < 14; v++) {
          const int* cl = v < 9 ? STATE_CELL_LIKE[v] : PRIM_CELL_LIKE;
          bool owned = true, inside = true;
          for (int a = 0; a < 3; a++) {
            const int hi = cl[a] ? F.g + F.n[a] - 1 : F.g + F.n[a];
            owned = owned && p[a] >= F.g && p[a] <= hi;
            inside = inside && p[a] < F.N[a] + (cl[a] ? 0 : 1);  // cell-like axes end at N-1
          }
          if ((owned && !all) || !inside) continue;
          const double* src = v < 9 ? Uc[v] : Pc[v - 9];
          double* dst = v < 9 ? Uf[v] : Pf[v - 9];
          dst[c] = prolong_point(C, src, L, cl, fr);
        }
      }
}

// coarse points covered by the fine interior, from the fine state (9 fields)
static void restrict_grid(const Grid& C, const Grid& F, const int L[3], double* const Uc[9], double* const Uf[9]) {
  const int m[3] = {F.n[0] / 2, F.n[1] / 2, F.n[2] / 2};
  for (int v = 0; v < 9; v++) {
    const int* cl = STATE_CELL_LIKE[v];
    int hi[3];
    for (int a = 0; a < 3; a++) hi[a] = cl[a] ? m[a] - 1 : m[a];
    for (int qz = 0; qz <= hi[2]; qz++)
      for (int qy = 0; qy <= hi[1]; qy++)
        for (int qx = 0; qx <= hi[0]; qx++) {
          const int q[3] = {qx, qy, qz};
          double sum = 0.0;
          int cnt = 0;
          for (int dz = 0; dz <= cl[2]; dz++)
            for (int dy = 0; dy <= cl[1]; dy++)
              for (int dx = 0; dx <= cl[0]; dx++) {
                sum += Uf[v][F.at(F.g + 2 * q[0] + dx, F.g + 2 * q[1] + dy, F.g + 2 * q[2] + dz)];
                cnt++;
              }
          Uc[v][C.at(C.g + L[0] + q[0], C.g + L[1] + q[1], C.g + L[2] + q[2])] = sum / cnt;
        }
  }
}

// ------------------------------------------------------------------------------------------------------
// Jacobian-vector products of the stage operator L(U) = RHS(ghost fill, recovery, primitive ghost fill) and
// of one RK4 step, in the direction dU, by the one-direction dual number.  The recovery keeps its values from
// c2p_cell (the recovery above, as it stands) and takes its derivative from the implicit-function theorem:
// one Noble Newton step in dual arithmetic from the converged root (z, v^2), whose value change is ~0 and
// whose derivative is -J^{-1} (df / dinputs) (the Palenzuela root satisfies the same two equations).  Cells
// set to the atmosphere keep constant primitives; their conserved variables are reset as con2prim does.

static void con2prim_jvp(const Grid& G, const VertexMetric& vm, const OParams& P, Dual1* const U[9],
                         Dual1* const prim[5], signed char* flags) {
  std::vector<Dual1> Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  const int g = G.g;
  for (int k = g; k < g + G.n[2]; k++)
    for (int j = g; j < g + G.n[1]; j++)
      for (int i = g; i < g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        C2PIn in;
        in.Dtilde = U[0][c].v;
        in.D = U[0][c].v / m.sqrtg;
        for (int a = 0; a < 3; a++) in.S[a] = U[1 + a][c].v / m.sqrtg;
        in.tau = U[4][c].v / m.sqrtg;
        for (int a = 0; a < 3; a++) in.B[a] = Bc[a][c].v;
        in.guess_rho = prim[0][c].v;
        in.guess_press = prim[1][c].v;
        for (int a = 0; a < 3; a++) in.guess_vel[a] = prim[2 + a][c].v;
        const C2POut o = c2p_cell(m, in, P);
        if (flags) flags[c] = (signed char)o.flag;
        double dr = 0.0, dp = 0.0, dv[3] = {0.0, 0.0, 0.0};
        if (o.flag == 0 || o.flag == 1) {
          const Dual1 sg(m.sqrtg);
          const Dual1 D = U[0][c] / sg, tau = U[4][c] / sg;
          Dual1 S[3], B[3];
          for (int a = 0; a < 3; a++) {
            S[a] = U[1 + a][c] / sg;
            B[a] = Bc[a][c];
          }
          Dual1 S2(0.0), B2(0.0), BS(0.0);
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
              S2 += Dual1(m.gu[a][b]) * S[a] * S[b];
              B2 += Dual1(m.g[a][b]) * B[a] * B[b];
            }
          for (int a = 0; a < 3; a++) BS += B[a] * S[a];
          // the root from the recovered primitives: z = rho h W^2, v^2
          double v2 = 0.0;
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) v2 += m.g[a][b] * o.vel[a] * o.vel[b];
          const double W = 1.0 / std::sqrt(1.0 - v2);
          const double eps = o.press / ((P.gamma - 1.0) * o.rho);
          const double z = o.rho * (1.0 + eps + o.press / o.rho) * W * W;
          Dual1 f[2], J[2][2];
          noble_residual<Dual1>(Dual1(z), Dual1(v2), D, tau, S2, B2, BS, P.gamma, f, J);
          const Dual1 det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
          const Dual1 zd = Dual1(z) + (-f[0] * J[1][1] + J[0][1] * f[1]) / det;
          const Dual1 v2d = Dual1(v2) + (-J[0][0] * f[1] + J[1][0] * f[0]) / det;
          const Dual1 Wd = Dual1(1.0) / sqrt(Dual1(1.0) - v2d);
          const Dual1 rhod = D / Wd;
          const Dual1 epsd = (zd / (rhod * Wd * Wd) - Dual1(1.0)) / Dual1(P.gamma);
          const Dual1 pd = Dual1(P.gamma - 1.0) * rhod * epsd;
          dr = rhod.d;
          dp = pd.d;
          for (int a = 0; a < 3; a++) {  // Eq. (Noble2D v)
            Dual1 Su(0.0);
            for (int b = 0; b < 3; b++) Su += Dual1(m.gu[a][b]) * S[b];
            dv[a] = (Su / (zd + B2) + BS * B[a] / (zd * (zd + B2))).d;
          }
        }
        prim[0][c] = Dual1(o.rho, dr);
        prim[1][c] = Dual1(o.press, dp);
        for (int a = 0; a < 3; a++) prim[2 + a][c] = Dual1(o.vel[a], dv[a]);
        if (o.reset) {  // as con2prim: conserved variables from the atmosphere primitives, B kept (Sec. 3.6)
          Prim<Dual1> pr;
          pr.rho = Dual1(o.rho);
          pr.press = Dual1(o.press);
          pr.eps = Dual1(o.press / ((P.gamma_atm - 1.0) * o.rho));
          for (int a = 0; a < 3; a++) {
            pr.vel[a] = Dual1(0.0);
            pr.B[a] = Bc[a][c];
          }
          const Metric3<Dual1> md = lift<Dual1>(m);
          const Cons<Dual1> uc = prim2con(md, pr, comoving(md, pr));
          U[0][c] = uc.D;
          for (int a = 0; a < 3; a++) U[1 + a][c] = uc.S[a];
          U[4][c] = uc.tau;
        }
      }
}

typedef std::vector<std::vector<Dual1>> DualFields;

static DualFields dual_fields(int n, long size) { return DualFields(n, std::vector<Dual1>(size)); }

template <int N> static void ptrs_of(DualFields& f, Dual1* out[N]) {
  for (int v = 0; v < N; v++) out[v] = f[v].data();
}

// k = L(Y) with its derivative (Y: 9 dual fields, ghosts filled here; prim: 5 dual fields, guess in, out)
static void stage_rhs_jvp(const Grid& G, const VertexMetric& vm, const OParams& P, double dt, Dual1* const Y[9],
                          Dual1* const prim[5], Dual1* const k[9]) {
  ghost_fill_state(G, Y);
  con2prim_jvp(G, vm, P, Y, prim, nullptr);
  ghost_fill_prims(G, prim);
  for (int v = 0; v < 9; v++)
    for (long c = 0; c < G.size(); c++) k[v][c] = Dual1(0.0);
  rhs(G, vm, P, dt, Y, prim, k, (RhsStats*)nullptr);
}

}  // namespace asterx_oracle

// ------------------------------------------------------------------------------------------------------
// C entry points for the test suite (ctypes).

using namespace asterx_oracle;

static VertexMetric vmetric(const double* const* m) {
  VertexMetric vm;
  for (int a = 0; a < 16; a++) vm.f[a] = m[a];
  return vm;
}

extern "C" {

int oracle_abi_version(void) { return 1; }

// Threads of the OpenMP loops (1 = serial); returns the count in effect.
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void oracle_ghost_fill_state(const OBlock* b, double* const* U) {
  Grid G(*b);
  ghost_fill_state(G, U);
}

void oracle_ghost_fill_prims(const OBlock* b, double* const* P) {
  Grid G(*b);
  ghost_fill_prims(G, P);
}

void oracle_prim2con(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                     double* const* prim) {
  Grid G(*b);
  prim2con_grid(G, vmetric(metric), *p, U, prim);
}

// The conserved fields (D, S, tau) from the potentials and primitives and their derivative in the direction
// (dA, dprim): U[0..4] and JU[0..4] receive value and derivative; U[5..7] are read (A), dA the potentials'
// direction (3 fields), prim and dprim the primitives and their direction.
void oracle_prim2con_jvp(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                         const double* const* dA, const double* const* prim, const double* const* dprim,
                         double* const* JU) {
  Grid G(*b);
  DualFields Ad = dual_fields(3, G.size()), Pd = dual_fields(5, G.size()), Ud = dual_fields(5, G.size());
  for (int v = 0; v < 3; v++)
    for (long c = 0; c < G.size(); c++) Ad[v][c] = Dual1(U[5 + v][c], dA[v][c]);
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) {
      Pd[v][c] = Dual1(prim[v][c], dprim[v][c]);
      Ud[v][c] = Dual1(U[v][c]);  // entries outside the cells keep their values (and no derivative)
    }
  const Dual1* Ap[3] = {Ad[0].data(), Ad[1].data(), Ad[2].data()};
  const Dual1* Pp[5] = {Pd[0].data(), Pd[1].data(), Pd[2].data(), Pd[3].data(), Pd[4].data()};
  Dual1* Up[5] = {Ud[0].data(), Ud[1].data(), Ud[2].data(), Ud[3].data(), Ud[4].data()};
  prim2con_fields<Dual1>(G, vmetric(metric), *p, Ap, Pp, Up);
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) {
      U[v][c] = Ud[v][c].v;
      JU[v][c] = Ud[v][c].d;
    }
}

void oracle_con2prim(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                     double* const* prim, signed char* flags, OStats* stats) {
  Grid G(*b);
  con2prim(G, vmetric(metric), *p, U, prim, flags, stats);
}

void oracle_rhs(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                double* const* prim, double* const* dU, double dt, unsigned long long* speed_iters) {
  Grid G(*b);
  RhsStats st{0, 0};
  rhs(G, vmetric(metric), *p, dt, U, prim, dU, &st);
  if (speed_iters) {
    speed_iters[0] = st.speed_iters;
    speed_iters[1] = st.faces;
  }
}

void oracle_face_B(const OBlock* b, double* const* U, double* const* Bf) {
  Grid G(*b);
  Field f[3];
  face_B(G, U[5], U[6], U[7], f);
  for (int d = 0; d < 3; d++) std::memcpy(Bf[d], f[d].data(), sizeof(double) * G.size());
}

void oracle_rk_stage(const OParams* p, const OBlock* b, const double* const* metric, int stage, double dt,
                     double* const* Un, double* const* Us, double* const* Unext, double* const* Uacc,
                     double* const* prim, signed char* flags, OStats* stats) {
  Grid G(*b);
  rk_stage(G, vmetric(metric), *p, stage, dt, Un, Us, Unext, Uacc, prim, flags, stats);
}

// As oracle_rk_stage, with the ghost layers of U_s and of the primitives taken as given (a refined block whose
// ghosts were prolonged from the coarse level).
void oracle_rk_stage_given_ghosts(const OParams* p, const OBlock* b, const double* const* metric, int stage,
                                  double dt, double* const* Un, double* const* Us, double* const* Unext,
                                  double* const* Uacc, double* const* prim, signed char* flags, OStats* stats) {
  Grid G(*b);
  rk_stage(G, vmetric(metric), *p, stage, dt, Un, Us, Unext, Uacc, prim, flags, stats, false);
}

// Prolongation from a coarse block to the ghost points (all != 0: every point) of a nested fine block whose
// interior starts at coarse interior cell L (state 9 fields, primitives 5 fields on each level).
void oracle_prolong(const OBlock* coarse, const OBlock* fine, const int* L, double* const* Uc, double* const* Pc,
                    double* const* Uf, double* const* Pf, int all) {
  Grid C(*coarse), F(*fine);
  prolong_grid(C, F, L, Uc, Pc, Uf, Pf, all != 0);
}

// Restriction of the fine interior's state to the coarse points it covers.
void oracle_restrict(const OBlock* coarse, const OBlock* fine, const int* L, double* const* Uc,
                     double* const* Uf) {
  Grid C(*coarse), F(*fine);
  restrict_grid(C, F, L, Uc, Uf);
}

// The interpolated metric (Sec. 3.2) at every cell centre of the padded block, for checks of precomputed
// geometry elsewhere: 53 fields, alpha, beta^i (3), gamma_ij (6: xx, xy, xz, yy, yz, zz), gamma^ij (6),
// sqrt(gamma), K_ij (6), d_i alpha (3), d_i beta^j (9, index 3 i + j), d_i gamma_jk (18, index 6 i + jk).
void oracle_centre_metric(const OBlock* b, const double* const* metric, double* const* out) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  for (int k = 0; k < G.N[2]; k++)
    for (int j = 0; j < G.N[1]; j++)
      for (int i = 0; i < G.N[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        const MetricDeriv<double> dm = metric_deriv_at_centre(G, vm, i, j, k);
        int q = 0;
        out[q++][c] = m.alp;
        for (int a = 0; a < 3; a++) out[q++][c] = m.beta[a];
        for (int a = 0; a < 3; a++)
          for (int e = a; e < 3; e++) out[q++][c] = m.g[a][e];
        for (int a = 0; a < 3; a++)
          for (int e = a; e < 3; e++) out[q++][c] = m.gu[a][e];
        out[q++][c] = m.sqrtg;
        for (int a = 0; a < 3; a++)
          for (int e = a; e < 3; e++) out[q++][c] = m.K[a][e];
        for (int d = 0; d < 3; d++) out[q++][c] = dm.dalp[d];
        for (int d = 0; d < 3; d++)
          for (int a = 0; a < 3; a++) out[q++][c] = dm.dbeta[d][a];
        for (int d = 0; d < 3; d++)
          for (int a = 0; a < 3; a++)
            for (int e = a; e < 3; e++) out[q++][c] = dm.dg[d][a][e];
      }
}

// The interpolated metric at the faces normal to d (index 0..N along d, cells across): 17 fields, alpha,
// beta^i (3), gamma_ij (6), gamma^ij (6), sqrt(gamma).
void oracle_face_metric(const OBlock* b, const double* const* metric, int d, double* const* out) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  int hi[3] = {G.N[0] - 1, G.N[1] - 1, G.N[2] - 1};
  hi[d] = G.N[d];
  for (int k = 0; k <= hi[2]; k++)
    for (int j = 0; j <= hi[1]; j++)
      for (int i = 0; i <= hi[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_face(G, vm, d, i, j, k);
        int q = 0;
        out[q++][c] = m.alp;
        for (int a = 0; a < 3; a++) out[q++][c] = m.beta[a];
        for (int a = 0; a < 3; a++)
          for (int e = a; e < 3; e++) out[q++][c] = m.g[a][e];
        for (int a = 0; a < 3; a++)
          for (int e = a; e < 3; e++) out[q++][c] = m.gu[a][e];
        out[q++][c] = m.sqrtg;
      }
}

// T_{mu nu} at the vertices g..g+n of every axis (U's A and the primitives ghost-filled); 10 output fields.
void oracle_tmunu(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                  double* const* prim, double* const* T) {
  Grid G(*b);
  tmunu_vertices(G, vmetric(metric), *p, U, prim, T);
}

// L(U) and its derivative in direction dir (9 fields each; U's ghosts are filled on a copy).  prim: the
// recovery's guess in, the recovered primitives out.
void oracle_stage_jvp(const OParams* p, const OBlock* b, const double* const* metric, const double* const* U,
                      const double* const* dir, double* const* prim, double* const* L, double* const* JL,
                      double dt) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  DualFields Y = dual_fields(9, G.size()), Pd = dual_fields(5, G.size()), k = dual_fields(9, G.size());
  for (int v = 0; v < 9; v++)
    for (long c = 0; c < G.size(); c++) Y[v][c] = Dual1(U[v][c], dir[v][c]);
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) Pd[v][c] = Dual1(prim[v][c]);
  Dual1 *Yp[9], *Pp[5], *kp[9];
  ptrs_of<9>(Y, Yp);
  ptrs_of<5>(Pd, Pp);
  ptrs_of<9>(k, kp);
  stage_rhs_jvp(G, vm, *p, dt, Yp, Pp, kp);
  for (int v = 0; v < 9; v++)
    for (long c = 0; c < G.size(); c++) {
      L[v][c] = k[v][c].v;
      JL[v][c] = k[v][c].d;
    }
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) prim[v][c] = Pd[v][c].v;
}

// One classical RK4 step of U (9 fields, ghosts filled) and its derivative in direction dir: U1, JU1 on the
// owned ranges (the stages as oracle_rk_stage forms them).  prim: guess in, last recovery out.
void oracle_rk4_jvp(const OParams* p, const OBlock* b, const double* const* metric, const double* const* U,
                    const double* const* dir, double* const* prim, double* const* U1, double* const* JU1,
                    double dt) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  DualFields Un = dual_fields(9, G.size()), Ys = dual_fields(9, G.size()), acc = dual_fields(9, G.size());
  DualFields k = dual_fields(9, G.size()), Pd = dual_fields(5, G.size());
  for (int v = 0; v < 9; v++)
    for (long c = 0; c < G.size(); c++) Un[v][c] = Dual1(U[v][c], dir[v][c]);
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) Pd[v][c] = Dual1(prim[v][c]);
  Ys = Un;
  Dual1 *Ysp[9], *Pp[5], *kp[9];
  ptrs_of<5>(Pd, Pp);
  ptrs_of<9>(k, kp);
  static const double cnext[3] = {0.5, 0.5, 1.0};
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  for (int stage = 0; stage < 4; stage++) {
    DualFields next = Ys;  // entries outside the owned ranges keep the stage state's values
    ptrs_of<9>(Ys, Ysp);
    stage_rhs_jvp(G, vm, *p, dt, Ysp, Pp, kp);
    if (stage == 0) Un = Ys;  // the first stage fills U_n's ghosts (and U_s = U_n)
    for (int v = 0; v < 9; v++) {
      int lo[3], hi[3];
      owned_range(G, v, lo, hi);
      for (int kk = lo[2]; kk <= hi[2]; kk++)
        for (int j = lo[1]; j <= hi[1]; j++)
          for (int i = lo[0]; i <= hi[0]; i++) {
            const long c = G.at(i, j, kk);
            const Dual1 kv = k[v][c];
            if (stage == 0) {
              acc[v][c] = Dual1(bw[0] * dt) * kv;
              next[v][c] = Un[v][c] + Dual1(cnext[0] * dt) * kv;
            } else if (stage < 3) {
              acc[v][c] = acc[v][c] + Dual1(bw[stage] * dt) * kv;
              next[v][c] = Un[v][c] + Dual1(cnext[stage] * dt) * kv;
            } else {
              next[v][c] = Un[v][c] + acc[v][c] + Dual1(bw[3] * dt) * kv;
            }
          }
    }
    Ys = next;
  }
  for (int v = 0; v < 9; v++)
    for (long c = 0; c < G.size(); c++) {
      U1[v][c] = Ys[v][c].v;
      JU1[v][c] = Ys[v][c].d;
    }
  for (int v = 0; v < 5; v++)
    for (long c = 0; c < G.size(); c++) prim[v][c] = Pd[v][c].v;
}

// Algorithmic flop count of the face solve (Sec. 3.3: prim->cons, fluxes, magnetosonic speeds, HLLE and the
// upwind velocities of Eq. uct1) along direction d, over every `stride`-th face of the face domain
// (faces g..g+n along d, all transverse indices), with the flop-counting scalar.  Interpolation of the frozen
// metric is not counted (the face metric is an input of the face solve).  out: faces, add, mul, div, sqrt,
// speed iterations.  U and prim must hold ghost-filled state and recovered, ghost-filled primitives.
void oracle_face_flops(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                       double* const* prim, int d, int stride, double* out) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  Field Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  Field cellvar[8];
  for (int v = 0; v < 8; v++) cellvar[v].assign(G.size(), 0.0);
  for (int k = 0; k < G.N[2]; k++)
    for (int j = 0; j < G.N[1]; j++)
      for (int i = 0; i < G.N[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        double v2 = 0.0;
        for (int a = 0; a < 3; a++)
          for (int q = 0; q < 3; q++) v2 += m.g[a][q] * prim[2 + a][c] * prim[2 + q][c];
        const double W = 1.0 / std::sqrt(1.0 - v2);
        cellvar[0][c] = prim[0][c];
        cellvar[1][c] = prim[1][c];
        for (int a = 0; a < 3; a++) cellvar[2 + a][c] = W * prim[2 + a][c];
        for (int a = 0; a < 3; a++) cellvar[5 + a][c] = Bc[a][c];
      }
  const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
  double faces = 0, iters = 0;
  Flops before = g_flops;
  long counter = 0;
  for (int q2 = 0; q2 < G.N[a2]; q2++)
    for (int q1 = 0; q1 < G.N[a1]; q1++)
      for (int f = G.g; f <= G.g + G.n[d]; f++) {
        if ((counter++ % stride) != 0) continue;
        int pp[3];
        pp[d] = f;
        pp[a1] = q1;
        pp[a2] = q2;
        FaceInput in;
        for (int sd = 0; sd < 2; sd++) {
          const int cell = f - 1 + sd;
          double rec[8];
          for (int v = 0; v < 8; v++) {
            double st5[5];
            for (int t = 0; t < 5; t++) {
              int q[3] = {pp[0], pp[1], pp[2]};
              q[d] = cell - 2 + t;
              st5[t] = cellvar[v][G.at(q)];
            }
            double aL, aR;
            recon_cell<double>(p->recon, st5, &aL, &aR);
            rec[v] = (sd == 0) ? aR : aL;
          }
          in.rho[sd] = rec[0];
          in.press[sd] = rec[1];
          for (int a = 0; a < 3; a++) in.u[sd][a] = rec[2 + a];
          for (int a = 0; a < 3; a++) in.Bt[sd][a] = rec[5 + a];
        }
        in.Bn = Bf[d][G.at(pp)];
        const Metric3<double> md = metric_at_face(G, vm, d, pp[0], pp[1], pp[2]);
        Metric3<Fc> mf;
        mf.alp = Fc(md.alp);
        mf.sqrtg = Fc(md.sqrtg);
        for (int a = 0; a < 3; a++) {
          mf.beta[a] = Fc(md.beta[a]);
          for (int q = 0; q < 3; q++) {
            mf.g[a][q] = Fc(md.g[a][q]);
            mf.gu[a][q] = Fc(md.gu[a][q]);
            mf.K[a][q] = Fc(md.K[a][q]);
          }
        }
        FaceInputT<Fc> fin;  // the reconstructed states are data
        for (int sd = 0; sd < 2; sd++) {
          fin.rho[sd] = fc_data(in.rho[sd]);
          fin.press[sd] = fc_data(in.press[sd]);
          for (int a = 0; a < 3; a++) {
            fin.u[sd][a] = fc_data(in.u[sd][a]);
            fin.Bt[sd][a] = fc_data(in.Bt[sd][a]);
          }
        }
        fin.Bn = fc_data(in.Bn);
        FaceOut<Fc> o = face_solve<Fc>(mf, fin, p->gamma, d);
        faces += 1;
        iters += o.iters;
      }
  out[0] = faces;
  out[1] = (double)(g_flops.add - before.add);
  out[2] = (double)(g_flops.mul - before.mul);
  out[3] = (double)(g_flops.div - before.div);
  out[4] = (double)(g_flops.sqrt - before.sqrt);
  out[5] = iters;
}

// Algorithmic flop count of the per-cell reconstruction of the 7 face variables (one cell, both faces).
void oracle_recon_flops(int scheme, const double* a5, double* out) {
  Flops before = g_flops;
  Fc a[5];
  for (int t = 0; t < 5; t++) a[t] = fc_data(a5[t]);
  Fc lo, hi;
  recon_cell<Fc>(scheme, a, &lo, &hi);
  out[0] = (double)(g_flops.add - before.add);
  out[1] = (double)(g_flops.mul - before.mul);
  out[2] = (double)(g_flops.div - before.div);
  out[3] = (double)(g_flops.sqrt - before.sqrt);
}

// Algorithmic flop count of one RK stage (Sec. 3.12 workflow) with the flop-counting scalar, part by part:
// ghost fill of the state (linear extrapolation of A), recovery over the interior cells (face and centre field,
// undensitisation, Noble / Palenzuela / atmosphere reset), ghost fill of the primitives, the right-hand side
// (faces: u = W v, reconstruction and face solve of the three directions; cells: flux divergence and sources;
// potentials at vertices; edge fields and dA/dt; dPsi/dt) and the RK4 combine of stage `stage` (0..3) over the
// owned entries.  Interpolation of the frozen metric is not counted (an input of every step).  U is the stage
// state (its ghosts are filled here, on a copy), prim the recovery's guess.  out (60 values): [0] interior
// cells; then (add, mul, div, sqrt) of: [1] state ghost fill, [5] recovery, [9] primitive ghost fill, [13]
// faces, [17] cells, [21] potentials, [25] edges, [29] Psi, [33] combine, [45] the right-hand side's own
// recomputation of the face and centre field (the recovery's are reused by an implementation, so it is
// reported apart); [37] speed iterations, [38] faces solved, [39] flops inside the speed Newton loops, [40]
// Noble iterations, [41..44] cells recovered by Noble / Palenzuela / atmosphere / both failed; flops (all
// kinds) of [49] u = W v as the faces part forms it (once per direction), [50] the reconstruction as the faces
// part forms it (twice per cell), [51] the face solves, [52] the edge fields' PPM interfaces (twice per face
// value), [53] the recovery's face and centre field; [54..59] unused.
void oracle_stage_flops(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                        double* const* prim, int stage, double dt, double* out) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  for (int q = 0; q < 60; q++) out[q] = 0.0;
  g_cellvar_flops = g_recon_flops = g_facesolve_flops = g_edge_ppm_flops = 0;
  std::vector<Fc> Uv[9], Pv[5], kv[9];
  Fc *Up[9], *Pp[5], *kp[9];
  for (int v = 0; v < 9; v++) {
    Uv[v].resize(G.size());
    kv[v].assign(G.size(), Fc(0.0));
    for (long c = 0; c < G.size(); c++) Uv[v][c] = fc_data(U[v][c]);
    Up[v] = Uv[v].data();
    kp[v] = kv[v].data();
  }
  for (int v = 0; v < 5; v++) {
    Pv[v].resize(G.size());
    for (long c = 0; c < G.size(); c++) Pv[v][c] = fc_data(prim[v][c]);
    Pp[v] = Pv[v].data();
  }
  auto put = [&](int at, const Flops& a, const Flops& z) {
    out[at] = (double)(z.add - a.add);
    out[at + 1] = (double)(z.mul - a.mul);
    out[at + 2] = (double)(z.div - a.div);
    out[at + 3] = (double)(z.sqrt - a.sqrt);
  };
  Flops f0 = g_flops;
  ghost_fill_state<Fc>(G, Up);
  Flops f1 = g_flops;
  put(1, f0, f1);
  // recovery, as con2prim does it, in the counting scalar
  std::vector<Fc> Bf[3], Bc[3];
  face_B<Fc>(G, Up[5], Up[6], Up[7], Bf);
  centre_B<Fc>(G, vm, Bf, Bc);
  out[53] = (double)(flops_total(g_flops) - flops_total(f1));
  const int g = G.g;
  double iters = 0, nflag[4] = {0, 0, 0, 0};
  for (int k = g; k < g + G.n[2]; k++)
    for (int j = g; j < g + G.n[1]; j++)
      for (int i = g; i < g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<Fc> m = lift<Fc>(metric_at_centre(G, vm, i, j, k));
        C2PIn in;
        in.Dtilde = Up[0][c].v;
        in.D = (Up[0][c] / m.sqrtg).v;
        for (int a = 0; a < 3; a++) in.S[a] = (Up[1 + a][c] / m.sqrtg).v;
        in.tau = (Up[4][c] / m.sqrtg).v;
        for (int a = 0; a < 3; a++) in.B[a] = Bc[a][c].v;
        in.guess_rho = Pp[0][c].v;
        in.guess_press = Pp[1][c].v;
        for (int a = 0; a < 3; a++) in.guess_vel[a] = Pp[2 + a][c].v;
        C2POut o = c2p_cell<Fc>(m, in, *p);
        iters += o.iters;
        nflag[o.flag == 0 ? 0 : o.flag == 1 ? 1 : o.flag == 2 ? 2 : 3] += 1;
        Pp[0][c] = fc_data(o.rho);
        Pp[1][c] = fc_data(o.press);
        for (int a = 0; a < 3; a++) Pp[2 + a][c] = fc_data(o.vel[a]);
        if (o.reset) {
          Prim<Fc> pr;
          pr.rho = Fc(o.rho);
          pr.press = Fc(o.press);
          pr.eps = pr.press / (Fc(p->gamma_atm - 1.0) * pr.rho);
          for (int a = 0; a < 3; a++) {
            pr.vel[a] = Fc(0.0);
            pr.B[a] = Bc[a][c];
          }
          Comoving<Fc> cm = comoving(m, pr);
          Cons<Fc> uc = prim2con(m, pr, cm);
          Up[0][c] = uc.D;
          for (int a = 0; a < 3; a++) Up[1 + a][c] = uc.S[a];
          Up[4][c] = uc.tau;
        }
      }
  Flops f2 = g_flops;
  put(5, f1, f2);
  ghost_fill_prims<Fc>(G, Pp);
  Flops f3 = g_flops;
  put(9, f2, f3);
  // right-hand side, phase by phase
  Flops marks[5];
  g_rhs_marks = marks;
  const unsigned long long loop0 = g_speed_loop_flops;
  RhsStats st = {0, 0};
  rhs<Fc>(G, vm, *p, dt, Up, Pp, kp, &st);
  g_rhs_marks = nullptr;
  Flops f4 = g_flops;
  put(45, f3, marks[0]);
  put(13, marks[0], marks[1]);
  put(17, marks[1], marks[2]);
  put(21, marks[2], marks[3]);
  put(25, marks[3], marks[4]);
  put(29, marks[4], f4);
  // RK4 combine of this stage over the owned entries (as rk_stage forms it)
  static const double cnext[3] = {0.5, 0.5, 1.0};
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  for (int v = 0; v < 9; v++) {
    int lo[3], hi[3];
    owned_range(G, v, lo, hi);
    for (int kk = lo[2]; kk <= hi[2]; kk++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          const long c = G.at(i, j, kk);
          const Fc k1 = kp[v][c], un = Up[v][c];
          Fc acc = Fc(0.0), next;
          if (stage == 0) {
            acc = Fc(bw[0]) * Fc(dt) * k1;
            next = un + Fc(cnext[0]) * Fc(dt) * k1;
          } else if (stage < 3) {
            acc = acc + Fc(bw[stage]) * Fc(dt) * k1;
            next = un + Fc(cnext[stage]) * Fc(dt) * k1;
          } else {
            next = un + acc + Fc(bw[3]) * Fc(dt) * k1;
          }
          (void)next;
        }
  }
  Flops f5 = g_flops;
  put(33, f4, f5);
  out[0] = (double)G.n[0] * G.n[1] * G.n[2];
  out[37] = (double)st.speed_iters;
  out[38] = (double)st.faces;
  out[39] = (double)(g_speed_loop_flops - loop0);
  out[40] = iters;
  for (int q = 0; q < 4; q++) out[41 + q] = nflag[q];
  out[49] = (double)g_cellvar_flops;
  out[50] = (double)g_recon_flops;
  out[51] = (double)g_facesolve_flops;
  out[52] = (double)g_edge_ppm_flops;
}

// Pointwise helpers for the pins of the test suite.

void oracle_point_prim2con(const OParams* p, const double* m16, const double* prim5, const double* B3,
                           double* cons5, double* flux15) {
  Metric3<double> m;
  m.alp = m16[0];
  for (int a = 0; a < 3; a++) m.beta[a] = m16[1 + a];
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) {
      m.g[a][c] = m16[4 + SYM[a][c]];
      m.K[a][c] = m16[10 + SYM[a][c]];
    }
  metric_complete(m);
  Prim<double> pr;
  pr.rho = prim5[0];
  pr.press = prim5[1];
  pr.eps = pr.press / ((p->gamma - 1.0) * pr.rho);
  for (int a = 0; a < 3; a++) {
    pr.vel[a] = prim5[2 + a];
    pr.B[a] = B3[a];
  }
  Comoving<double> c = comoving(m, pr);
  Cons<double> U = prim2con(m, pr, c);
  cons5[0] = U.D;
  for (int a = 0; a < 3; a++) cons5[1 + a] = U.S[a];
  cons5[4] = U.tau;
  if (flux15)
    for (int d = 0; d < 3; d++) flux(m, pr, c, U, d, flux15 + 5 * d);
}

void oracle_point_wave_speeds(const OParams* p, const double* m16, const double* prim5, const double* B3, int d,
                              double* lam) {
  Metric3<double> m;
  m.alp = m16[0];
  for (int a = 0; a < 3; a++) m.beta[a] = m16[1 + a];
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) {
      m.g[a][c] = m16[4 + SYM[a][c]];
      m.K[a][c] = m16[10 + SYM[a][c]];
    }
  metric_complete(m);
  Prim<double> pr;
  pr.rho = prim5[0];
  pr.press = prim5[1];
  pr.eps = pr.press / ((p->gamma - 1.0) * pr.rho);
  for (int a = 0; a < 3; a++) {
    pr.vel[a] = prim5[2 + a];
    pr.B[a] = B3[a];
  }
  Comoving<double> c = comoving(m, pr);
  int it;
  wave_speeds(m, pr, c, p->gamma, d, &lam[0], &lam[1], &it);
}

// c2p of one undensitised state (cons5 = D, S_i, tau; B3 undensitised) with the solver chosen by `which`:
// 0 = full chain, 1 = Noble only, 2 = Palenzuela only.  Returns the flag (or -9 if the solver failed).
int oracle_point_c2p(const OParams* p, const double* m16, const double* cons5, const double* B3,
                     const double* guess5, double* prim5, int which, int* iters) {
  Metric3<double> m;
  m.alp = m16[0];
  for (int a = 0; a < 3; a++) m.beta[a] = m16[1 + a];
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) {
      m.g[a][c] = m16[4 + SYM[a][c]];
      m.K[a][c] = m16[10 + SYM[a][c]];
    }
  metric_complete(m);
  C2PIn in;
  in.D = cons5[0];
  in.Dtilde = cons5[0] * m.sqrtg;
  for (int a = 0; a < 3; a++) in.S[a] = cons5[1 + a];
  in.tau = cons5[4];
  for (int a = 0; a < 3; a++) in.B[a] = B3[a];
  in.guess_rho = guess5[0];
  in.guess_press = guess5[1];
  for (int a = 0; a < 3; a++) in.guess_vel[a] = guess5[2 + a];
  C2POut o;
  o.iters = 0;
  o.flag = 0;
  o.reset = false;
  int flag;
  if (which == 0) {
    o = c2p_cell(m, in, *p);
    flag = o.flag;
  } else {
    double S2 = 0.0, B2 = 0.0, BS = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        S2 += m.gu[a][b] * in.S[a] * in.S[b];
        B2 += m.g[a][b] * in.B[a] * in.B[b];
      }
    for (int a = 0; a < 3; a++) BS += in.B[a] * in.S[a];
    bool ok = (which == 1) ? c2p_noble(m, in, *p, S2, B2, BS, &o) : c2p_palenzuela(m, in, *p, S2, B2, BS, &o);
    flag = ok ? (which == 1 ? 0 : 1) : -9;
  }
  prim5[0] = o.rho;
  prim5[1] = o.press;
  for (int a = 0; a < 3; a++) prim5[2 + a] = o.vel[a];
  if (iters) *iters = o.iters;
  return flag;
}

// Batched version of oracle_point_c2p over n independent states (arrays of 16, 5, 3, 5 doubles per state).
void oracle_batch_c2p(const OParams* p, long n, const double* m16, const double* cons5, const double* B3,
                      const double* guess5, double* prim5, int which, int* flags, int* iters) {
  for (long q = 0; q < n; q++)
    flags[q] = oracle_point_c2p(p, m16 + 16 * q, cons5 + 5 * q, B3 + 3 * q, guess5 + 5 * q, prim5 + 5 * q, which,
                                iters ? iters + q : nullptr);
}

// Batched prim->cons over n states (undensitised output when the metric is flat; densitised in general).
void oracle_batch_prim2con(const OParams* p, long n, const double* m16, const double* prim5, const double* B3,
                           double* cons5) {
  for (long q = 0; q < n; q++) oracle_point_prim2con(p, m16 + 16 * q, prim5 + 5 * q, B3 + 3 * q, cons5 + 5 * q,
                                                     nullptr);
}

// One face solve from explicit states (for pins): L8 and R8 hold rho, p, u^x, u^y, u^z (u = W v) and the
// undensitised B^x, B^y, B^z of the left and right sides (the normal entry unused), Bn the densitised normal
// field, m16 the face metric.  out (13): the hydro flux (5), the induction fluxes along d of B~^x,y,z (3, the
// normal one 0; computed when p->efield selects flux constrained transport), c_max, c_min, the upwind v~ (3).
void oracle_point_face(const OParams* p, const double* m16, const double* L8, const double* R8, double Bn, int d,
                       double* out) {
  Metric3<double> m;
  m.alp = m16[0];
  for (int a = 0; a < 3; a++) m.beta[a] = m16[1 + a];
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) {
      m.g[a][c] = m16[4 + SYM[a][c]];
      m.K[a][c] = m16[10 + SYM[a][c]];
    }
  metric_complete(m);
  FaceInput in;
  const double* side[2] = {L8, R8};
  for (int s = 0; s < 2; s++) {
    in.rho[s] = side[s][0];
    in.press[s] = side[s][1];
    for (int a = 0; a < 3; a++) {
      in.u[s][a] = side[s][2 + a];
      in.Bt[s][a] = side[s][5 + a];
    }
  }
  in.Bn = Bn;
  const FaceOut<double> o = face_solve<double>(m, in, p->gamma, d, p->flux, p->efield == EFIELD_FCT);
  for (int v = 0; v < 5; v++) out[v] = o.F[v];
  for (int a = 0; a < 3; a++) out[5 + a] = o.Fb[a];
  out[8] = o.cmax;
  out[9] = o.cmin;
  for (int a = 0; a < 3; a++) out[10 + a] = o.vbar[a];
}

// Reconstruction of one cell from five values: returns the lower and upper face values.
void oracle_point_recon(int scheme, const double* a5, double* aL, double* aR) {
  recon_cell<double>(scheme, a5, aL, aR);
}

// Sources at one point from an explicit metric, its derivatives and the primitives (for the 4-covariant pin).
void oracle_point_sources(const OParams* p, const double* m16, const double* dalp3, const double* dbeta9,
                          const double* dg27, const double* prim5, const double* B3, double* src5) {
  Metric3<double> m;
  m.alp = m16[0];
  for (int a = 0; a < 3; a++) m.beta[a] = m16[1 + a];
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) {
      m.g[a][c] = m16[4 + SYM[a][c]];
      m.K[a][c] = m16[10 + SYM[a][c]];
    }
  metric_complete(m);
  MetricDeriv<double> dm;
  for (int i = 0; i < 3; i++) {
    dm.dalp[i] = dalp3[i];
    for (int a = 0; a < 3; a++) dm.dbeta[i][a] = dbeta9[3 * i + a];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) dm.dg[i][a][b] = dg27[9 * i + 3 * a + b];
  }
  Prim<double> pr;
  pr.rho = prim5[0];
  pr.press = prim5[1];
  pr.eps = pr.press / ((p->gamma - 1.0) * pr.rho);
  for (int a = 0; a < 3; a++) {
    pr.vel[a] = prim5[2 + a];
    pr.B[a] = B3[a];
  }
  source_terms<double>(m, dm, pr, src5);
}

// Sources at the interior cells of a grid from the vertex metric (4th-order interpolation and derivatives).
void oracle_grid_sources(const OParams* p, const OBlock* b, const double* const* metric, double* const* U,
                         double* const* prim, double* const* src) {
  Grid G(*b);
  VertexMetric vm = vmetric(metric);
  Field Bf[3], Bc[3];
  face_B(G, U[5], U[6], U[7], Bf);
  centre_B(G, vm, Bf, Bc);
  for (int k = G.g; k < G.g + G.n[2]; k++)
    for (int j = G.g; j < G.g + G.n[1]; j++)
      for (int i = G.g; i < G.g + G.n[0]; i++) {
        const long c = G.at(i, j, k);
        const Metric3<double> m = metric_at_centre(G, vm, i, j, k);
        const MetricDeriv<double> dm = metric_deriv_at_centre(G, vm, i, j, k);
        Prim<double> pr;
        pr.rho = prim[0][c];
        pr.press = prim[1][c];
        pr.eps = pr.press / ((p->gamma - 1.0) * pr.rho);
        for (int a = 0; a < 3; a++) {
          pr.vel[a] = prim[2 + a][c];
          pr.B[a] = Bc[a][c];
        }
        double s[5];
        source_terms<double>(m, dm, pr, s);
        for (int v = 0; v < 5; v++) src[v][c] = s[v];
      }
}

}  // extern "C"
