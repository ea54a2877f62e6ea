// Forward-mode dual numbers with N derivative directions, used by the adjoint kernels to form the local
// Jacobian of a pointwise map (face solve, reconstruction, edge field, sources) in one pass of the same
// templated code that the forward kernels run with T = double.  Branches (limiters, max/min, floors) compare
// values, so the derivative is that of the branch taken (a one-sided derivative at a kink).
#pragma once

#include <cuda_runtime.h>

namespace asterx {

template <int N>
struct Dual {
  double v;
  double d[N];
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; i++) d[i] = 0.0;
  }
  __host__ __device__ static Dual seed(double x, int k) {
    Dual r(x);
    r.d[k] = 1.0;
    return r;
  }
};

template <int N> __host__ __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = -a.d[i];
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v += b;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator+(double a, const Dual<N>& b) { return b + a; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v -= b;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(double a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a - b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = -b.d[i];
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a * ib;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = -r.v * b.d[i] * ib;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { return a = a + b; }
template <int N> __host__ __device__ __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { return a = a - b; }

template <int N> __host__ __device__ __forceinline__ Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * h;
  return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> fabs(const Dual<N>& a) { return a.v < 0.0 ? -a : a; }
template <int N> __host__ __device__ __forceinline__ Dual<N> fmax(const Dual<N>& a, const Dual<N>& b) {
  return (b.v > a.v) ? b : a;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> fmin(const Dual<N>& a, const Dual<N>& b) {
  return (b.v < a.v) ? b : a;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> fmax(const Dual<N>& a, double b) { return fmax(a, Dual<N>(b)); }
template <int N> __host__ __device__ __forceinline__ Dual<N> fmin(const Dual<N>& a, double b) { return fmin(a, Dual<N>(b)); }
template <int N> __host__ __device__ __forceinline__ Dual<N> fmax(double a, const Dual<N>& b) { return fmax(Dual<N>(a), b); }
template <int N> __host__ __device__ __forceinline__ Dual<N> fmin(double a, const Dual<N>& b) { return fmin(Dual<N>(a), b); }

#define ASTERX_DUAL_CMP(op)                                                                              \
  template <int N> __host__ __device__ __forceinline__ bool operator op(const Dual<N>& a, const Dual<N>& b) {    \
    return a.v op b.v;                                                                                   \
  }                                                                                                      \
  template <int N> __host__ __device__ __forceinline__ bool operator op(const Dual<N>& a, double b) { return a.v op b; } \
  template <int N> __host__ __device__ __forceinline__ bool operator op(double a, const Dual<N>& b) { return a op b.v; }
ASTERX_DUAL_CMP(<)
ASTERX_DUAL_CMP(>)
ASTERX_DUAL_CMP(<=)
ASTERX_DUAL_CMP(>=)
#undef ASTERX_DUAL_CMP

// the double versions stay visible next to the dual overloads
using ::fabs;
using ::fmax;
using ::fmin;
using ::sqrt;

// value of a scalar (double or dual)
__host__ __device__ __forceinline__ double val(double x) { return x; }
template <int N> __host__ __device__ __forceinline__ double val(const Dual<N>& x) { return x.v; }

}  // namespace asterx
