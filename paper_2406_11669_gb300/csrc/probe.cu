// FP64 fused multiply-add throughput probe: the ALU roofline of an FP64-bound kernel is the rate at which
// the SMs retire DFMA.  Eight independent chains per thread keep the FP64 pipe busy regardless of latency.
#include <mutex>

#include "kernels.h"
#include "physics.cuh"

namespace asterx {

int device_sm_count() {
  static std::mutex mu;
  static int count[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  std::lock_guard<std::mutex> lock(mu);
  if (count[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    count[dev] = n;
  }
  return count[dev];
}

__global__ void k_dfma_probe(double* out, long iters) {
  const double s = 1.0 + 1e-12 * (threadIdx.x + 1);
  double a0 = 1.0 + 1e-9 * threadIdx.x, a1 = a0 + 1e-3, a2 = a0 + 2e-3, a3 = a0 + 3e-3;
  double a4 = a0 + 4e-3, a5 = a0 + 5e-3, a6 = a0 + 6e-3, a7 = a0 + 7e-3;
  const double c = -1e-12;
#pragma unroll 1
  for (long i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 8; r++) {
      a0 = fma(a0, s, c); a1 = fma(a1, s, c); a2 = fma(a2, s, c); a3 = fma(a3, s, c);
      a4 = fma(a4, s, c); a5 = fma(a5, s, c); a6 = fma(a6, s, c); a7 = fma(a7, s, c);
    }
  }
  out[blockIdx.x * (long)blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

cudaError_t launch_dfma_probe(double* out, int blocks, int threads, long iters, cudaStream_t s) {
  k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters);
  return cudaGetLastError();
}

// the Newton-correction reciprocal of the quartic solver applied to n values (its error bound is tested)
__global__ void k_newton_rcp(const double* __restrict__ d, double* __restrict__ out, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = newton_rcp(d[i]);
}

cudaError_t launch_newton_rcp(const double* d, double* out, long n, cudaStream_t s) {
  long blocks = (n + 255) / 256;
  const long cap = 16L * device_sm_count();
  if (blocks > cap) blocks = cap;
  k_newton_rcp<<<(int)blocks, 256, 0, s>>>(d, out, n);
  return cudaGetLastError();
}

// the two-step reciprocal applied to n values (its error bound is tested)
__global__ void k_recip(const double* __restrict__ d, double* __restrict__ out, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = recip(d[i]);
}

// the corrected quotient applied to n pairs (checked against the correctly rounded quotient)
__global__ void k_quotient(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                           long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = quotient_by(a[i], b[i], 1.0 / b[i]);
}

cudaError_t launch_quotient(const double* a, const double* b, double* out, long n, cudaStream_t s) {
  long blocks = (n + 255) / 256;
  const long cap = 16L * device_sm_count();
  if (blocks > cap) blocks = cap;
  k_quotient<<<(int)blocks, 256, 0, s>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_recip(const double* d, double* out, long n, cudaStream_t s) {
  long blocks = (n + 255) / 256;
  const long cap = 16L * device_sm_count();
  if (blocks > cap) blocks = cap;
  k_recip<<<(int)blocks, 256, 0, s>>>(d, out, n);
  return cudaGetLastError();
}

}  // namespace asterx
