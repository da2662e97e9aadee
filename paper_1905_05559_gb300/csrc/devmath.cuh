// Device helpers shared by the FP64 eigensolvers: a counter-based random
// draw, warp and block sums, and refined reciprocal / reciprocal square root.
#pragma once
#include <cstdint>

namespace hm {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// SplitMix64 in counter mode: uniform in [-1, 1)
__device__ __forceinline__ double rnd_sym(uint64_t key, uint64_t i) {
  uint64_t z = mix64(key + (i + 1) * 0x9E3779B97F4A7C15ull);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1/x to about one ulp: the hardware reciprocal estimate refined by two
// Newton-Raphson steps r <- r + r (1 - x r) (quadratic convergence from the
// estimate's ~2^-23 relative error).  Used inside the long dependent chains of
// the tridiagonal recurrences, where a full-precision division would dominate.
__device__ __forceinline__ double rcp64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(x) for x > 0: the hardware estimate refined by two Newton-Raphson
// steps r <- r (3 - x r^2) / 2.  On this GPU an FP64 operation has a long
// dependent latency, and this chain is shorter than a square root followed
// by a division.
__device__ __forceinline__ double rsqrt64(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double hx = 0.5 * x;
  r = r * fma(-hx * r, r, 1.5);
  return r * fma(-hx * r, r, 1.5);
}

// sum over a block of up to 1024 threads
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

}  // namespace
}  // namespace hm
