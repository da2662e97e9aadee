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

// 1/x within one ulp for |x| in [2^-1022, 2^1022]: the hardware reciprocal
// estimate refined by two Newton-Raphson steps r <- r + r (1 - x r)
// (quadratic convergence from the estimate's ~2^-23 relative error).  The
// estimate flushes subnormals: huge |x| gives 0, subnormal x a value that is
// not finite.  Used inside the long dependent chains of the tridiagonal
// recurrences, where a full-precision division would dominate.
__device__ __forceinline__ double rcp64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(x) for x in [2^-1022, 2^1022], within two ulps: the hardware
// estimate refined by two Newton-Raphson steps r <- r (3 - x r^2) / 2.  On this GPU an FP64 operation has a long
// dependent latency, and this chain is shorter than a square root followed
// by a division.
__device__ __forceinline__ double rsqrt64(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double hx = 0.5 * x;
  r = r * fma(-hx * r, r, 1.5);
  return r * fma(-hx * r, r, 1.5);
}

// ------------------------------------------------------- double-float ----
// A value carried as an unevaluated sum hi + lo of two FP32 numbers (|lo| <=
// half an ulp of hi): about 48 significant bits, with every operation on the
// FP32 pipe.  The building blocks are the error-free transformations of
// Dekker and Knuth: TwoSum (a + b = s + e exactly) and the FMA product
// (a b = p + e exactly, e = fma(a, b, -p)).  Used by the Lanczos kernel of the
// Gram matrix, where an FP64 operation would cost 64 times the FP32 issue
// slots of this GPU.
__device__ __forceinline__ float2 df_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
// The same pair from the bits of v with integer and FP32 operations only (no
// FP64 conversion or arithmetic, which this GPU issues at a small fraction of
// its FP32 rate): hi = v with its significand cut to 24 bits, lo = the other
// 29 bits rounded to 24 (|lo| < ulp(hi)), so hi + lo = v to 2^-48 relative.
// |v| below 2^-126 gives (0, 0); |v| of 2^128 and up, infinities and NaN take
// the conversions of df_split.
__device__ __forceinline__ float2 df_split_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;  // unbiased exponent
  if (e < -126) return make_float2(0.0f, 0.0f);
  if (e > 127) return df_split(v);
  const unsigned long long m = b & 0x000fffffffffffffull;
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  // lo = (the low 29 bits of the significand) 2^(e - 52)
  const int el = e - 52;
  float lo = __uint2float_rn((unsigned)(m & 0x1fffffffull));
  lo = el >= -126 ? lo * __uint_as_float((unsigned)(el + 127) << 23) : ldexpf(lo, el);
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sgn));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (s, c) + (0, 0) as a normalised pair
__device__ __forceinline__ float2 df_norm(float s, float c) {
  const float h = s + c;
  return make_float2(h, c - (h - s));
}
// running sum (s, c), unnormalised: s takes the leading parts exactly, c
// collects the rounding errors and low-order terms; adds a * b
__device__ __forceinline__ void df_mac(float2 a, float2 b, float& s, float& c) {
  const float p = a.x * b.x;
  float pe = fmaf(a.x, b.x, -p);
  pe = fmaf(a.x, b.y, pe);
  pe = fmaf(a.y, b.x, pe);
  float t, e;
  two_sum(s, p, t, e);
  s = t;
  c += e + pe;
}
__device__ __forceinline__ void df_acc(float2 a, float& s, float& c) {
  float t, e;
  two_sum(s, a.x, t, e);
  s = t;
  c += e + a.y;
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  return df_norm(s, e + (a.y + b.y));
}
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_norm(p, e);
}
// sqrt(a) for a >= 0: one correction of the FP32 root with the exact residual
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  if (!(a.x > 0.0f)) return make_float2(0.0f, 0.0f);
  const float x = sqrtf(a.x);
  const float p = x * x;
  const float pe = fmaf(x, x, -p);
  const float r = ((a.x - p) - pe) + a.y;
  return df_norm(x, r * (0.5f / x));
}
// 1 / a for a != 0: one correction of the FP32 reciprocal with the exact residual
__device__ __forceinline__ float2 df_rcp(float2 a) {
  const float x = 1.0f / a.x;
  const float p = a.x * x;
  const float pe = fmaf(a.x, x, -p);
  const float r = ((1.0f - p) - pe) - a.y * x;
  return df_norm(x, x * r);
}
// (s, c) summed over the warp; every lane gets the same bits (TwoSum is
// exact, so the order of its operands does not matter)
__device__ __forceinline__ float2 df_warp_sum(float s, float c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float t, e;
    two_sum(s, s2, t, e);
    s = t;
    c = (c + c2) + e;
  }
  return df_norm(s, c);
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
