// Test hook for the refined FP64 reciprocal and reciprocal square root that
// the eigensolvers use inside their dependent chains, evaluated next to
// CUDA's correctly rounded division and square root on the same inputs, and
// for the bit-level double-float split of FP64 inputs.
#include "devmath.cuh"
#include "internal.h"

namespace hm {
namespace {

__global__ void devmath_kernel(const double* x, int64_t n, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = rcp64(v);
    out[n + i] = 1.0 / v;
    out[2 * n + i] = v > 0.0 ? rsqrt64(v) : 0.0;
    out[3 * n + i] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    const float2 h = df_split_bits(v);
    out[4 * n + i] = (double)h.x;
    out[5 * n + i] = (double)h.y;
  }
}

// Eight independent FP64 FMA chains per thread: with enough warps resident,
// the SMs' FP64 pipes never wait on a dependency, so the launch's flops over
// its duration is the FP64 issue rate.
__global__ void fp64_probe_kernel(int64_t iters, double* sink) {
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = 1e-3 * (threadIdx.x + 1) + u;
  const double m = 0.9999999999, c = 1e-12;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], m, c);
  }
  const double t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  if (t == -1.0) sink[0] = t;  // never true; keeps the chains live
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" hess_status hess_check_devmath(const double* x, int64_t n, double* out, void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!x || !out))) return set_error(HESS_ERR_INVALID_ARG, "x and out must be non-NULL");
  if (n == 0) return HESS_OK;
  cudaPointerAttributes ax, ao;
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ao, out) != cudaSuccess) {
    cudaGetLastError();
    return set_error(HESS_ERR_INVALID_ARG, "x and out must be device memory");
  }
  if (ax.type != cudaMemoryTypeDevice || ao.type != cudaMemoryTypeDevice)
    return set_error(HESS_ERR_INVALID_ARG, "x and out must be device memory");
  const int64_t blocks = cdiv(n, 256) < 4096 ? cdiv(n, 256) : 4096;
  devmath_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, out);
  HM_LAUNCHED();
  return HESS_OK;
}

extern "C" hess_status hess_probe_fp64(int64_t iters, double* flops, double* sink, void* stream) {
  clear_error();
  if (iters < 1 || !flops) return set_error(HESS_ERR_INVALID_ARG, "iters >= 1 and flops non-NULL");
  int dev = 0, sms = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * sms, threads = 256;
  fp64_probe_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, sink);
  HM_LAUNCHED();
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return HESS_OK;
}
