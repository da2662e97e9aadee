// Per-example gradients without any allocation.
//
// Some callers cannot call cudaMalloc: their device memory belongs to someone
// else (a framework's caching allocator, a fixed pool with a hard budget) or
// they run a latency-bound loop in which an allocation, with its implicit
// synchronisation and possible failure, is not acceptable.  This entry point
// serves them: the caller passes device inputs and the output, and the
// forward/backward caches live in one file-scope device array instead of the
// handle's workspace.
#include <mutex>

#include "internal.h"

namespace hm {
namespace {

// 32 MiB of FP64 scratch.  Every GPU that loads the library holds this array
// until the process exits.
constexpr size_t kStaticScratchDoubles = (size_t)1 << 22;
__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Device address of the array, looked up once per device (in host code the
// symbol's name is only a host-side stand-in, never a device address).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

hess_status static_scratch_for_current_device(void** out) {
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(HESS_ERR_UNSUPPORTED, "device index %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return set_error(HESS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HESS_OK;
}

hess_status require_device_ptr(const void* p, int dev, const char* name) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HESS_ERR_INVALID_ARG, "%s must be device memory", name);
  }
  if (!(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
    return set_error(HESS_ERR_INVALID_ARG, "%s must be device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    return set_error(HESS_ERR_INVALID_ARG, "%s lives on device %d, the current device is %d", name,
                     at.device, dev);
  return HESS_OK;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" hess_status per_example_grads_noalloc(const hess_mlp_desc* desc, const double* omega,
                                                  const double* X, const double* Y, int64_t N,
                                                  double* G, void* stream) {
  clear_error();
  if (!omega || !X || !Y || !G)
    return set_error(HESS_ERR_INVALID_ARG, "omega, X, Y and G must be non-NULL");
  if (N < 1 || N > (1ll << 31) - 1)
    return set_error(HESS_ERR_INVALID_ARG, "N must be in [1, 2^31) (got %lld)", (long long)N);
  Net net;
  HM_TRY(make_net(desc, &net));
  // size the caches before touching the GPU
  Arena ar;
  Caches<double> c;
  plan_caches(ar, net, N, c);
  const size_t cap = kStaticScratchDoubles * sizeof(double);
  if (ar.off > cap)
    return set_error(HESS_ERR_INVALID_ARG,
                     "this network and N need %zu bytes of scratch; the static buffer holds %zu",
                     ar.off, cap);
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_TRY(require_device_ptr(omega, dev, "omega"));
  HM_TRY(require_device_ptr(X, dev, "X"));
  HM_TRY(require_device_ptr(Y, dev, "Y"));
  HM_TRY(require_device_ptr(G, dev, "G"));
  void* base = nullptr;
  HM_TRY(static_scratch_for_current_device(&base));
  ar = Arena{static_cast<char*>(base), 0};
  plan_caches(ar, net, N, c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every cache entry is written before it is read, so stale contents from an
  // earlier call need no clearing
  HM_TRY(forward_backward<double>(net, omega, X, Y, c, s));
  HM_TRY(write_grads<double>(net, c, G, net.P, s));
  return HESS_OK;
}
