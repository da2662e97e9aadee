// Per-example gradients without any allocation.
//
// Some callers cannot call cudaMalloc: their device memory belongs to someone
// else (a framework's caching allocator, a fixed pool with a hard budget) or
// they run a latency-bound loop in which an allocation, with its implicit
// synchronisation and possible failure, is not acceptable.  This entry point
// serves them: the caller passes device inputs and the output, and the
// forward/backward caches live in one file-scope device array instead of the
// handle's workspace.
#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace hm {
namespace {

// 32 MiB of FP64 scratch.  Every GPU that loads the library holds this array
// until the process exits.
constexpr size_t kStaticScratchDoubles = (size_t)1 << 22;
__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Device address of the array.  cudaGetSymbolAddress answers for the
// context current on the calling thread (in host code the symbol's name is
// only a host-side stand-in, never a device address), and a module's globals
// get a fresh address in every context that loads it: after a
// cudaDeviceReset, or under a caller's own driver-API context on the same
// device, an address cached per device index would be stale.  So the lookup
// runs once per context, with that context current, and is cached under the
// context's handle.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext* ctx);
constexpr int kMaxContexts = 64;
std::mutex g_scratch_mu;
struct ScratchEntry {
  void* ctx;
  void* addr;
};
ScratchEntry g_scratch[kMaxContexts] = {};
int g_scratch_n = 0;
PfnCtxGetCurrent g_ctx_get_current = nullptr;

// Driver entry points, resolved once through the runtime (the library links
// no driver stub).
typedef CUresult (*PfnPointerGetAttribute)(void* data, CUpointer_attribute attribute, CUdeviceptr ptr);
std::once_flag g_driver_once;
PfnPointerGetAttribute g_ptr_attr = nullptr;

void resolve_driver_entry_points() {
  std::call_once(g_driver_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      g_ptr_attr = reinterpret_cast<PfnPointerGetAttribute>(fn);
    cudaGetLastError();
  });
}

hess_status current_context(void** ctx) {
  resolve_driver_entry_points();
  if (!g_ctx_get_current) return set_error(HESS_ERR_CUDA, "cuCtxGetCurrent unavailable");
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return set_error(HESS_ERR_CUDA, "no CUDA context is current");
  *ctx = c;
  return HESS_OK;
}

hess_status static_scratch_for_current_context(void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  void* ctx = nullptr;
  HM_TRY(current_context(&ctx));
  for (int i = 0; i < g_scratch_n; ++i)
    if (g_scratch[i].ctx == ctx) {
      *out = g_scratch[i].addr;
      return HESS_OK;
    }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return set_error(HESS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
  }
  // once the table is full the oldest entry makes room
  if (g_scratch_n == kMaxContexts) {
    for (int i = 0; i + 1 < kMaxContexts; ++i) g_scratch[i] = g_scratch[i + 1];
    --g_scratch_n;
  }
  g_scratch[g_scratch_n++] = ScratchEntry{ctx, p};
  *out = p;
  return HESS_OK;
}

// Start and length of the allocation that contains p.
hess_status pointer_range(const void* p, size_t* start, size_t* size) {
  resolve_driver_entry_points();
  if (!g_ptr_attr) return HESS_ERR_UNSUPPORTED;
  CUdeviceptr st = 0;
  size_t sz = 0;
  const CUdeviceptr addr = reinterpret_cast<CUdeviceptr>(p);
  if (g_ptr_attr(&st, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, addr) != CUDA_SUCCESS ||
      g_ptr_attr(&sz, CU_POINTER_ATTRIBUTE_RANGE_SIZE, addr) != CUDA_SUCCESS)
    return HESS_ERR_UNSUPPORTED;
  *start = (size_t)st;
  *size = sz;
  return HESS_OK;
}

// Device (or managed) memory of device dev holding at least `bytes` bytes from
// p to the end of its allocation.  A buffer carved out of a larger allocation
// (a caching allocator's segment) passes whenever the segment is long enough:
// the check catches a buffer that is too short for its allocation, not one
// that is too short for the caller's own bookkeeping.
hess_status require_device_ptr(const void* p, int dev, size_t bytes, const char* name) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HESS_ERR_INVALID_ARG, "%s must be device memory", name);
  }
  if (!(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
    return set_error(HESS_ERR_INVALID_ARG, "%s must be device memory", name);
  if (at.device != dev)
    return set_error(HESS_ERR_INVALID_ARG, "%s lives on device %d, the current device is %d", name,
                     at.device, dev);
  size_t start = 0, size = 0;
  if (pointer_range(p, &start, &size) == HESS_OK) {
    const size_t avail = start + size - reinterpret_cast<size_t>(p);
    if (avail < bytes)
      return set_error(HESS_ERR_INVALID_ARG, "%s: %zu bytes from the pointer to the end of its allocation, %zu needed",
                       name, avail, bytes);
  }
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
  const int T1 = net.T[0], TL = net.T[net.L - 1];
  HM_TRY(require_device_ptr(omega, dev, (size_t)net.P * sizeof(double), "omega"));
  HM_TRY(require_device_ptr(X, dev, (size_t)N * T1 * sizeof(double), "X"));
  HM_TRY(require_device_ptr(Y, dev, (size_t)N * TL * sizeof(double), "Y"));
  HM_TRY(require_device_ptr(G, dev, (size_t)N * net.P * sizeof(double), "G"));
  void* base = nullptr;
  HM_TRY(static_scratch_for_current_context(&base));
  ar = Arena{static_cast<char*>(base), 0};
  plan_caches(ar, net, N, c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every cache entry is written before it is read, so stale contents from an
  // earlier call need no clearing
  HM_TRY(forward_backward<double>(net, omega, X, Y, c, s));
  HM_TRY(write_grads<double>(net, c, G, net.P, s));
  return HESS_OK;
}
