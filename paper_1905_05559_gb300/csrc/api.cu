// C-ABI entry points: argument checks, host/device staging, workspace
// planning and the orchestration of the kernels of every call.
#include <cstring>
#include <string>
#include <type_traits>

#include "internal.h"

namespace hm {

static thread_local char g_err[1024];
std::atomic<int64_t> g_launches{0};

static cudaEvent_t take_event(hess_mlp* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

Tick::Tick(hess_mlp* h, int cls, double flops, double bytes) : h_(h) {
  if (!h || !h->timing) return;
  rec_.a = take_event(h);
  rec_.b = take_event(h);
  if (!rec_.a || !rec_.b) return;
  rec_.cls = cls;
  rec_.flops = flops;
  rec_.bytes = bytes;
  live_ = cudaEventRecord(rec_.a, h->stream) == cudaSuccess;
}

void Tick::stop() {
  if (!live_) return;
  live_ = false;
  if (cudaEventRecord(rec_.b, h_->stream) == cudaSuccess) h_->pending.push_back(rec_);
}

hess_status set_error(hess_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}
// Every entry point starts here: a stale, non-sticky CUDA error left by
// someone else's call on this thread must not be reported as this call's.
void clear_error() {
  g_err[0] = 0;
  cudaGetLastError();
}

hess_status make_net(const hess_mlp_desc* desc, Net* out) {
  if (!desc) return set_error(HESS_ERR_INVALID_ARG, "desc is NULL");
  if (desc->L < 2 || !desc->widths) return set_error(HESS_ERR_INVALID_ARG, "need L >= 2 and widths");
  if (desc->L > kMaxLayers) return set_error(HESS_ERR_INVALID_ARG, "at most %d layers", kMaxLayers);
  if (desc->L > 2 && !desc->act) return set_error(HESS_ERR_INVALID_ARG, "hidden activations missing");
  Net net;
  net.L = desc->L;
  for (int l = 0; l < desc->L; ++l) {
    if (desc->widths[l] < 1 || desc->widths[l] > (1 << 20))
      return set_error(HESS_ERR_INVALID_ARG, "width T_%d = %d out of range", l + 1, desc->widths[l]);
    net.T[l] = desc->widths[l];
  }
  if (net.T[net.L - 1] < 2) return set_error(HESS_ERR_INVALID_ARG, "softmax output needs T_L >= 2");
  for (int l = 0; l < desc->L - 2; ++l) {
    int a = desc->act[l];
    if (a < HESS_ACT_SIGMOID || a > HESS_ACT_RELU)
      return set_error(HESS_ERR_INVALID_ARG, "unknown activation %d for layer %d", a, l + 2);
    net.act[l] = a;
  }
  int64_t o = 0;
  for (int w = 1; w < net.L; ++w) {
    net.woff[w - 1] = o;
    net.boff[w - 1] = o + (int64_t)net.T[w - 1] * net.T[w];
    o += (int64_t)net.T[w - 1] * net.T[w] + net.T[w];
  }
  net.P = o;
  if (net.P > (1ll << 31) - 1) return set_error(HESS_ERR_INVALID_ARG, "P = %lld too large", (long long)net.P);
  *out = net;
  return HESS_OK;
}

thread_local size_t* g_dry_bytes = nullptr;

hess_status host_side_init(hess_mlp* h) {
  if (cudaMallocHost(&h->host_pinned, 4096) != cudaSuccess) return set_error(HESS_ERR_OOM, "pinned scratch");
  if (cudaHostAlloc(&h->err_host, 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&h->err_dev, h->err_host, 0) != cudaSuccess)
    return set_error(HESS_ERR_OOM, "mapped error flag");
  *h->err_host = 0;
  return HESS_OK;
}

void host_side_free(hess_mlp* h) {
  if (h->mb_batch) hess_batch_destroy(h->mb_batch);
  h->mb_batch = nullptr;
  if (h->stream2) cudaStreamDestroy(h->stream2);
  if (h->stream3) cudaStreamDestroy(h->stream3);
  if (h->stream4) cudaStreamDestroy(h->stream4);
  if (h->stream5) cudaStreamDestroy(h->stream5);
  h->stream2 = h->stream3 = h->stream4 = h->stream5 = nullptr;
  for (cudaEvent_t& e : h->fused_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (h->host_pinned) cudaFreeHost(h->host_pinned);
  if (h->err_host) cudaFreeHost(h->err_host);
  h->host_pinned = nullptr;
  h->err_host = h->err_dev = nullptr;
  stage_free(h->stage);
}

hess_status take_sticky_error(hess_mlp* h) {
  if (h->err_host && *(volatile int*)h->err_host) {
    *(volatile int*)h->err_host = 0;
    return set_error(HESS_ERR_TIMEOUT,
                     "a tensor-core pipeline wait gave up (in this or an earlier call on the handle)");
  }
  return HESS_OK;
}

hess_status stage_copy(PinnedStage& ring, const void* const* src, const size_t* bytes, void* const* dst, int n,
                       cudaStream_t s) {
  PinnedSlot& st = ring.slot[ring.next];
  ring.next = (ring.next + 1) % kStageSlots;
  size_t total = 0;
  for (int i = 0; i < n; ++i) total += align_up(bytes[i], 256);
  if (st.ev) {
    HM_CUDA(cudaEventSynchronize(st.ev));  // the previous copy has left the buffer
  } else {
    HM_CUDA(cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming));
  }
  if (total > st.cap) {
    if (st.p) cudaFreeHost(st.p);
    st.p = nullptr;
    st.cap = 0;
    const size_t want = total > ((size_t)64 << 10) ? total : ((size_t)64 << 10);
    HM_CUDA(cudaHostAlloc(&st.p, want, cudaHostAllocDefault));
    st.cap = want;
  }
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    memcpy(st.p + off, src[i], bytes[i]);
    HM_CUDA(cudaMemcpyAsync(dst[i], st.p + off, bytes[i], cudaMemcpyHostToDevice, s));
    off += align_up(bytes[i], 256);
  }
  // inside a graph capture the record becomes a node of the graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HM_CUDA(cudaStreamIsCapturing(s, &cs));
  HM_CUDA(cudaEventRecordWithFlags(st.ev, s,
                                   cs == cudaStreamCaptureStatusNone ? cudaEventRecordDefault
                                                                     : cudaEventRecordExternal));
  return HESS_OK;
}

void stage_free(PinnedStage& ring) {
  for (PinnedSlot& st : ring.slot) {
    if (st.ev) {
      cudaEventSynchronize(st.ev);
      cudaEventDestroy(st.ev);
    }
    if (st.p) cudaFreeHost(st.p);
  }
  ring = PinnedStage{};
  cudaGetLastError();
}

hess_status ensure_ws2(hess_mlp* h, size_t bytes) {
  if (bytes <= h->ws2_bytes) return HESS_OK;
  if (h->ws2) {
    HM_CUDA(cudaStreamSynchronize(h->stream));
    HM_CUDA(cudaFree(h->ws2));
    h->ws2 = nullptr;
    h->ws2_bytes = 0;
  }
  const size_t nb = align_up(bytes, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(&h->ws2, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ws2 = nullptr;
    return set_error(HESS_ERR_OOM, "second workspace of %zu bytes: %s", nb, cudaGetErrorString(e));
  }
  h->ws2_bytes = nb;
  return HESS_OK;
}

hess_status ensure_ws(hess_mlp* h, size_t bytes) {
  if (g_dry_bytes) {
    *g_dry_bytes = bytes;
    return kDryRun;
  }
  if (bytes <= h->ws_bytes) return HESS_OK;
  if (h->ws) {
    HM_CUDA(cudaStreamSynchronize(h->stream));
    HM_CUDA(cudaFree(h->ws));
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  size_t nb = align_up(bytes + (bytes >> 4), (size_t)1 << 20);
  cudaError_t e = cudaMalloc(&h->ws, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return set_error(HESS_ERR_OOM, "workspace of %zu bytes: %s", nb, cudaGetErrorString(e));
  }
  h->ws_bytes = nb;
  return HESS_OK;
}

namespace {

// 1: device (or managed) memory of the handle's device, 0: host memory
hess_status classify(const hess_mlp* h, const void* p, const char* name, int* on_dev) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *on_dev = 0;
    return HESS_OK;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    if (at.type == cudaMemoryTypeDevice && at.device != h->device)
      return set_error(HESS_ERR_INVALID_ARG, "%s lives on device %d, handle on device %d", name,
                       at.device, h->device);
    *on_dev = 1;
  } else {
    *on_dev = 0;
  }
  return HESS_OK;
}

hess_status check_common(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec,
                         const void* out) {
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (!X || !Y || !out) return set_error(HESS_ERR_INVALID_ARG, "X, Y and the output must be non-NULL");
  if (N < 1) return set_error(HESS_ERR_INVALID_ARG, "N must be >= 1 (got %lld)", (long long)N);
  if (N > (1ll << 31) - 1)
    return set_error(HESS_ERR_INVALID_ARG, "N must be < 2^31 (got %lld)", (long long)N);
  if (prec < HESS_FP64 || prec > HESS_BF16X3)
    return set_error(HESS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  return take_sticky_error(h);
}

// An input buffer: device pointer used as is, host pointer staged.
template <typename T>
struct In {
  const T* user = nullptr;
  int on_dev = 0;
  const T* dev = nullptr;
  T* stage = nullptr;
};
template <typename T>
void plan_in(Arena& ar, In<T>& in, int64_t n) {
  in.stage = in.on_dev ? nullptr : ar.take<T>(n);
  in.dev = in.on_dev ? in.user : in.stage;
}
template <typename T>
hess_status upload(const In<T>& in, int64_t n, cudaStream_t s) {
  if (!in.on_dev) HM_CUDA(cudaMemcpyAsync(in.stage, in.user, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return HESS_OK;
}

// Choose the direction-block size so that the R-operator buffers stay within
// a budget and B * N fits the 32-bit GEMM row count.
int pick_block(const Net& net, int64_t N, int jm, size_t elem) {
  int64_t sumT = 0, maxP = 0;
  for (int j = jm; j < net.L; ++j) sumT += 3 * net.T[j] + 1;
  for (int w = jm; w < net.L; ++w) {
    int64_t pl = (int64_t)net.T[w - 1] * net.T[w] + net.T[w];
    maxP = pl > maxP ? pl : maxP;
  }
  const double budget = 4.0e9;  // bytes
  double per_dir = (double)elem * ((double)N * sumT + (double)maxP) + 8.0 * N;
  int64_t B = (int64_t)(budget / per_dir);
  int64_t cap = ((1ll << 31) - 1) / (N * 64);
  if (B > cap) B = cap;
  if (B > 8192) B = 8192;
  if (B < 1) B = 1;
  if (B > 128) B = B / 128 * 128;
  return (int)B;
}

}  // namespace

hess_status locate(const hess_mlp* h, const void* p, const char* name, int* on_dev) {
  return classify(h, p, name, on_dev);
}

// Algorithmic flops of the Hessian row block d0..d0+B-1 against the columns
// of weight layer jl that lie in the upper triangle (column >= row): 2 N per
// entry (one multiply-add per example; the R{a} term of layers above the
// direction's own layer doubles that for the weight columns).
double hcontract_flops(const Net& net, int64_t N, int jm, int jl, int64_t d0, int B) {
  const int64_t Tin = net.T[jl - 1], Tout = net.T[jl];
  const int64_t c0 = net.woff[jl - 1], c1 = net.boff[jl - 1] + Tout;
  double entries = 0.0;
  for (int64_t d = d0; d < d0 + B; ++d) {
    int64_t lo = d > c0 ? d : c0;
    if (lo < c1) entries += (double)(c1 - lo);
  }
  double per = 2.0 * N * (jl > jm ? 2.0 : 1.0);
  (void)Tin;
  return entries * per;
}

// ------------------------------------------------------------ generic FP
template <typename T>
static hess_status run_grads(hess_mlp* h, const void* X, const void* Y, int64_t N, void* Gout) {
  const Net& net = h->net;
  const T* omega = std::is_same<T, double>::value ? (const T*)h->omega64 : (const T*)h->omega32;
  In<T> x, y;
  x.user = (const T*)X;
  y.user = (const T*)Y;
  int g_dev = 0;
  HM_TRY(classify(h, X, "X", &x.on_dev));
  HM_TRY(classify(h, Y, "Y", &y.on_dev));
  HM_TRY(classify(h, Gout, "G", &g_dev));
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1];
  char* split = nullptr;
  auto plan = [&](Arena& ar, Caches<T>& c, T*& G) {
    plan_in(ar, x, N * T1);
    plan_in(ar, y, N * TL);
    plan_caches(ar, net, N, c);
    G = g_dev ? (T*)Gout : ar.take<T>(N * net.P);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  Caches<T> c;
  T* G = nullptr;
  plan(ar, c, G);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar, c, G);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  HM_TRY(upload(x, N * T1, s));
  HM_TRY(upload(y, N * TL, s));
  HM_TRY(forward_backward(net, omega, x.dev, y.dev, c, s));
  {
    Tick t(h, HESS_K_GRADS, 0.0, (double)N * net.P * sizeof(T));
    HM_TRY(write_grads(net, c, G, net.P, s));
  }
  if (!g_dev) {
    HM_CUDA(cudaMemcpyAsync(Gout, G, N * net.P * sizeof(T), cudaMemcpyDeviceToHost, s));
  }
  if (!x.on_dev || !y.on_dev || !g_dev) HM_CUDA(cudaStreamSynchronize(s));
  return HESS_OK;
}

template <typename T>
static hess_status run_opg(hess_mlp* h, const void* X, const void* Y, int64_t N, void* Oout) {
  const Net& net = h->net;
  const T* omega = std::is_same<T, double>::value ? (const T*)h->omega64 : (const T*)h->omega32;
  In<T> x, y;
  x.user = (const T*)X;
  y.user = (const T*)Y;
  int o_dev = 0;
  HM_TRY(classify(h, X, "X", &x.on_dev));
  HM_TRY(classify(h, Y, "Y", &y.on_dev));
  HM_TRY(classify(h, Oout, "OPG", &o_dev));
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1], P = net.P;
  char* split = nullptr;
  auto plan = [&](Arena& ar, Caches<T>& c, T*& G, T*& O) {
    plan_in(ar, x, N * T1);
    plan_in(ar, y, N * TL);
    plan_caches(ar, net, N, c);
    G = ar.take<T>(N * P);
    O = o_dev ? (T*)Oout : ar.take<T>(P * P);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  Caches<T> c;
  T *G = nullptr, *O = nullptr;
  plan(ar, c, G, O);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar, c, G, O);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  HM_TRY(upload(x, N * T1, s));
  HM_TRY(upload(y, N * TL, s));
  HM_TRY(forward_backward(net, omega, x.dev, y.dev, c, s));
  HM_TRY(write_grads(net, c, G, P, s));
  // OPG = G^T G / N on the upper tiles, then mirrored
  Gemm<T> g;
  g.M = (int)P;
  g.N = (int)P;
  g.K = (int)N;
  g.alpha = T(1) / T(N);
  g.A = G;
  g.sam = 1;
  g.sak = P;
  g.B = G;
  g.sbk = P;
  g.sbn = 1;
  g.C = O;
  g.scm = P;
  g.scn = 1;
  g.upper = 1;
  {
    // algorithmic work of the symmetric rank-N update: N P (P + 1) flops
    Tick t(h, HESS_K_SYRK, (double)N * P * (P + 1), 0.0);
    HM_TRY(gemm(g, s));
  }
  HM_TRY(mirror_upper(O, P, P, s));
  if (!o_dev) HM_CUDA(cudaMemcpyAsync(Oout, O, P * P * sizeof(T), cudaMemcpyDeviceToHost, s));
  if (!x.on_dev || !y.on_dev || !o_dev) HM_CUDA(cudaStreamSynchronize(s));
  return HESS_OK;
}

// Split-BF16 OPG on the tensor cores.
hess_status run_opg_tc(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3, void* Oout);
// Hessian with the tensor-core contraction for the block's own layer.
hess_status run_hessian_tc(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3, void* Hout);

template <typename T>
static hess_status run_hessian(hess_mlp* h, const void* X, const void* Y, int64_t N, void* Hout) {
  const Net& net = h->net;
  const T* omega = std::is_same<T, double>::value ? (const T*)h->omega64 : (const T*)h->omega32;
  In<T> x, y;
  x.user = (const T*)X;
  y.user = (const T*)Y;
  int o_dev = 0;
  HM_TRY(classify(h, X, "X", &x.on_dev));
  HM_TRY(classify(h, Y, "Y", &y.on_dev));
  HM_TRY(classify(h, Hout, "H", &o_dev));
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1], P = net.P;
  // one block size for all layers keeps the plan simple: size it for the
  // most demanding layer
  int Bmax = 1 << 30;
  int64_t most_dirs = 0;
  for (int jm = 1; jm < net.L; ++jm) {
    int b = pick_block(net, N, jm, sizeof(T));
    Bmax = b < Bmax ? b : Bmax;
    int64_t nd = (int64_t)net.T[jm - 1] * net.T[jm] + net.T[jm];
    most_dirs = nd > most_dirs ? nd : most_dirs;
  }
  if (Bmax > most_dirs) Bmax = (int)most_dirs;
  int64_t maxPl = 0;
  for (int w = 1; w < net.L; ++w) {
    int64_t pl = (int64_t)net.T[w - 1] * net.T[w] + net.T[w];
    maxPl = pl > maxPl ? pl : maxPl;
  }
  char* split = nullptr;
  auto plan = [&](Arena& ar, Caches<T>& c, RopBufs<T>& r, T*& tmp, T*& O) {
    plan_in(ar, x, N * T1);
    plan_in(ar, y, N * TL);
    plan_caches(ar, net, N, c);
    plan_rop(ar, net, N, 1, Bmax, r);
    tmp = ar.take<T>((int64_t)Bmax * maxPl);
    O = o_dev ? (T*)Hout : ar.take<T>(P * P);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  Caches<T> c;
  RopBufs<T> r;
  T *tmp = nullptr, *O = nullptr;
  plan(ar, c, r, tmp, O);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar, c, r, tmp, O);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  HM_TRY(upload(x, N * T1, s));
  HM_TRY(upload(y, N * TL, s));
  HM_TRY(forward_backward(net, omega, x.dev, y.dev, c, s));
  for (int jm = 1; jm < net.L; ++jm) {
    const int64_t lo = net.woff[jm - 1], hi = net.boff[jm - 1] + net.T[jm];
    for (int64_t d0 = lo; d0 < hi; d0 += Bmax) {
      int B = (int)((hi - d0) < Bmax ? (hi - d0) : Bmax);
      RopBufs<T> rb = r;
      rb.B = B;
      {
        Tick t(h, HESS_K_ROP, 0.0, 0.0);
        HM_TRY(rop_block(net, omega, c, jm, d0, B, rb, s));
      }
      for (int jl = jm; jl < net.L; ++jl) {
        // one product over N per computed Hessian entry of this row block
        Tick t(h, HESS_K_HCONTRACT, hcontract_flops(net, N, jm, jl, d0, B), 0.0);
        HM_TRY(contract_layer(net, c, rb, jm, jl, d0, tmp, O, s));
      }
    }
  }
  if (!o_dev) HM_CUDA(cudaMemcpyAsync(Hout, O, P * P * sizeof(T), cudaMemcpyDeviceToHost, s));
  if (!x.on_dev || !y.on_dev || !o_dev) HM_CUDA(cudaStreamSynchronize(s));
  return HESS_OK;
}

static hess_status run_eig(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                           hess_precision prec, double* evals, double* evecs) {
  const Net& net = h->net;
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1], P = net.P;
  const bool dbl = prec == HESS_FP64;
  const size_t es = dbl ? sizeof(double) : sizeof(float);
  int x_dev = 0, y_dev = 0, ev_dev = 0, q_dev = 0;
  HM_TRY(classify(h, X, "X", &x_dev));
  HM_TRY(classify(h, Y, "Y", &y_dev));
  HM_TRY(classify(h, evals, "evals", &ev_dev));
  HM_TRY(classify(h, evecs, "evecs", &q_dev));
  char* split = nullptr;
  auto plan = [&](Arena& ar, void*& xs, void*& ys, double*& xd, double*& yd, Caches<double>& c,
                  double*& evd, double*& eqd) {
    xs = (x_dev ? nullptr : ar.take<char>(N * T1 * es));
    ys = (y_dev ? nullptr : ar.take<char>(N * TL * es));
    xd = dbl && x_dev ? (double*)X : ar.take<double>(N * T1);
    yd = dbl && y_dev ? (double*)Y : ar.take<double>(N * TL);
    plan_caches(ar, net, N, c);
    evd = ev_dev ? evals : ar.take<double>(k);
    eqd = q_dev ? evecs : ar.take<double>(P * (int64_t)k);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  void *xs, *ys;
  double *xd, *yd, *evd, *eqd;
  Caches<double> c;
  EigResult res;
  plan(ar, xs, ys, xd, yd, c, evd, eqd);
  HM_TRY(topk_eig_gram(h, net, c, N, k, evd, eqd, ar, true, &res));
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar, xs, ys, xd, yd, c, evd, eqd);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  const void* xsrc = X;
  const void* ysrc = Y;
  if (!x_dev) {
    HM_CUDA(cudaMemcpyAsync(xs, X, N * T1 * es, cudaMemcpyHostToDevice, s));
    xsrc = xs;
  }
  if (!y_dev) {
    HM_CUDA(cudaMemcpyAsync(ys, Y, N * TL * es, cudaMemcpyHostToDevice, s));
    ysrc = ys;
  }
  if (dbl) {
    if (xsrc != xd) HM_CUDA(cudaMemcpyAsync(xd, xsrc, N * T1 * 8, cudaMemcpyDeviceToDevice, s));
    if (ysrc != yd) HM_CUDA(cudaMemcpyAsync(yd, ysrc, N * TL * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    HM_TRY(convert((const float*)xsrc, xd, N * T1, s));
    HM_TRY(convert((const float*)ysrc, yd, N * TL, s));
  }
  HM_TRY(forward_backward(net, (const double*)h->omega64, (const double*)xd, (const double*)yd, c, s, true));
  {
    Tick t(h, HESS_K_EIG, 0.0, 0.0);
    HM_TRY(topk_eig_gram(h, net, c, N, k, evd, eqd, ar, false, &res));
    t.set_work(res.flops, 0.0);
  }
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evals, evd, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(evecs, eqd, P * k * sizeof(double), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  if (!res.converged)
    return set_error(HESS_ERR_NOT_CONVERGED, "Lanczos did not converge in %d steps",
                     res.lanczos_steps);
  if (res.rank_deficient)
    return set_error(HESS_ERR_RANK_DEFICIENT, "some of the top-%d OPG eigenvalues are null", k);
  return HESS_OK;
}

}  // namespace hm

using namespace hm;

extern "C" {

hess_status hess_mlp_create(const hess_mlp_desc* desc, const double* omega, void* stream,
                            hess_mlp** out) {
  clear_error();
  if (!desc || !out || !omega) return set_error(HESS_ERR_INVALID_ARG, "desc, omega and out must be non-NULL");
  *out = nullptr;
  Net net;
  HM_TRY(make_net(desc, &net));
  hess_mlp* h = new hess_mlp();
  h->net = net;
  h->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return set_error(HESS_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  hess_status st = HESS_OK;
  if (cudaMalloc(&h->omega64, net.P * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->omega32, net.P * sizeof(float)) != cudaSuccess ||
      host_side_init(h) != HESS_OK) {
    cudaGetLastError();
    st = set_error(HESS_ERR_OOM, "cannot allocate parameters");
  }
  if (st == HESS_OK) st = hess_mlp_set_params(h, omega);
  if (st != HESS_OK) {
    hess_mlp_destroy(h);
    return st;
  }
  *out = h;
  return HESS_OK;
}

hess_status hess_mlp_destroy(hess_mlp* h) {
  if (!h) return HESS_OK;
  Guard g(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->owns_params) {
    cudaFree(h->omega64);
    cudaFree(h->omega32);
  }
  cudaFree(h->ws);
  if (h->ws2) cudaFree(h->ws2);
  host_side_free(h);
  for (auto& r : h->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  cudaGetLastError();
  delete h;
  return HESS_OK;
}

int64_t hess_mlp_num_params(const hess_mlp* h) { return h ? h->net.P : -1; }

hess_status hess_mlp_set_params(hess_mlp* h, const double* omega) {
  clear_error();
  if (!h || !omega) return set_error(HESS_ERR_INVALID_ARG, "handle and omega must be non-NULL");
  Guard g(h->device);
  int on_dev = 0;
  HM_TRY(classify(h, omega, "omega", &on_dev));
  HM_CUDA(cudaMemcpyAsync(h->omega64, omega, h->net.P * sizeof(double),
                          on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  HM_TRY(convert(h->omega64, h->omega32, h->net.P, h->stream));
  if (!on_dev) HM_CUDA(cudaStreamSynchronize(h->stream));
  return HESS_OK;
}

hess_status hess_mlp_set_stream(hess_mlp* h, void* stream) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  h->stream = (cudaStream_t)stream;
  return HESS_OK;
}

hess_status hess_mlp_set_operand_limit(hess_mlp* h, int64_t bytes) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (bytes < (1 << 20)) return set_error(HESS_ERR_INVALID_ARG, "operand limit must be at least 1 MiB");
  h->op_limit = (size_t)bytes;
  return HESS_OK;
}

hess_status hess_mlp_set_eig_blocks(hess_mlp* h, int blocks) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (blocks < 0) return set_error(HESS_ERR_INVALID_ARG, "blocks must be >= 0");
  h->lz_blocks = blocks;
  return HESS_OK;
}

hess_status per_example_grads(hess_mlp* h, const void* X, const void* Y, int64_t N,
                              hess_precision prec, void* G) {
  clear_error();
  HM_TRY(check_common(h, X, Y, N, prec, G));
  if (N * h->net.P > (1ll << 40)) return set_error(HESS_ERR_INVALID_ARG, "N * P too large");
  Guard g(h->device);
  if (prec == HESS_FP64) return run_grads<double>(h, X, Y, N, G);
  return run_grads<float>(h, X, Y, N, G);
}

hess_status opg(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec, void* OPG) {
  clear_error();
  HM_TRY(check_common(h, X, Y, N, prec, OPG));
  Guard g(h->device);
  switch (prec) {
    case HESS_FP64:
      return run_opg<double>(h, X, Y, N, OPG);
    case HESS_FP32:
      return run_opg<float>(h, X, Y, N, OPG);
    case HESS_BF16:
      return run_opg_tc(h, X, Y, N, false, OPG);
    default:
      return run_opg_tc(h, X, Y, N, true, OPG);
  }
}

hess_status exact_hessian(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec,
                          void* H) {
  clear_error();
  HM_TRY(check_common(h, X, Y, N, prec, H));
  Guard g(h->device);
  switch (prec) {
    case HESS_FP64:
      return run_hessian<double>(h, X, Y, N, H);
    case HESS_FP32:
      return run_hessian<float>(h, X, Y, N, H);
    case HESS_BF16:
      return run_hessian_tc(h, X, Y, N, false, H);
    default:
      return run_hessian_tc(h, X, Y, N, true, H);
  }
}

hess_status opg_topk_eig(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                         hess_precision prec, double* evals, double* evecs) {
  clear_error();
  if (!evals) return set_error(HESS_ERR_INVALID_ARG, "evals must be non-NULL");
  HM_TRY(check_common(h, X, Y, N, prec, evecs));
  if (k < 1 || k > N || k > h->net.P)
    return set_error(HESS_ERR_INVALID_ARG, "need 1 <= k <= min(N, P) (k = %d, N = %lld, P = %lld)", k,
                     (long long)N, (long long)h->net.P);
  if (N > 65536) return set_error(HESS_ERR_INVALID_ARG, "the Gram route supports N <= 65536");
  Guard g(h->device);
  return run_eig(h, X, Y, N, k, prec, evals, evecs);
}

hess_status hess_param_permutation(int L, const int* widths, int64_t* perm) {
  clear_error();
  if (L < 2 || !widths || !perm) return set_error(HESS_ERR_INVALID_ARG, "need L >= 2, widths, perm");
  int64_t o = 0, idx = 0;
  for (int w = 1; w < L; ++w) {
    int64_t tin = widths[w - 1], tout = widths[w];
    if (tin < 1 || tout < 1) return set_error(HESS_ERR_INVALID_ARG, "bad width");
    int64_t boff = o + tin * tout;
    for (int64_t i = 0; i < tout; ++i) {
      for (int64_t j = 0; j < tin; ++j) perm[idx++] = o + i * tin + j;
      perm[idx++] = boff + i;
    }
    o = boff + tout;
  }
  return HESS_OK;
}

hess_status hess_timing_enable(hess_mlp* h, int enable) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  h->timing = enable != 0;
  return HESS_OK;
}

hess_status hess_timing_read(hess_mlp* h, int cls, hess_kernel_stats* out) {
  clear_error();
  if (!h || !out || cls < 0 || cls >= HESS_K_COUNT)
    return set_error(HESS_ERR_INVALID_ARG, "bad handle, class or output");
  Guard g(h->device);
  HM_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& r : h->pending) {
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    hess_kernel_stats& a = h->acc[r.cls];
    a.launches += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
    a.sm_ms += (double)ms * (r.sms > 0 && r.sms < h->sm_count ? r.sms : h->sm_count);
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->pending.clear();
  *out = h->acc[cls];
  h->acc[cls] = hess_kernel_stats{};
  return HESS_OK;
}

int64_t hess_launch_count(void) { return g_launches.load(); }

const char* hess_last_error(void) { return g_err; }

}  // extern "C"
