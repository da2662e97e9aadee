// Batched curvature matrices: the OPG and exact Hessian of many networks,
// each with its own data, contracted in waves of one persistent tensor-core
// launch each.
//
//   * the batch owns one device workspace, allocated at create time;
//   * a wave takes items in order while their planned operands (the same
//     layout the single-network call uses, found by a planning pass of
//     tc_prep) fit the workspace; each item's forward/backward pass, operand
//     builders and SIMT Hessian parts run on the batch stream, then one launch
//     walks the tiles of every job of every item in the wave, longest first;
//   * an item that does not fit the workspace even alone runs by itself
//     through the single-network call (chunked when its operands exceed its
//     handle's operand limit);
//   * the per-tile arithmetic does not depend on the schedule, so every matrix
//     is bit-identical to what the single-network call returns.
#include <algorithm>

#include "internal.h"

struct hess_batch {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  // CUDA-graph replay of repeated runs (same items and precision)
  struct GraphEntry {
    std::vector<hess_batch_item> items;
    int prec = -1;
    int seen = 0;                        // runs of this list so far
    cudaGraphExec_t exec = nullptr;
    std::vector<hm::PinnedStage> stages; // the graph's table copies read these
    hess_batch_info info{};
    int64_t kernels = 0;                 // kernels in the graph
    bool capturable = true;
  };
  bool graphs = false;
  cudaStream_t cap_stream = nullptr;     // capture stream (never the legacy one)
  std::vector<GraphEntry> cache;         // most recently used last
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int* err_host = nullptr;  // mapped pinned error flag of the tensor-core kernels
  int* err_dev = nullptr;
  hm::PinnedStage stage;
  std::vector<cudaEvent_t> events;  // pairs bracketing the wave launches
};

namespace hm {
namespace {

hess_status check_item(const hess_batch* b, const hess_batch_item& it, int idx) {
  if (!it.net) return set_error(HESS_ERR_INVALID_ARG, "item %d: network handle is NULL", idx);
  if (it.net->device != b->device)
    return set_error(HESS_ERR_INVALID_ARG, "item %d: network on device %d, batch on device %d", idx,
                     it.net->device, b->device);
  if (it.N < 1) return set_error(HESS_ERR_INVALID_ARG, "item %d: N must be >= 1", idx);
  if (!it.X || !it.Y) return set_error(HESS_ERR_INVALID_ARG, "item %d: X and Y must be non-NULL", idx);
  if (!it.opg && !it.hessian) return set_error(HESS_ERR_INVALID_ARG, "item %d: no output requested", idx);
  const void* ptrs[4] = {it.X, it.Y, it.opg, it.hessian};
  for (int q = 0; q < 4; ++q) {
    if (!ptrs[q]) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptrs[q]) != cudaSuccess) {
      cudaGetLastError();
      return set_error(HESS_ERR_INVALID_ARG, "item %d: buffers must be device memory", idx);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return set_error(HESS_ERR_INVALID_ARG, "item %d: buffers must be device memory", idx);
    if (at.type == cudaMemoryTypeDevice && at.device != b->device)
      return set_error(HESS_ERR_INVALID_ARG, "item %d: buffer on device %d, batch on device %d", idx,
                       at.device, b->device);
    if (reinterpret_cast<uintptr_t>(ptrs[q]) & 3)
      return set_error(HESS_ERR_INVALID_ARG, "item %d: buffers must be 4-byte aligned", idx);
  }
  return HESS_OK;
}

// Workspace bytes of one item inside a wave (its arena share).
size_t item_bytes(const hess_batch_item& it, TcPlan& plan) {
  Arena ar;
  TcItem ti{it.X, it.Y, it.N, it.opg != nullptr, it.hessian != nullptr, it.opg, it.hessian};
  tc_prep(it.net, ti, ar, false, plan, nullptr);
  return align_up(ar.off, 256);
}

// Bytes of a wave's job and tile tables (the layout tc_launch_plan takes).
size_t table_bytes(size_t njobs, size_t ntiles) {
  Arena ar;
  ar.take<tc::Job>(njobs ? njobs : 1);
  ar.take<int4>(ntiles ? ntiles : 1);
  return align_up(ar.off, 256);
}

// Runs one item alone through the single-network calls on the batch stream.
hess_status run_alone(hess_batch* b, const hess_batch_item& it, hess_precision prec) {
  hess_mlp* h = it.net;
  cudaStream_t keep = h->stream;
  h->stream = b->stream;
  hess_status st = HESS_OK;
  if (it.opg) st = opg(h, it.X, it.Y, it.N, prec, it.opg);
  if (st == HESS_OK && it.hessian) st = exact_hessian(h, it.X, it.Y, it.N, prec, it.hessian);
  if (st == HESS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
    st = set_error(HESS_ERR_CUDA, "batch stream: %s", cudaGetErrorString(cudaGetLastError()));
  if (st == HESS_OK) st = take_sticky_error(h);
  h->stream = keep;
  return st;
}

// Queues every wave of the run on stream s.  While capturing (stages given),
// each wave copies its tables from its own pinned buffer, which the graph
// keeps; an item too large for the workspace cannot be captured
// (HESS_ERR_UNSUPPORTED, nothing else queued).
hess_status enqueue_waves(hess_batch* b, const hess_batch_item* items, int count, hess_precision prec,
                          cudaStream_t s, std::vector<PinnedStage>* stages, hess_batch_info* infp) {
  hess_batch_info& inf = *infp;
  const bool x3 = prec == HESS_BF16X3;
    // fixed head of the workspace: split-K scratch
    Arena head{b->ws, 0};
    char* split = head.take<char>(kSplitBytes);
    const size_t base = align_up(head.off, 256);
    SplitGuard sg(split, kSplitBytes, b->sm_count);
    int i = 0;
    while (i < count) {
      // gather the wave
      size_t used = base, njobs = 0, ntiles = 0;
      int j = i;
      while (j < count) {
        TcPlan one;
        const size_t need = item_bytes(items[j], one);
        const size_t nj = njobs + one.jobs.size(), nt = ntiles + one.tiles.size();
        if (used + need + table_bytes(nj, nt) > b->ws_bytes) break;
        used += need;
        njobs = nj;
        ntiles = nt;
        ++j;
      }
      if (j == i) {
        // too large for the workspace: alone, through the single-network calls
        if (stages) return HESS_ERR_UNSUPPORTED;
        HM_TRY(run_alone(b, items[i], prec));
        ++inf.items_chunked;
        ++i;
        continue;
      }
      TcPlan plan;
      Arena ar{b->ws, base};
      for (int q = i; q < j; ++q) {
        const hess_batch_item& it = items[q];
        TcItem ti{it.X, it.Y, it.N, it.opg != nullptr, it.hessian != nullptr, it.opg, it.hessian, x3};
        const size_t at = ar.off;
        HM_TRY(tc_prep(it.net, ti, ar, true, plan, s));
        ar.off = at + align_up(ar.off - at, 256);
      }
      const size_t e0 = 2 * (size_t)inf.waves;
      while (b->events.size() < e0 + 2) {
        cudaEvent_t e;
        HM_CUDA(cudaEventCreate(&e));
        b->events.push_back(e);
      }
      // inside a capture the records become graph nodes (external records)
      const unsigned rec = stages ? cudaEventRecordExternal : cudaEventRecordDefault;
      HM_CUDA(cudaEventRecordWithFlags(b->events[e0], s, rec));
      PinnedStage* st = &b->stage;
      if (stages) {
        stages->emplace_back();
        st = &stages->back();
      }
      HM_TRY(tc_launch_plan(b->sm_count, plan, ar, true, x3, b->err_dev, *st, s));
      HM_CUDA(cudaEventRecordWithFlags(b->events[e0 + 1], s, rec));
      inf.tiles += (int64_t)plan.tiles.size();
      inf.flops += (plan.syrk_flops + plan.hess_flops) * (x3 ? 3.0 : 1.0);
      ++inf.waves;
      i = j;
    }
  return HESS_OK;
}

constexpr size_t kGraphCache = 8;  // item lists with a graph kept at once

bool same_items(const hess_batch::GraphEntry& g, const hess_batch_item* items, int count, hess_precision prec) {
  if ((int)g.items.size() != count || g.prec != (int)prec) return false;
  for (int i = 0; i < count; ++i) {
    const hess_batch_item& x = g.items[i];
    const hess_batch_item& y = items[i];
    if (x.net != y.net || x.X != y.X || x.Y != y.Y || x.N != y.N || x.opg != y.opg || x.hessian != y.hessian)
      return false;
  }
  return true;
}

void drop_entry(hess_batch::GraphEntry& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  for (auto& st : g.stages) stage_free(st);
  g.stages.clear();
}

void drop_graphs(hess_batch* b) {
  for (auto& g : b->cache) drop_entry(g);
  b->cache.clear();
}

// Captures the run's waves into a graph (on the capture stream, ordered
// after the user's stream).  HESS_ERR_UNSUPPORTED: the list cannot be
// captured (an item runs alone); nothing was queued.
hess_status capture(hess_batch* b, hess_batch::GraphEntry& g, const hess_batch_item* items, int count,
                    hess_precision prec) {
  cudaEvent_t dep;
  HM_CUDA(cudaEventCreateWithFlags(&dep, cudaEventDisableTiming));
  cudaEventRecord(dep, b->stream);
  cudaStreamWaitEvent(b->cap_stream, dep, 0);
  cudaEventDestroy(dep);
  HM_CUDA(cudaStreamSynchronize(b->cap_stream));
  std::vector<PinnedStage> stages;
  hess_batch_info ci{};
  const int64_t l0 = g_launches.load();
  // relaxed: the waves allocate their pinned table buffers while capturing
  HM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
  hess_status st = enqueue_waves(b, items, count, prec, b->cap_stream, &stages, &ci);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
  // captured kernels run when the graph does: count them then
  const int64_t kernels = g_launches.load() - l0;
  g_launches -= kernels;
  if (st != HESS_OK || ec != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    for (auto& x : stages) stage_free(x);
    if (st != HESS_OK) return st;
    return set_error(HESS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    for (auto& x : stages) stage_free(x);
    g.exec = nullptr;
    return set_error(HESS_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ei));
  }
  g.stages = std::move(stages);
  g.info = ci;
  g.kernels = kernels;
  return HESS_OK;
}

// One run: directly, or (graphs on, a list seen before) through its graph,
// captured on the second run of the list and replayed afterwards.
hess_status run_batch(hess_batch* b, const hess_batch_item* items, int count, hess_precision prec,
                      hess_batch_info* inf) {
  if (!b->graphs) return enqueue_waves(b, items, count, prec, b->stream, nullptr, inf);
  size_t at = b->cache.size();
  for (size_t i = 0; i < b->cache.size(); ++i)
    if (same_items(b->cache[i], items, count, prec)) at = i;
  if (at == b->cache.size()) {
    if (b->cache.size() >= kGraphCache) {
      drop_entry(b->cache.front());
      b->cache.erase(b->cache.begin());
    }
    hess_batch::GraphEntry g;
    g.items.assign(items, items + count);
    g.prec = (int)prec;
    b->cache.push_back(std::move(g));
    at = b->cache.size() - 1;
  } else if (at + 1 != b->cache.size()) {
    std::rotate(b->cache.begin() + at, b->cache.begin() + at + 1, b->cache.end());  // most recent last
    at = b->cache.size() - 1;
  }
  hess_batch::GraphEntry& g = b->cache[at];
  ++g.seen;
  if (g.seen < 2 || !g.capturable) return enqueue_waves(b, items, count, prec, b->stream, nullptr, inf);
  if (!g.exec) {
    const hess_status st = capture(b, g, items, count, prec);
    if (st == HESS_ERR_UNSUPPORTED) {
      g.capturable = false;
      return enqueue_waves(b, items, count, prec, b->stream, nullptr, inf);
    }
    HM_TRY(st);
  }
  HM_CUDA(cudaGraphLaunch(g.exec, b->stream));
  g_launches += g.kernels;
  *inf = g.info;
  inf->graph_replayed = 1;
  return HESS_OK;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

hess_status hess_batch_create(int64_t workspace_bytes, void* stream, hess_batch** out) {
  clear_error();
  if (!out) return set_error(HESS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (workspace_bytes < ((int64_t)kSplitBytes + (1 << 20)))
    return set_error(HESS_ERR_INVALID_ARG, "workspace must be at least %lld bytes",
                     (long long)(kSplitBytes + (1 << 20)));
  hess_batch* b = new hess_batch();
  b->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return set_error(HESS_ERR_CUDA, "no CUDA device");
  }
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (cudaMalloc(&b->ws, (size_t)workspace_bytes) != cudaSuccess ||
      cudaHostAlloc(&b->err_host, 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&b->err_dev, b->err_host, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->ws);
    if (b->err_host) cudaFreeHost(b->err_host);
    delete b;
    return set_error(HESS_ERR_OOM, "cannot allocate a %lld-byte batch workspace", (long long)workspace_bytes);
  }
  b->ws_bytes = (size_t)workspace_bytes;
  *b->err_host = 0;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->cap_stream = nullptr;  // graphs stay unavailable
  }
  *out = b;
  return HESS_OK;
}

hess_status hess_batch_run(hess_batch* b, const hess_batch_item* items, int count, hess_precision prec,
                           hess_batch_info* info) {
  clear_error();
  if (!b) return set_error(HESS_ERR_INVALID_ARG, "batch is NULL");
  if (count < 0 || (count > 0 && !items)) return set_error(HESS_ERR_INVALID_ARG, "bad item list");
  if (prec != HESS_BF16 && prec != HESS_BF16X3)
    return set_error(HESS_ERR_INVALID_ARG, "batches run on the tensor cores: precision BF16 or BF16X3");
  for (int i = 0; i < count; ++i) HM_TRY(check_item(b, items[i], i));
  Guard g(b->device);
  hess_batch_info inf{};
  if (count > 0) {
    HM_TRY(tc_available(items[0].net));
    HM_TRY(run_batch(b, items, count, prec, &inf));
    HM_CUDA(cudaStreamSynchronize(b->stream));
    if (*(volatile int*)b->err_host) {
      *(volatile int*)b->err_host = 0;
      return set_error(HESS_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
    }
    for (int w = 0; w < inf.waves; ++w) {
      float ms = 0.f;
      HM_CUDA(cudaEventElapsedTime(&ms, b->events[2 * w], b->events[2 * w + 1]));
      inf.launch_ms += ms;
    }
  }
  if (info) *info = inf;
  return HESS_OK;
}

hess_status hessian_minibatches(hess_mlp* h, const void* X, const void* Y, int64_t N, int64_t bs,
                                hess_precision prec, void* H) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (!X || !Y || !H) return set_error(HESS_ERR_INVALID_ARG, "X, Y and H must be non-NULL");
  if (N < 1 || N > (1ll << 31) - 1) return set_error(HESS_ERR_INVALID_ARG, "N must be in 1 .. 2^31 - 1");
  if (bs < 1) return set_error(HESS_ERR_INVALID_ARG, "the mini-batch size must be >= 1 (got %lld)", (long long)bs);
  if (prec < HESS_FP64 || prec > HESS_BF16X3) return set_error(HESS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  HM_TRY(take_sticky_error(h));
  const Net& net = h->net;
  const int64_t P = net.P, T1 = net.T[0], TL = net.T[net.L - 1];
  const int64_t nb = cdiv(N, bs);
  const size_t es = prec == HESS_FP64 ? sizeof(double) : sizeof(float);
  auto slice = [&](const void* base, int64_t b, int64_t per) {
    return (const void*)((const char*)base + (size_t)(b * bs) * per * es);
  };
  const bool tc = prec == HESS_BF16 || prec == HESS_BF16X3;
  int x_dev = 0, y_dev = 0, o_dev = 0;
  HM_TRY(locate(h, X, "X", &x_dev));
  HM_TRY(locate(h, Y, "Y", &y_dev));
  HM_TRY(locate(h, H, "H", &o_dev));
  if (!tc || !x_dev || !y_dev || !o_dev || nb == 1) {
    // the single call per mini-batch
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t n = N - b * bs < bs ? N - b * bs : bs;
      void* Hb = (char*)H + (size_t)b * P * P * es;
      HM_TRY(exact_hessian(h, slice(X, b, T1), slice(Y, b, TL), n, prec, Hb));
    }
    return HESS_OK;
  }
  Guard g(h->device);
  if (!h->mb_batch) {
    size_t fr = 0, tot = 0;
    HM_CUDA(cudaMemGetInfo(&fr, &tot));
    int64_t ws = (int64_t)4 << 30;
    if ((int64_t)(fr / 4) < ws) ws = (int64_t)(fr / 4);
    const int64_t floor_bytes = (int64_t)kSplitBytes + ((int64_t)256 << 20);
    if (ws < floor_bytes) ws = floor_bytes;
    HM_TRY(hess_batch_create(ws, h->stream, &h->mb_batch));
  }
  h->mb_batch->stream = h->stream;
  std::vector<hess_batch_item> items((size_t)nb);
  for (int64_t b = 0; b < nb; ++b) {
    hess_batch_item& it = items[(size_t)b];
    it.net = h;
    it.X = static_cast<const float*>(slice(X, b, T1));
    it.Y = static_cast<const float*>(slice(Y, b, TL));
    it.N = N - b * bs < bs ? N - b * bs : bs;
    it.opg = nullptr;
    it.hessian = reinterpret_cast<float*>((char*)H + (size_t)b * P * P * es);
  }
  if (nb > 1 << 30) return set_error(HESS_ERR_INVALID_ARG, "too many mini-batches");
  return hess_batch_run(h->mb_batch, items.data(), (int)nb, prec, nullptr);
}

hess_status hess_batch_set_graphs(hess_batch* b, int enable) {
  clear_error();
  if (!b) return set_error(HESS_ERR_INVALID_ARG, "batch is NULL");
  if (enable && !b->cap_stream) return set_error(HESS_ERR_CUDA, "no capture stream");
  Guard g(b->device);
  if (!enable) drop_graphs(b);
  b->graphs = enable != 0;
  return HESS_OK;
}

hess_status hess_batch_destroy(hess_batch* b) {
  if (!b) return HESS_OK;
  Guard g(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  cudaFree(b->ws);
  cudaFreeHost(b->err_host);
  stage_free(b->stage);
  delete b;
  return HESS_OK;
}

}  // extern "C"
