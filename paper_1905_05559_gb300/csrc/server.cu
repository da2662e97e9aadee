// Request server: continuous batching of Hessian, OPG and top-k eigenpair
// requests on one GPU.
//
//   * networks are registered once; their weights stay on the device and are
//     shared (borrowed, not copied) by every slot's handle;
//   * a slot = a worker thread + a CUDA stream + a workspace; admitted
//     requests run on different slots at the same time, so their kernels
//     overlap on the device;
//   * admission: requests wait in arrival order; the head request is started
//     as soon as a slot is free and its workspace (planned by a dry run of the
//     same call) fits the memory budget together with the workspaces the
//     other slots hold -- idle slots give theirs back when room is needed; a
//     request that cannot fit even alone is refused with HESS_ERR_ADMISSION.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "internal.h"

namespace hm {
namespace {

struct Ticket {
  hess_request req{};
  size_t bytes = 0;
  bool done = false;
  hess_status status = HESS_OK;
  char message[256] = {0};
  // device timestamps: recorded on the slot's stream before and after the
  // request's work (timing events; destroyed when the ticket is released)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ~Ticket() {
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

struct Slot {
  int id = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t cap = 0;
  bool busy = false;
  int64_t ticket = -1;
  std::map<int, hess_mlp*> views;  // per network: a handle borrowing its weights
  std::thread worker;
  std::condition_variable cv;
};

}  // namespace
}  // namespace hm

struct hess_server {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;  // queue / slot / completion changes
  std::vector<hess_mlp*> nets;
  std::vector<std::unique_ptr<hm::Slot>> slots;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<hm::Ticket>> tickets;
  int64_t next_ticket = 1;
  bool stopping = false;
  std::thread scheduler;
  cudaEvent_t ref = nullptr;  // completed at creation: the origin of request times
};

namespace hm {
namespace {

int64_t held_bytes(hess_server* sv) {
  int64_t s = 0;
  for (auto& sl : sv->slots) s += (int64_t)sl->cap;
  return s;
}

hess_status run_request(hess_mlp* h, const hess_request& r) {
  switch (r.kind) {
    case HESS_REQ_HESSIAN:
      return exact_hessian(h, r.X, r.Y, r.N, (hess_precision)r.prec, r.out);
    case HESS_REQ_OPG:
      return opg(h, r.X, r.Y, r.N, (hess_precision)r.prec, r.out);
    case HESS_REQ_EIG:
      return opg_topk_eig(h, r.X, r.Y, r.N, r.k, (hess_precision)r.prec, r.evals, (double*)r.out);
    default:
      return set_error(HESS_ERR_INVALID_ARG, "unknown request kind %d", r.kind);
  }
}

void worker_loop(hess_server* sv, Slot* sl) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    sl->cv.wait(lk, [&] { return sv->stopping || sl->ticket >= 0; });
    if (sl->ticket < 0 && sv->stopping) return;
    Ticket* t = sv->tickets[sl->ticket].get();
    hess_mlp* h = sl->views[t->req.net];
    h->ws = sl->ws;
    h->ws_bytes = sl->cap;
    lk.unlock();
    if (!t->ev0 && cudaEventCreate(&t->ev0) == cudaSuccess) cudaEventRecord(t->ev0, sl->stream);
    hess_status st = run_request(h, t->req);
    if (!t->ev1 && cudaEventCreate(&t->ev1) == cudaSuccess) cudaEventRecord(t->ev1, sl->stream);
    cudaGetLastError();
    if (st == HESS_OK || st == HESS_ERR_RANK_DEFICIENT) {
      cudaError_t e = cudaStreamSynchronize(sl->stream);
      if (e != cudaSuccess) st = set_error(HESS_ERR_CUDA, "request stream: %s", cudaGetErrorString(e));
      else if (take_sticky_error(h) != HESS_OK) st = HESS_ERR_TIMEOUT;
    }
    const char* msg = hess_last_error();
    lk.lock();
    // a call may have grown the workspace (it never shrinks it)
    sl->ws = h->ws;
    sl->cap = h->ws_bytes;
    h->ws = nullptr;
    h->ws_bytes = 0;
    t->status = st;
    snprintf(t->message, sizeof t->message, "%s", st == HESS_OK ? "" : msg);
    t->done = true;
    sl->ticket = -1;
    sl->busy = false;
    sv->cv.notify_all();
  }
}

void scheduler_loop(hess_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    sv->cv.wait(lk, [&] {
      if (sv->stopping) return true;
      if (sv->queue.empty()) return false;
      for (auto& sl : sv->slots)
        if (!sl->busy) return true;
      return false;
    });
    if (sv->stopping) return;
    const int64_t id = sv->queue.front();
    Ticket* t = sv->tickets[id].get();
    // prefer a free slot that already holds enough workspace
    Slot* pick = nullptr;
    for (auto& sl : sv->slots)
      if (!sl->busy && (!pick || (sl->cap >= t->bytes && pick->cap < t->bytes))) pick = sl.get();
    int64_t extra = (int64_t)t->bytes - (int64_t)pick->cap;
    if (extra > 0 && held_bytes(sv) + extra > sv->budget) {
      // idle slots give their workspaces back
      for (auto& sl : sv->slots) {
        if (sl.get() == pick || sl->busy || !sl->ws) continue;
        cudaFree(sl->ws);
        sl->ws = nullptr;
        sl->cap = 0;
        if (held_bytes(sv) + extra <= sv->budget) break;
      }
    }
    if (extra > 0 && held_bytes(sv) + extra > sv->budget) {
      // wait for a running request to finish and free memory
      sv->cv.wait(lk);
      continue;
    }
    if (extra > 0) {
      if (pick->ws) cudaFree(pick->ws);
      pick->ws = nullptr;
      pick->cap = 0;
      char* p = nullptr;
      if (cudaMalloc(&p, t->bytes) != cudaSuccess) {
        cudaGetLastError();
        sv->queue.pop_front();
        t->status = HESS_ERR_OOM;
        snprintf(t->message, sizeof t->message, "workspace of %zu bytes not available", t->bytes);
        t->done = true;
        sv->cv.notify_all();
        continue;
      }
      pick->ws = p;
      pick->cap = t->bytes;
    }
    sv->queue.pop_front();
    pick->busy = true;
    pick->ticket = id;
    pick->cv.notify_one();
  }
}

// Workspace bytes a request needs (dry run of the same call), 0 on error.
hess_status plan_request(hess_mlp* h, const hess_request& r, size_t* bytes) {
  size_t b = 0;
  g_dry_bytes = &b;
  hess_status st = run_request(h, r);
  g_dry_bytes = nullptr;
  if (st == kDryRun) {
    *bytes = b;
    return HESS_OK;
  }
  return st == HESS_OK ? set_error(HESS_ERR_INVALID_ARG, "request needs no planning") : st;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

hess_status hess_server_create(int slots, int64_t budget_bytes, hess_server** out) {
  clear_error();
  if (!out || slots < 1 || slots > 64 || budget_bytes <= 0)
    return set_error(HESS_ERR_INVALID_ARG, "need out, 1 <= slots <= 64 and a positive budget");
  *out = nullptr;
  auto* sv = new hess_server();
  sv->budget = budget_bytes;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return set_error(HESS_ERR_CUDA, "no CUDA device");
  }
  for (int i = 0; i < slots; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->id = i;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      sv->stopping = true;
      hess_server_destroy(sv);
      return set_error(HESS_ERR_CUDA, "cannot create a stream");
    }
    sv->slots.push_back(std::move(sl));
  }
  if (cudaEventCreate(&sv->ref) != cudaSuccess || cudaEventRecord(sv->ref, sv->slots[0]->stream) != cudaSuccess ||
      cudaEventSynchronize(sv->ref) != cudaSuccess) {
    cudaGetLastError();
    sv->stopping = true;
    hess_server_destroy(sv);
    return set_error(HESS_ERR_CUDA, "cannot record the server's reference event");
  }
  for (auto& sl : sv->slots) sl->worker = std::thread(worker_loop, sv, sl.get());
  sv->scheduler = std::thread(scheduler_loop, sv);
  *out = sv;
  return HESS_OK;
}

hess_status hess_server_add_network(hess_server* sv, const hess_mlp_desc* desc, const double* omega,
                                    int* net_id) {
  clear_error();
  if (!sv || !net_id) return set_error(HESS_ERR_INVALID_ARG, "server and net_id must be non-NULL");
  hess_mlp* master = nullptr;
  HM_TRY(hess_mlp_create(desc, omega, nullptr, &master));
  std::lock_guard<std::mutex> lk(sv->mu);
  const int id = (int)sv->nets.size();
  sv->nets.push_back(master);
  for (auto& sl : sv->slots) {
    auto* v = new hess_mlp();
    v->net = master->net;
    v->device = master->device;
    v->sm_count = master->sm_count;
    v->stream = sl->stream;
    v->omega64 = master->omega64;
    v->omega32 = master->omega32;
    v->owns_params = false;
    if (host_side_init(v) != HESS_OK) {
      cudaGetLastError();
      host_side_free(v);
      delete v;
      return set_error(HESS_ERR_OOM, "pinned scratch");
    }
    sl->views[id] = v;
  }
  *net_id = id;
  return HESS_OK;
}

hess_status hess_server_submit(hess_server* sv, const hess_request* req, int64_t* ticket) {
  clear_error();
  if (!sv || !req || !ticket) return set_error(HESS_ERR_INVALID_ARG, "server, request and ticket must be non-NULL");
  hess_mlp* master = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (req->net < 0 || req->net >= (int)sv->nets.size())
      return set_error(HESS_ERR_INVALID_ARG, "unknown network %d", req->net);
    master = sv->nets[req->net];
  }
  size_t bytes = 0;
  HM_TRY(plan_request(master, *req, &bytes));  // also validates the arguments
  if ((int64_t)bytes > sv->budget)
    return set_error(HESS_ERR_ADMISSION, "request needs %zu bytes of workspace, the budget is %lld",
                     bytes, (long long)sv->budget);
  auto t = std::make_unique<Ticket>();
  t->req = *req;
  t->bytes = bytes;
  std::lock_guard<std::mutex> lk(sv->mu);
  const int64_t id = sv->next_ticket++;
  sv->tickets[id] = std::move(t);
  sv->queue.push_back(id);
  sv->cv.notify_all();
  *ticket = id;
  return HESS_OK;
}

hess_status hess_server_wait(hess_server* sv, int64_t ticket, double timeout_seconds,
                             hess_status* result) {
  return hess_server_wait_timed(sv, ticket, timeout_seconds, result, nullptr, nullptr);
}

hess_status hess_server_wait_timed(hess_server* sv, int64_t ticket, double timeout_seconds,
                                   hess_status* result, double* gpu_start_ms, double* gpu_end_ms) {
  clear_error();
  if (!sv || !result) return set_error(HESS_ERR_INVALID_ARG, "server and result must be non-NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return set_error(HESS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  Ticket* t = it->second.get();
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_seconds < 0 ? 1e9 : timeout_seconds));
  if (!sv->cv.wait_until(lk, deadline, [&] { return t->done; }))
    return set_error(HESS_ERR_TIMEOUT, "ticket %lld not finished", (long long)ticket);
  *result = t->status;
  if (gpu_start_ms || gpu_end_ms) {
    float a = -1.0f, b = -1.0f;
    if (!t->ev0 || !t->ev1 || cudaEventSynchronize(t->ev1) != cudaSuccess ||
        cudaEventElapsedTime(&a, sv->ref, t->ev0) != cudaSuccess ||
        cudaEventElapsedTime(&b, sv->ref, t->ev1) != cudaSuccess) {
      cudaGetLastError();
      a = b = -1.0f;
    }
    if (gpu_start_ms) *gpu_start_ms = a;
    if (gpu_end_ms) *gpu_end_ms = b;
  }
  if (t->status != HESS_OK) set_error(t->status, "%s", t->message);
  sv->tickets.erase(it);
  return HESS_OK;
}

hess_status hess_server_destroy(hess_server* sv) {
  if (!sv) return HESS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
    sv->cv.notify_all();
    for (auto& sl : sv->slots) sl->cv.notify_all();
  }
  if (sv->scheduler.joinable()) sv->scheduler.join();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int64_t id : sv->queue) {
      Ticket* t = sv->tickets[id].get();
      t->status = HESS_ERR_INVALID_ARG;
      snprintf(t->message, sizeof t->message, "server destroyed before the request started");
      t->done = true;
    }
    sv->queue.clear();
    sv->cv.notify_all();
  }
  for (auto& sl : sv->slots) {
    if (sl->worker.joinable()) sl->worker.join();
  }
  cudaSetDevice(sv->device);
  for (auto& sl : sv->slots) {
    for (auto& kv : sl->views) {
      kv.second->ws = nullptr;
      hess_mlp_destroy(kv.second);
    }
    if (sl->ws) cudaFree(sl->ws);
    if (sl->stream) cudaStreamDestroy(sl->stream);
  }
  sv->tickets.clear();
  if (sv->ref) cudaEventDestroy(sv->ref);
  for (auto* n : sv->nets) hess_mlp_destroy(n);
  cudaGetLastError();
  delete sv;
  return HESS_OK;
}

}  // extern "C"
