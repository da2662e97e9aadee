// All curvature matrices of one network and one data set in one call, with
// the work of the three on five streams:
//
//   stream A (the handle's)    : forward/backward, the tensor-core operands
//                                and the contractions of the OPG and the
//                                Hessian (FP32 / split-BF16)
//   stream B (the handle's 2nd): the FP64 forward/backward, Gram matrix,
//                                Lanczos launches, tridiagonal eigenpairs and
//                                back-projection
//   streams C and D (3rd, 4th): each matrix's copy to a host buffer, queued
//                                behind its contraction, in two halves (one
//                                per stream, so that two copy engines share
//                                each transfer)
//   stream E (5th)             : the Hessian's tensor-core operands (R-operator
//                                blocks, W rows, F planes), behind A's
//                                forward/backward pass (the Hessian's
//                                contraction waits for them, the OPG's does
//                                not); then the eigen step's side work (the
//                                back-projection's digit split of the
//                                activations, its narrow layers)
//
// Stream B has the higher priority: the eigen step is the longer chain of
// short launches, and its blocks are scheduled first when both streams have
// work waiting.  The contractions fill the SMs around it.  (Holding the
// contractions back until the Lanczos launches are done measured slower.)
// Host outputs are written to device memory and copied by the copy engines,
// so that the OPG's transfer overlaps the Hessian's contraction and both
// overlap the eigen step.  The streams use separate regions of the handle's
// workspace (and separate split-K scratch).
#include <algorithm>
#include <functional>

#include "internal.h"

using namespace hm;

namespace {

// Device memory (on the handle's device) or not.
hess_status on_device(const hess_mlp* h, const void* p, bool* dev) {
  cudaPointerAttributes at;
  *dev = false;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return HESS_OK;
  }
  if (at.type == cudaMemoryTypeDevice && at.device != h->device)
    return set_error(HESS_ERR_INVALID_ARG, "buffer on device %d, handle on device %d", at.device, h->device);
  *dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  return HESS_OK;
}

}  // namespace

extern "C" hess_status hess_curvature(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec,
                                      void* OPG, void* H, int k, double* evals, double* evecs) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (!X || !Y) return set_error(HESS_ERR_INVALID_ARG, "X and Y must be non-NULL");
  if (N < 1 || N > (1ll << 31) - 1) return set_error(HESS_ERR_INVALID_ARG, "N must be in 1 .. 2^31 - 1");
  if (prec < HESS_FP64 || prec > HESS_BF16X3) return set_error(HESS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  if (!OPG && !H && k == 0) return set_error(HESS_ERR_INVALID_ARG, "no output requested");
  const Net& net = h->net;
  const int64_t P = net.P;
  if (k < 0 || (k > 0 && (!evals || !evecs || k > N || k > P)))
    return set_error(HESS_ERR_INVALID_ARG, "k must be 0, or 1 .. min(N, P) with evals and evecs");
  HM_TRY(take_sticky_error(h));
  const bool tc = prec == HESS_BF16 || prec == HESS_BF16X3;
  if (!tc || k == 0 || (!OPG && !H)) {
    // nothing to overlap: the single calls in turn
    if (OPG) HM_TRY(opg(h, X, Y, N, prec, OPG));
    if (H) HM_TRY(exact_hessian(h, X, Y, N, prec, H));
    if (k > 0) return opg_topk_eig(h, X, Y, N, k, prec, evals, evecs);
    return HESS_OK;
  }
  Guard g(h->device);
  HM_TRY(tc_available(h));
  const bool x3 = prec == HESS_BF16X3;
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1];
  bool x_dev, y_dev, o_dev = true, hh_dev = true, ev_dev, q_dev;
  HM_TRY(on_device(h, X, &x_dev));
  HM_TRY(on_device(h, Y, &y_dev));
  if (OPG) HM_TRY(on_device(h, OPG, &o_dev));
  if (H) HM_TRY(on_device(h, H, &hh_dev));
  HM_TRY(on_device(h, evals, &ev_dev));
  HM_TRY(on_device(h, evecs, &q_dev));
  const bool host_io = !x_dev || !y_dev || !o_dev || !hh_dev || !ev_dev || !q_dev;
  if (!h->stream2) {
    int lo = 0, hi = 0;
    HM_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    HM_CUDA(cudaStreamCreateWithPriority(&h->stream2, cudaStreamNonBlocking, hi));
  }
  if (!h->stream3) HM_CUDA(cudaStreamCreateWithFlags(&h->stream3, cudaStreamNonBlocking));
  if (!h->stream4) HM_CUDA(cudaStreamCreateWithFlags(&h->stream4, cudaStreamNonBlocking));
  if (!h->stream5) HM_CUDA(cudaStreamCreateWithFlags(&h->stream5, cudaStreamNonBlocking));
  const cudaStream_t sA = h->stream, sB = h->stream2, sC = h->stream3, sD = h->stream4, sE = h->stream5;
  // the persistent contractions take the SMs the eigen step's Lanczos
  // launches leave free, so that the two overlap -- unless a matrix goes to
  // a host buffer: then its copy (the longest part of such a call) should
  // start as early as possible, and the contractions run first on every SM
  const int lz_g = eig_lanczos_blocks(h, N, k);
  const bool host_out = (OPG && !o_dev) || (H && !hh_dev);
  const int sm_tc = (lz_g < h->sm_count && !host_out) ? h->sm_count - lz_g : h->sm_count;
  // a device matrix to the host in two halves, one per copy stream, both
  // behind event e of stream A
  auto to_host = [&](void* dstv, const float* src, cudaEvent_t e) -> hess_status {
    float* dst = static_cast<float*>(dstv);
    const int64_t n = P * P, half = n / 2;
    HM_CUDA(cudaEventRecord(e, sA));
    HM_CUDA(cudaStreamWaitEvent(sC, e, 0));
    HM_CUDA(cudaStreamWaitEvent(sD, e, 0));
    HM_CUDA(cudaMemcpyAsync(dst, src, half * 4, cudaMemcpyDeviceToHost, sC));
    HM_CUDA(cudaMemcpyAsync(dst + half, src + half, (n - half) * 4, cudaMemcpyDeviceToHost, sD));
    return HESS_OK;
  };
  auto drain_copies = [&]() {
    cudaStreamSynchronize(sC);
    cudaStreamSynchronize(sD);
    cudaStreamSynchronize(sE);
  };

  // ---- workspace: region A (tensor-core operands and tables), region B
  // (the eigen step); the planning pass and the live pass take the same
  // sizes in the same order
  float *xs = nullptr, *ys = nullptr, *os = nullptr, *hs = nullptr;
  double *xd = nullptr, *yd = nullptr, *evd = nullptr, *eqd = nullptr;
  char *splitA = nullptr, *splitB = nullptr;
  size_t tabO = 0, tabH = 0, offEig = 0;
  Caches<double> c64;
  TcPlan plan_o, plan_h;
  EigResult res;
  cudaEvent_t ev_in = nullptr, ev_fb = nullptr;
  // ---- workspace, in the order taken: the inputs' and eigen step's buffers
  // (head), the contraction operands and tables (prep), the eigen step's own
  // scratch; the planning pass and the live pass take the same sizes
  auto head = [&](Arena& ar, bool live) -> hess_status {
    xs = x_dev ? (float*)X : ar.take<float>(N * T1);
    ys = y_dev ? (float*)Y : ar.take<float>(N * TL);
    os = OPG ? (o_dev ? (float*)OPG : ar.take<float>(P * P)) : nullptr;
    hs = H ? (hh_dev ? (float*)H : ar.take<float>(P * P)) : nullptr;
    splitA = ar.take<char>(kSplitBytes);
    xd = ar.take<double>(N * T1);
    yd = ar.take<double>(N * TL);
    plan_caches(ar, net, N, c64);
    evd = ev_dev ? evals : ar.take<double>(k);
    eqd = q_dev ? evecs : ar.take<double>(P * (int64_t)k);
    splitB = ar.take<char>(kSplitBytes);
    if (live) {
      if (!x_dev) HM_CUDA(cudaMemcpyAsync(xs, X, N * T1 * 4, cudaMemcpyHostToDevice, sA));
      if (!y_dev) HM_CUDA(cudaMemcpyAsync(ys, Y, N * TL * 4, cudaMemcpyHostToDevice, sA));
      // stream B may start once the inputs are on the device (and after
      // earlier work on the handle's stream): its FP64 forward/backward pass
      // (the head of the eigen step, the call's longest chain) goes first,
      // and stream A's preparation of the contraction operands waits for
      // it instead of sharing the SMs with it
      HM_CUDA(cudaEventRecord(ev_in, sA));
      HM_CUDA(cudaStreamWaitEvent(sB, ev_in, 0));
      SplitGuard sg(splitB, kSplitBytes, h->sm_count);
      HM_TRY(convert(xs, xd, N * T1, sB));
      HM_TRY(convert(ys, yd, N * TL, sB));
      HM_TRY(forward_backward(net, (const double*)h->omega64, (const double*)xd, (const double*)yd, c64, sB, true));
      HM_CUDA(cudaEventRecord(ev_fb, sB));
      HM_CUDA(cudaStreamWaitEvent(sA, ev_fb, 0));
    }
    return HESS_OK;
  };
  // the Hessian's operands are prepared on stream E (behind the FP32
  // forward/backward pass on A), so that the OPG's contraction starts as
  // soon as its own operands and the Gram matrix are ready
  TcFork fork;
  fork.s = sE;
  auto prep = [&](Arena& ar, bool live) -> hess_status {
    {
      // one preparation (one forward/backward pass) for both matrices, then
      // the OPG's job and the Hessian's jobs as two launches, so that the
      // OPG's copy can start while the Hessian is contracted
      SplitGuard sg(splitA, kSplitBytes, h->sm_count);
      TcPlan both;
      HM_TRY(tc_prep(h, TcItem{xs, ys, N, OPG != nullptr, H != nullptr, os, hs, x3}, ar, live, both, sA,
                     live && H ? &fork : nullptr));
      tc_split_plan(both, OPG ? 1 : 0, plan_o, plan_h);
    }
    tabO = ar.off;
    HM_TRY(tc_launch_plan(sm_tc, plan_o, ar, false, x3, h->err_dev, h->stage, sA));
    tabH = ar.off;
    HM_TRY(tc_launch_plan(sm_tc, plan_h, ar, false, x3, h->err_dev, h->stage, sA));
    return HESS_OK;
  };
  for (cudaEvent_t& e : h->fused_ev)
    if (!e) HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEvent_t* const ev = h->fused_ev;
  ev_in = ev[0];
  ev_fb = ev[6];
  fork.after_fb = ev[7];
  fork.done = ev[8];
  // the eigen step's side work goes to stream E too, behind the Hessian's
  // operands
  EigSide eside;
  eside.s = sE;
  for (int i = 0; i < 4; ++i) eside.ev[i] = ev[9 + i];
  eside.gram_done = ev[1];
  // the planning pass, or its result for a call of the same shape
  const int64_t key[16] = {N, (int64_t)prec, k, OPG ? 1 : 0, H ? 1 : 0, x_dev, y_dev, o_dev, hh_dev, ev_dev,
                           q_dev, sm_tc, (int64_t)h->op_limit, h->lz_blocks, P, 0};
  size_t offPrep = 0;
  if (h->fplan.valid && std::equal(key, key + 16, h->fplan.key)) {
    offPrep = h->fplan.off_prep;
    offEig = h->fplan.off_eig;
    HM_TRY(ensure_ws(h, h->fplan.ws));
  } else {
    h->fplan.valid = false;
    Arena ar;
    HM_TRY(head(ar, false));
    offPrep = ar.off;
    HM_TRY(prep(ar, false));
    offEig = ar.off;
    HM_TRY(topk_eig_gram(h, net, c64, N, k, evd, eqd, ar, true, &res));
    HM_TRY(ensure_ws(h, ar.off));
    std::copy(key, key + 16, h->fplan.key);
    h->fplan.ws = ar.off;
    h->fplan.off_prep = offPrep;
    h->fplan.off_eig = offEig;
    h->fplan.valid = true;
  }
  plan_o = TcPlan{};
  plan_h = TcPlan{};
  {
    Arena ar{h->ws, 0};
    HM_TRY(head(ar, true));  // queues A's input staging and B's forward/backward
  }
  // A's operand preparation (queued on A, with A's timing)
  auto prep_live = [&]() -> hess_status {
    cudaStream_t keep = h->stream;
    h->stream = sA;
    Arena ar{h->ws, offPrep};
    const hess_status st = prep(ar, true);
    h->stream = keep;
    return st;
  };

  // stream A: the contractions, right behind their operands (queued with the
  // handle's stream set to A, so that their timing runs there)
  hess_status tc_status = HESS_OK;
  auto contractions = [&]() -> hess_status {
    cudaStream_t keep = h->stream;
    h->stream = sA;
    if (OPG) {
      Tick t(h, HESS_K_SYRK, plan_o.syrk_flops, 0.0);
      t.set_sms(sm_tc);
      Arena at{h->ws, tabO};
      tc_status = tc_launch_plan(sm_tc, plan_o, at, true, x3, h->err_dev, h->stage, sA);
    }
    hess_status st = HESS_OK;
    if (OPG && !o_dev && tc_status == HESS_OK) st = to_host(OPG, os, ev[2]);
    if (H && tc_status == HESS_OK && st == HESS_OK) {
      HM_CUDA(cudaStreamWaitEvent(sA, fork.done, 0));  // its operands (stream E)
      Tick t(h, HESS_K_HCONTRACT, plan_h.hess_flops, 0.0);
      t.set_sms(sm_tc);
      Arena at{h->ws, tabH};
      tc_status = tc_launch_plan(sm_tc, plan_h, at, true, x3, h->err_dev, h->stage, sA);
    }
    if (H && !hh_dev && tc_status == HESS_OK && st == HESS_OK) st = to_host(H, hs, ev[3]);
    h->stream = keep;
    return tc_status != HESS_OK ? tc_status : st;
  };
  // When the Lanczos launches leave SMs free, the contractions wait for the
  // Gram matrix (whose exact-digit product wants every SM) and then run on
  // the free SMs beside the Lanczos launches; otherwise they are queued at
  // once and interleave with the eigen step.
  const bool overlap = sm_tc < h->sm_count;
  // (the host builds A's operand preparation there, once the GPU has B's
  // forward/backward pass, Gram matrix and first Lanczos launch queued; the
  // contractions wait for the Gram matrix, ev[1] on B)
  std::function<hess_status()> after_gram = [&]() -> hess_status {
    HM_TRY(prep_live());
    HM_CUDA(cudaStreamWaitEvent(sA, ev[1], 0));
    return contractions();
  };
  if (!overlap) {
    hess_status st = prep_live();
    if (st == HESS_OK) st = contractions();
    if (st != HESS_OK) {
      cudaStreamSynchronize(sB);
      drain_copies();
      return st;
    }
  }

  // ---- stream B: the eigen step (the handle's stream is B meanwhile, so that
  // the eigen kernels and their timing run there)
  hess_status eig_status = HESS_OK;
  h->stream = sB;
  {
    // (the caches of the eigen step were formed on stream B at the start)
    SplitGuard sg(splitB, kSplitBytes, h->sm_count);
    {
      Tick t(h, HESS_K_EIG, 0.0, 0.0);
      Arena are{h->ws, offEig};
      eig_status = topk_eig_gram(h, net, c64, N, k, evd, eqd, are, false, &res, overlap ? &after_gram : nullptr,
                                 &eside);
      t.set_work(res.flops, 0.0);
    }
  }
  h->stream = sA;
  if (eig_status == HESS_OK && tc_status != HESS_OK) eig_status = tc_status;
  if (eig_status != HESS_OK) {
    cudaStreamSynchronize(sB);  // nothing of B or the copies may run past the call
    drain_copies();
    return eig_status;
  }
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evals, evd, k * sizeof(double), cudaMemcpyDeviceToHost, sB));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(evecs, eqd, P * k * sizeof(double), cudaMemcpyDeviceToHost, sB));
  // stream A ends after everything of B and C
  HM_CUDA(cudaEventRecord(ev[1], sB));
  HM_CUDA(cudaStreamWaitEvent(sA, ev[1], 0));
  HM_CUDA(cudaEventRecord(ev[4], sC));
  HM_CUDA(cudaStreamWaitEvent(sA, ev[4], 0));
  HM_CUDA(cudaEventRecord(ev[5], sD));
  HM_CUDA(cudaStreamWaitEvent(sA, ev[5], 0));
  if (host_io) {
    HM_CUDA(cudaStreamSynchronize(sA));
    HM_TRY(take_sticky_error(h));
  }
  if (!res.converged)
    return set_error(HESS_ERR_NOT_CONVERGED, "Lanczos did not converge in %d steps", res.lanczos_steps);
  if (res.rank_deficient)
    return set_error(HESS_ERR_RANK_DEFICIENT, "some of the top-%d OPG eigenvalues are null", k);
  return HESS_OK;
}
