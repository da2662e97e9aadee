// Top-k OPG eigenpairs for data sets whose N x P gradient matrix is not held
// at once (Sec. 5.4 computes them from mini-batches of examples; here
// uncentred, as Eq. J states): the examples are taken in chunks, the OPG of
// each chunk comes from opg() (so at most one chunk's gradients exist at a
// time), and the P x P FP64 sum
//
//   OPG = sum_c (n_c / N) OPG_c = (1/N) sum_n g_n g_n^T
//
// is then solved by the same FP64 Lanczos, tridiagonal eigensolver and
// checks as the Gram route, on the P x P matrix itself.  The route suits N
// larger than the Gram route allows (the N x N Gram matrix), with P^2 doubles
// resident.
#include "internal.h"

namespace hm {

namespace {

// M += w * C (n entries; C in FP32 or FP64)
template <typename T>
__global__ void axpy_kernel(double* M, const T* C, double w, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    M[i] = fma(w, (double)C[i], M[i]);
}

unsigned blocks_for(int64_t n) {
  int64_t b = cdiv(n, 256);
  if (b > 16384) b = 16384;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hess_status opg_topk_eig_streaming(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                              hess_precision prec, int64_t chunk, double* evals, double* evecs) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (N < 1 || N > ((int64_t)1 << 40)) return set_error(HESS_ERR_INVALID_ARG, "N must be in 1 .. 2^40");
  if (prec < HESS_FP64 || prec > HESS_BF16X3) return set_error(HESS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  const Net& net = h->net;
  const int64_t P = net.P, T1 = net.T[0], TL = net.T[net.L - 1];
  if (k < 1 || k > N || k > P)
    return set_error(HESS_ERR_INVALID_ARG, "need 1 <= k <= min(N, P) (k = %d, N = %lld, P = %lld)", k, (long long)N,
                     (long long)P);
  if (!X || !Y || !evals || !evecs) return set_error(HESS_ERR_INVALID_ARG, "X, Y, evals and evecs must be non-NULL");
  if (chunk < 1 || chunk > (1ll << 31) - 1)
    return set_error(HESS_ERR_INVALID_ARG, "chunk must be in 1 .. 2^31 - 1 (got %lld)", (long long)chunk);
  HM_TRY(take_sticky_error(h));
  Guard g(h->device);
  int ev_dev = 0, q_dev = 0;
  HM_TRY(locate(h, evals, "evals", &ev_dev));
  HM_TRY(locate(h, evecs, "evecs", &q_dev));
  const bool dbl = prec == HESS_FP64;
  const size_t es = dbl ? sizeof(double) : sizeof(float);
  // second workspace: the P x P FP64 sum, one chunk's OPG, and the outputs
  // when they are host buffers
  const size_t m_bytes = (size_t)P * P * sizeof(double);
  const size_t c_bytes = (size_t)P * P * es;
  const size_t o_bytes = (ev_dev ? 0 : (size_t)k * 8 + 256) + (q_dev ? 0 : (size_t)P * k * 8 + 256);
  HM_TRY(ensure_ws2(h, m_bytes + 256 + c_bytes + 256 + o_bytes));
  char* base = h->ws2;
  double* M = reinterpret_cast<double*>(base);
  void* C = base + align_up(m_bytes, 256);
  char* tail = base + align_up(m_bytes, 256) + align_up(c_bytes, 256);
  double* evd = ev_dev ? evals : reinterpret_cast<double*>(tail);
  double* eqd = q_dev ? evecs : reinterpret_cast<double*>(tail + (ev_dev ? 0 : align_up((size_t)k * 8, 256)));
  cudaStream_t s = h->stream;
  HM_CUDA(cudaMemsetAsync(M, 0, m_bytes, s));
  // the chunks' OPGs, each weighted by its share of the examples
  for (int64_t n0 = 0; n0 < N; n0 += chunk) {
    const int64_t nc = N - n0 < chunk ? N - n0 : chunk;
    const void* Xc = (const char*)X + (size_t)n0 * T1 * es;
    const void* Yc = (const char*)Y + (size_t)n0 * TL * es;
    HM_TRY(opg(h, Xc, Yc, nc, prec, C));
    const double w = (double)nc / (double)N;
    if (dbl)
      axpy_kernel<double><<<blocks_for(P * P), 256, 0, s>>>(M, (const double*)C, w, P * P);
    else
      axpy_kernel<float><<<blocks_for(P * P), 256, 0, s>>>(M, (const float*)C, w, P * P);
    HM_LAUNCHED();
  }
  // the eigenpairs of the P x P sum
  EigResult res;
  Arena ar;
  HM_TRY(topk_eig_dense(h, M, P, k, evd, eqd, ar, true, &res));
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  {
    Tick t(h, HESS_K_EIG, 0.0, 0.0);
    HM_TRY(topk_eig_dense(h, M, P, k, evd, eqd, ar, false, &res));
    t.set_work(res.flops, 0.0);
  }
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evals, evd, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(evecs, eqd, P * k * sizeof(double), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  HM_TRY(take_sticky_error(h));
  if (!res.converged)
    return set_error(HESS_ERR_NOT_CONVERGED, "Lanczos did not converge in %d steps", res.lanczos_steps);
  if (res.rank_deficient)
    return set_error(HESS_ERR_RANK_DEFICIENT, "some of the top-%d OPG eigenvalues are null", k);
  return HESS_OK;
}
