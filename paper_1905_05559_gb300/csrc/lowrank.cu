// Low-rank and full-rank approximations of a curvature matrix from K of its
// eigenpairs (Sec. 4.1, 4.2), formed (Sec. 5.5, 5.6 first forms) or applied
// without forming them (Sec. 5.5, 5.6 implicit forms).
//
// With w_k = lam_k - s, s = lam_tilde for the full-rank form and 0 otherwise:
//   H~ (or H~~) = Q^T diag(w) Q + s I           (Q: K rows of P)
//   H~ x        = Q^T (w o (Q x)) + s x
//   x^T H~ x    = sum_k w_k (q_k . x)^2 + s ||x||^2
// which is the paper's H~ + lam_tilde (I - Q Q^T) rearranged (Q Q^T = I on
// the span of the eigenvectors).
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace hm {

namespace {

// out[k][p] = (lam_k - s) Q[k][p] in precision T
template <typename T>
__global__ void weight_rows_kernel(const double* Q, const double* lam, double s, int K, int64_t P, T* out) {
  const int64_t n = (int64_t)K * P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)((lam[i / P] - s) * Q[i]);
}

template <typename T>
__global__ void add_diag_kernel(T* C, int64_t P, T v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    C[i * P + i] += v;
}

// quad_i = sum_k (lam_k - s) C[k][i]^2 + s ||x_i||^2, one warp per vector;
// then C[k][i] *= lam_k - s for the product (each warp scales its column).
__global__ void quad_scale_kernel(const double* X, int64_t P, double* C, const double* lam, double s, int K, int b,
                                  double* quad) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= b) return;
  double xx = 0.0;
  if (s != 0.0) {
    const double* x = X + (int64_t)i * P;
    double a0 = 0.0, a1 = 0.0;
    int64_t p = lane;
    for (; p + 32 < P; p += 64) {
      a0 = fma(x[p], x[p], a0);
      a1 = fma(x[p + 32], x[p + 32], a1);
    }
    if (p < P) a0 = fma(x[p], x[p], a0);
    xx = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);
  }
  double qq = 0.0;
  for (int k = lane; k < K; k += 32) {
    const double c = C[(int64_t)k * b + i];
    const double w = lam[k] - s;
    qq = fma(w * c, c, qq);
    C[(int64_t)k * b + i] = w * c;
  }
  for (int o = 16; o > 0; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
  if (lane == 0 && quad) quad[i] = qq + s * xx;
}

__global__ void scale_copy_kernel(const double* X, double a, int64_t n, double* Y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = a * X[i];
}

unsigned blocks_for(int64_t n) {
  int64_t b = cdiv(n, 256);
  if (b > 8192) b = 8192;
  return (unsigned)(b < 1 ? 1 : b);
}

// The shift s of the full-rank form (lam_K for NaN), read from the host or
// device eigenvalues.
hess_status shift_of(hess_mlp* h, int full, double lam_tilde, const double* evals, int ev_dev, int K, double* s) {
  *s = 0.0;
  if (!full) return HESS_OK;
  if (!std::isnan(lam_tilde)) {
    *s = lam_tilde;
    return HESS_OK;
  }
  if (ev_dev) {
    // in stream order after the work that produced the eigenvalues
    HM_CUDA(cudaMemcpyAsync(h->host_pinned, evals + K - 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    *s = h->host_pinned[0];
  } else {
    *s = evals[K - 1];
  }
  return HESS_OK;
}

hess_status check_eigs(hess_mlp* h, int K, const double* evals, const double* evecs) {
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (!evals || !evecs) return set_error(HESS_ERR_INVALID_ARG, "evals and evecs must be non-NULL");
  if (K < 1 || K > h->net.P)
    return set_error(HESS_ERR_INVALID_ARG, "need 1 <= K <= P (K = %d, P = %lld)", K, (long long)h->net.P);
  return take_sticky_error(h);
}

template <typename T>
hess_status run_form(hess_mlp* h, int K, const double* evals, const double* evecs, int full, double lam_tilde,
                     void* out) {
  const int64_t P = h->net.P;
  int ev_dev, q_dev, o_dev;
  HM_TRY(locate(h, evals, "evals", &ev_dev));
  HM_TRY(locate(h, evecs, "evecs", &q_dev));
  HM_TRY(locate(h, out, "out", &o_dev));
  double s = 0.0;
  HM_TRY(shift_of(h, full, lam_tilde, evals, ev_dev, K, &s));
  constexpr bool dbl = std::is_same<T, double>::value;
  double *evd, *qd;
  T *qw, *qt, *od;
  auto plan = [&](Arena& ar) {
    evd = ev_dev ? (double*)evals : ar.take<double>(K);
    qd = q_dev ? (double*)evecs : ar.take<double>(P * (int64_t)K);
    qw = ar.take<T>(P * (int64_t)K);
    qt = dbl ? nullptr : ar.take<T>(P * (int64_t)K);
    od = o_dev ? (T*)out : ar.take<T>(P * P);
  };
  Arena ar;
  plan(ar);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar);
  cudaStream_t st = h->stream;
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evd, evals, K * sizeof(double), cudaMemcpyHostToDevice, st));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(qd, evecs, P * K * sizeof(double), cudaMemcpyHostToDevice, st));
  {
    Tick t(h, HESS_K_APPROX, (double)P * (P + 1) * K, 0.0);
    weight_rows_kernel<T><<<blocks_for(P * K), 256, 0, st>>>(qd, evd, s, K, P, qw);
    HM_LAUNCHED();
    if (!dbl) {
      HM_TRY(convert(qd, (float*)qt, P * K, st));
    }
    Gemm<T> g;  // upper tiles of Qw^T Q
    g.M = (int)P;
    g.N = (int)P;
    g.K = K;
    g.A = qw;
    g.sam = 1;
    g.sak = P;
    g.B = dbl ? (const T*)qd : (const T*)qt;
    g.sbk = P;
    g.sbn = 1;
    g.C = od;
    g.scm = P;
    g.scn = 1;
    g.upper = 1;
    HM_TRY(gemm(g, st));
    HM_TRY(mirror_upper(od, P, P, st));
    if (s != 0.0) {
      add_diag_kernel<T><<<blocks_for(P), 256, 0, st>>>(od, P, (T)s);
      HM_LAUNCHED();
    }
  }
  if (!o_dev) HM_CUDA(cudaMemcpyAsync(out, od, P * P * sizeof(T), cudaMemcpyDeviceToHost, st));
  if (!ev_dev || !q_dev || !o_dev) {
    HM_CUDA(cudaStreamSynchronize(st));
    HM_TRY(take_sticky_error(h));
  }
  return HESS_OK;
}

hess_status run_apply(hess_mlp* h, int K, const double* evals, const double* evecs, int full, double lam_tilde,
                      const double* X, int b, double* HX, double* quad) {
  const int64_t P = h->net.P;
  int ev_dev, q_dev, x_dev, o_dev = 1, u_dev = 1;
  HM_TRY(locate(h, evals, "evals", &ev_dev));
  HM_TRY(locate(h, evecs, "evecs", &q_dev));
  HM_TRY(locate(h, X, "X", &x_dev));
  if (HX) HM_TRY(locate(h, HX, "HX", &o_dev));
  if (quad) HM_TRY(locate(h, quad, "quad", &u_dev));
  double s = 0.0;
  HM_TRY(shift_of(h, full, lam_tilde, evals, ev_dev, K, &s));
  double *evd, *qd, *xd, *od = nullptr, *ud = nullptr, *C;
  char* split = nullptr;
  auto plan = [&](Arena& ar) {
    evd = ev_dev ? (double*)evals : ar.take<double>(K);
    qd = q_dev ? (double*)evecs : ar.take<double>(P * (int64_t)K);
    xd = x_dev ? (double*)X : ar.take<double>(P * (int64_t)b);
    if (HX) od = o_dev ? HX : ar.take<double>(P * (int64_t)b);
    if (quad) ud = u_dev ? quad : ar.take<double>(b);
    C = ar.take<double>((int64_t)K * b);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  plan(ar);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar);
  SplitGuard sg(split, kSplitBytes, h->sm_count);  // Q X^T splits its long K
  cudaStream_t st = h->stream;
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evd, evals, K * sizeof(double), cudaMemcpyHostToDevice, st));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(qd, evecs, P * K * sizeof(double), cudaMemcpyHostToDevice, st));
  if (!x_dev) HM_CUDA(cudaMemcpyAsync(xd, X, P * b * sizeof(double), cudaMemcpyHostToDevice, st));
  {
    Tick t(h, HESS_K_APPROX, (HX ? 4.0 : 2.0) * P * K * b, 0.0);
    Gemm<double> g;  // C = Q X^T: K x b
    g.M = K;
    g.N = b;
    g.K = (int)P;
    g.A = qd;
    g.sam = P;
    g.sak = 1;
    g.B = xd;
    g.sbk = 1;
    g.sbn = P;
    g.C = C;
    g.scm = b;
    g.scn = 1;
    HM_TRY(gemm(g, st));
    quad_scale_kernel<<<(unsigned)cdiv(b, 8), 256, 0, st>>>(xd, P, C, evd, s, K, b, ud);
    HM_LAUNCHED();
    if (HX) {
      if (s != 0.0) {
        scale_copy_kernel<<<blocks_for(P * b), 256, 0, st>>>(xd, s, P * b, od);
        HM_LAUNCHED();
      }
      Gemm<double> p;  // HX = (w o C)^T Q (+ s X)
      p.M = b;
      p.N = (int)P;
      p.K = K;
      p.beta = s != 0.0 ? 1.0 : 0.0;
      p.A = C;
      p.sam = 1;
      p.sak = b;
      p.B = qd;
      p.sbk = P;
      p.sbn = 1;
      p.C = od;
      p.scm = P;
      p.scn = 1;
      HM_TRY(gemm(p, st));
    }
  }
  if (HX && !o_dev) HM_CUDA(cudaMemcpyAsync(HX, od, P * b * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (quad && !u_dev) HM_CUDA(cudaMemcpyAsync(quad, ud, b * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (!ev_dev || !q_dev || !x_dev || !o_dev || !u_dev) {
    HM_CUDA(cudaStreamSynchronize(st));
    HM_TRY(take_sticky_error(h));
  }
  return HESS_OK;
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hess_status hess_approx_form(hess_mlp* h, int K, const double* evals, const double* evecs, int full,
                                        double lam_tilde, hess_precision prec, void* out) {
  clear_error();
  HM_TRY(check_eigs(h, K, evals, evecs));
  if (!out) return set_error(HESS_ERR_INVALID_ARG, "out must be non-NULL");
  if (prec != HESS_FP64 && prec != HESS_FP32)
    return set_error(prec == HESS_BF16 || prec == HESS_BF16X3 ? HESS_ERR_UNSUPPORTED : HESS_ERR_INVALID_ARG,
                     "the approximations are formed in FP64 or FP32 (precision %d)", (int)prec);
  Guard g(h->device);
  if (prec == HESS_FP64) return run_form<double>(h, K, evals, evecs, full, lam_tilde, out);
  return run_form<float>(h, K, evals, evecs, full, lam_tilde, out);
}

extern "C" hess_status hess_approx_apply(hess_mlp* h, int K, const double* evals, const double* evecs, int full,
                                         double lam_tilde, const double* X, int b, double* HX, double* quad) {
  clear_error();
  HM_TRY(check_eigs(h, K, evals, evecs));
  if (!X) return set_error(HESS_ERR_INVALID_ARG, "X must be non-NULL");
  if (b < 1) return set_error(HESS_ERR_INVALID_ARG, "b must be >= 1 (got %d)", b);
  if (!HX && !quad) return set_error(HESS_ERR_INVALID_ARG, "no output requested");
  Guard g(h->device);
  return run_apply(h, K, evals, evecs, full, lam_tilde, X, b, HX, quad);
}
