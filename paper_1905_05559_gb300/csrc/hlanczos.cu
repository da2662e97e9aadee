// The exact Hessian as an operator, without forming it:
//
//   hessian_vector_products : H v for a block of directions (Sec. 5.1, the
//                             R-operator; Appendix A)
//   hessian_topk_eig        : the k algebraically largest eigenpairs of H
//                             (Sec. 5.3), by Lanczos on the operator v -> H v
//
// The Lanczos recurrence runs in FP64 with full reorthogonalisation (two
// classical Gram-Schmidt passes against every earlier vector), extended in
// steps until the residual bounds |beta_m y_m| of the top-k Ritz pairs fall
// below 1e-10 of ||T_m||.  The products H q_j are computed in FP64 (or in
// FP32 for HESS_FP32, the recurrence staying FP64).  The tridiagonal
// eigenpairs use the same Sturm bisection and inverse iteration as the OPG
// eigensolver; the Ritz vectors are Q_m Y.
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "devmath.cuh"
#include "internal.h"

namespace hm {

namespace {

constexpr int kHlChunks = 16;  // slices of the vector length in the coefficient kernel

// q = a random unit vector (counter-based draws), one block.
__global__ void hl_start_kernel(double* q, int64_t P, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double v = rnd_sym(key, (uint64_t)i);
    q[i] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) q[i] *= inv;
}

// Partial coefficients part[ch][i] = sum over slice ch of q_i . w for
// i < cnt, and (self) part[ch][cnt] = slice of w . w.  One warp per vector,
// blockIdx.y = slice.  Does nothing once the recurrence has stopped.
__global__ void hl_coef_kernel(const double* Q, const double* w, int64_t P, int cnt, int self, int64_t pc,
                               double* part, int ldp, const int* stop) {
  if (*stop >= 0) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i > cnt || (i == cnt && !self)) return;
  const int64_t p0 = (int64_t)blockIdx.y * pc;
  const int64_t p1 = p0 + pc < P ? p0 + pc : P;
  const double* a = i < cnt ? Q + (int64_t)i * P : w;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t p = p0 + lane;
  for (; p + 96 < p1; p += 128) {
    s0 = fma(a[p], w[p], s0);
    s1 = fma(a[p + 32], w[p + 32], s1);
    s2 = fma(a[p + 64], w[p + 64], s2);
    s3 = fma(a[p + 96], w[p + 96], s3);
  }
  for (; p < p1; p += 32) s0 = fma(a[p], w[p], s0);
  const double s = warp_sum((s0 + s1) + (s2 + s3));
  if (lane == 0) part[(int64_t)blockIdx.y * ldp + i] = s;
}

// w -= sum_{i<cnt} c_i q_i with c_i = sum of the slices' partials (every
// block sums them into shared memory; block 0 also stores them, with the
// self product at index cnt when present, in c).  One thread per entry.
__global__ void hl_sub_kernel(const double* Q, const double* part, int ldp, int nch, int cnt, int self, int64_t P,
                              double* w, double* c, const int* stop) {
  extern __shared__ double cs[];
  if (*stop >= 0) return;
  const int ctot = cnt + (self ? 1 : 0);
  for (int i = threadIdx.x; i < ctot; i += blockDim.x) {
    double v = 0.0;
    for (int ch = 0; ch < nch; ++ch) v += part[(int64_t)ch * ldp + i];
    cs[i] = v;
    if (blockIdx.x == 0) c[i] = v;
  }
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < cnt; i += 4) {
      s0 = fma(cs[i], Q[(int64_t)i * P + p], s0);
      s1 = fma(cs[i + 1], Q[(int64_t)(i + 1) * P + p], s1);
      s2 = fma(cs[i + 2], Q[(int64_t)(i + 2) * P + p], s2);
      s3 = fma(cs[i + 3], Q[(int64_t)(i + 3) * P + p], s3);
    }
    for (; i < cnt; ++i) s0 = fma(cs[i], Q[(int64_t)i * P + p], s0);
    w[p] -= (s0 + s1) + (s2 + s3);
  }
}

// End of step j: alpha_j = c1_j + c2_j (both passes' coefficient of q_j),
// beta_j = ||w||, q_{j+1} = w / beta_j.  A breakdown (||w|| below 1e-8 of
// ||H q_j||, or zero) sets beta_j = 0 and stop = j instead.  One block.
__global__ void hl_next_kernel(const double* w, int64_t P, const double* c1, const double* c2, int j, double* alpha,
                               double* beta, double* qnext, int* stop) {
  __shared__ double sh[32];
  if (*stop >= 0) return;
  double s = 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s = fma(w[p], w[p], s);
  s = block_sum(s, sh);
  const double nrm = sqrt(s);
  const double nrm0 = sqrt(fmax(c1[j + 1], 0.0));
  const bool brk = !(nrm > 1e-8 * nrm0) || !(nrm > 0.0);
  if (threadIdx.x == 0) {
    alpha[j] = c1[j] + c2[j];
    beta[j] = brk ? 0.0 : nrm;
  }
  if (brk) {
    __syncthreads();
    if (threadIdx.x == 0) *stop = j;
    return;
  }
  const double inv = 1.0 / nrm;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) qnext[p] = w[p] * inv;
}

// Restart after a breakdown at step j - 1: w = a fresh random vector (the
// same counter-based draw on every run).
__global__ void hl_fill_kernel(double* w, int64_t P, uint64_t key, int j) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    w[p] = rnd_sym(key, (uint64_t)j * 0x100000000ull + (uint64_t)p);
}

// q = w / ||w|| and clear the stop flag (one block).
__global__ void hl_store_kernel(const double* w, int64_t P, double* q, int* stop) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s = fma(w[p], w[p], s);
  s = block_sum(s, sh);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) q[p] = w[p] * inv;
  if (threadIdx.x == 0) *stop = -1;
}

// out = max_i |a_i| + |b_{i-1}| + |b_i| (>= ||T_m||, Gershgorin), one warp.
__global__ void hl_tnorm_kernel(const double* a, const double* b, int m, double* out) {
  double t = 0.0;
  for (int i = threadIdx.x; i < m; i += 32)
    t = fmax(t, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0));
  for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  if (threadIdx.x == 0) *out = t;
}

// Final per-vector pass: evals, sign so that the largest-magnitude entry
// (lowest index on ties) is positive.
__global__ void hl_finalize_kernel(double* evecs, int64_t P, const double* theta, double* evals) {
  __shared__ double shv[32];
  __shared__ int64_t shi[32];
  const int c = blockIdx.x;
  double* q = evecs + (int64_t)c * P;
  if (threadIdx.x == 0) evals[c] = theta[c];
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double v = fabs(q[i]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    shv[threadIdx.x >> 5] = best;
    shi[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
      if (shv[i] > shv[0] || (shv[i] == shv[0] && shi[i] < shi[0])) {
        shv[0] = shv[i];
        shi[0] = shi[i];
      }
  }
  __syncthreads();
  if (q[shi[0]] < 0.0)
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) q[i] = -q[i];
}

__global__ void d2f_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f2d_kernel(const float* in, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

unsigned grid_for(int64_t n, int threads = 256) {
  int64_t b = cdiv(n, threads);
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
}

// 1: device (or managed) memory of the handle's device, 0: host memory.
hess_status where(const hess_mlp* h, const void* p, const char* name, int* on_dev) {
  cudaPointerAttributes at;
  *on_dev = 0;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return HESS_OK;
  }
  if (at.type == cudaMemoryTypeDevice && at.device != h->device)
    return set_error(HESS_ERR_INVALID_ARG, "%s lives on device %d, handle on device %d", name, at.device, h->device);
  *on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  return HESS_OK;
}

// Algorithmic flops of one product H v (per direction): the GEMMs of the
// R-forward pass, the R-back-propagation and the contraction (2 per
// multiply-add).
double hvp_flops(const Net& net, int64_t N) {
  double f = 0.0;
  for (int j = 1; j <= net.L - 1; ++j) {
    const double tin = net.T[j - 1], tout = net.T[j];
    f += 2.0 * N * tin * tout * (j > 1 ? 2.0 : 1.0);  // forward: V a (+ W R{a})
    f += 2.0 * N * tin * tout * (j > 1 ? 2.0 : 1.0);  // contraction: R{delta} a (+ delta R{a})
    if (j <= net.L - 2) f += 2.0 * 2.0 * N * tout * net.T[j + 1];  // backward: R{delta} W + delta V
  }
  return f;
}

// The network's caches at X, Y in precision T (inputs in the caller's dtype
// `in_dbl`, on the device or staged).
template <typename T>
struct Inputs {
  const void* xs = nullptr;  // staging of host inputs (caller dtype)
  const void* ys = nullptr;
  T* xt = nullptr;  // inputs in T
  T* yt = nullptr;
};

template <typename T>
void plan_inputs(Arena& ar, const Net& net, int64_t N, bool in_dbl, int x_dev, int y_dev, const void* X,
                 const void* Y, Inputs<T>& in) {
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1];
  const size_t es = in_dbl ? sizeof(double) : sizeof(float);
  const bool same = in_dbl == std::is_same<T, double>::value;
  in.xs = x_dev ? X : ar.take<char>(N * T1 * es);
  in.ys = y_dev ? Y : ar.take<char>(N * TL * es);
  in.xt = same && x_dev ? (T*)X : ar.take<T>(N * T1);
  in.yt = same && y_dev ? (T*)Y : ar.take<T>(N * TL);
}

template <typename T>
hess_status load_inputs(const Net& net, int64_t N, bool in_dbl, int x_dev, int y_dev, const void* X, const void* Y,
                        const Inputs<T>& in, cudaStream_t s) {
  const int64_t T1 = net.T[0], TL = net.T[net.L - 1];
  const size_t es = in_dbl ? sizeof(double) : sizeof(float);
  if (!x_dev) HM_CUDA(cudaMemcpyAsync((void*)in.xs, X, N * T1 * es, cudaMemcpyHostToDevice, s));
  if (!y_dev) HM_CUDA(cudaMemcpyAsync((void*)in.ys, Y, N * TL * es, cudaMemcpyHostToDevice, s));
  auto move = [&](const void* src, T* dst, int64_t n) -> hess_status {
    if ((const void*)dst == src) return HESS_OK;
    if (in_dbl == std::is_same<T, double>::value) {
      HM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      return HESS_OK;
    }
    if (in_dbl) return convert((const double*)src, (float*)dst, n, s);
    return convert((const float*)src, (double*)dst, n, s);
  };
  HM_TRY(move(in.xs, in.xt, N * T1));
  HM_TRY(move(in.ys, in.yt, N * TL));
  return HESS_OK;
}

// Directions per block of the product: R-operator buffers within ~2 GB and
// N B within the 32-bit GEMM row count.
int hvp_block_size(const Net& net, int64_t N, size_t elem, int b) {
  int64_t sumT = 0;
  for (int j = 1; j < net.L; ++j) sumT += 3 * net.T[j];
  const double per_dir = (double)elem * (double)N * (double)sumT;
  int64_t B = (int64_t)(2.0e9 / per_dir);
  const int64_t cap = ((1ll << 31) - 1) / N;
  if (B > cap) B = cap;
  if (B > 256) B = 256;
  if (B < 1) B = 1;
  return (int)(B < b ? B : b);
}

template <typename T>
hess_status run_hvp(hess_mlp* h, const void* X, const void* Y, int64_t N, const void* V, int b, void* HV) {
  const Net& net = h->net;
  const int64_t P = net.P;
  constexpr bool dbl = std::is_same<T, double>::value;
  int x_dev, y_dev, v_dev, o_dev;
  HM_TRY(where(h, X, "X", &x_dev));
  HM_TRY(where(h, Y, "Y", &y_dev));
  HM_TRY(where(h, V, "V", &v_dev));
  HM_TRY(where(h, HV, "HV", &o_dev));
  const int B = hvp_block_size(net, N, sizeof(T), b);
  Inputs<T> in;
  Caches<T> c;
  RopBufs<T> r;
  T *vd = nullptr, *od = nullptr;
  char* split = nullptr;
  auto plan = [&](Arena& ar) {
    plan_inputs(ar, net, N, dbl, x_dev, y_dev, X, Y, in);
    plan_caches(ar, net, N, c);
    plan_rop(ar, net, N, 1, B, r);
    vd = v_dev ? (T*)V : ar.take<T>(P * (int64_t)b);
    od = o_dev ? (T*)HV : ar.take<T>(P * (int64_t)b);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  plan(ar);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  HM_TRY(load_inputs(net, N, dbl, x_dev, y_dev, X, Y, in, s));
  if (!v_dev) HM_CUDA(cudaMemcpyAsync(vd, V, P * b * sizeof(T), cudaMemcpyHostToDevice, s));
  const T* omega = dbl ? (const T*)h->omega64 : (const T*)h->omega32;
  HM_TRY(forward_backward(net, omega, (const T*)in.xt, (const T*)in.yt, c, s));
  {
    Tick t(h, HESS_K_HVP, hvp_flops(net, N) * b, 0.0);
    for (int d0 = 0; d0 < b; d0 += B) {
      const int nb = b - d0 < B ? b - d0 : B;
      r.B = nb;
      HM_TRY(hvp_block(net, omega, c, vd + (int64_t)d0 * P, P, nb, r, od + (int64_t)d0 * P, P, s));
    }
  }
  if (!o_dev) {
    HM_CUDA(cudaMemcpyAsync(HV, od, P * b * sizeof(T), cudaMemcpyDeviceToHost, s));
  }
  if (!x_dev || !y_dev || !v_dev || !o_dev) {
    HM_CUDA(cudaStreamSynchronize(s));
    HM_TRY(take_sticky_error(h));
  }
  return HESS_OK;
}

// Lanczos on v -> H v with products in precision T.
template <typename T>
hess_status run_heig(hess_mlp* h, const void* X, const void* Y, int64_t N, bool in_dbl, int k, double* evals,
                     double* evecs, int* steps_out) {
  const Net& net = h->net;
  const int64_t P = net.P;
  constexpr bool dbl = std::is_same<T, double>::value;
  int x_dev, y_dev, ev_dev, q_dev;
  HM_TRY(where(h, X, "X", &x_dev));
  HM_TRY(where(h, Y, "Y", &y_dev));
  HM_TRY(where(h, evals, "evals", &ev_dev));
  HM_TRY(where(h, evecs, "evecs", &q_dev));
  // Krylov dimension cap and extension step
  int64_t mcap = (int64_t)8 * k + 1024;
  if (mcap > P) mcap = P;
  const int64_t step = k > 32 ? k : 32;
  const int ldp = (int)mcap + 2;
  const int64_t pc = cdiv(P, kHlChunks);
  Inputs<T> in;
  Caches<T> c;
  RopBufs<T> r;
  double *Q, *w, *part, *c1, *c2, *alpha, *beta, *theta, *Y_, *rr, *mx, *evd, *eqd, *tri;
  T *vt = nullptr, *ht = nullptr;  // FP32 products: the direction and result in T
  int *stop, *cstart;
  char* split = nullptr;
  auto plan = [&](Arena& ar) {
    plan_inputs(ar, net, N, in_dbl, x_dev, y_dev, X, Y, in);
    plan_caches(ar, net, N, c);
    plan_rop(ar, net, N, 1, 1, r);
    Q = ar.take<double>((mcap + 1) * P);
    w = ar.take<double>(P);
    if (!dbl) {
      vt = ar.take<T>(P);
      ht = ar.take<T>(P);
    }
    part = ar.take<double>((int64_t)kHlChunks * ldp);
    c1 = ar.take<double>(ldp);
    c2 = ar.take<double>(ldp);
    alpha = ar.take<double>(mcap + 1);
    beta = ar.take<double>(mcap + 1);
    theta = ar.take<double>(k);
    Y_ = ar.take<double>((int64_t)k * mcap);
    rr = ar.take<double>(k);
    mx = ar.take<double>(4);
    cstart = ar.take<int>(k);
    stop = ar.take<int>(1);
    const int64_t tn = tridiag_scratch_doubles(mcap, k);
    tri = tn ? ar.take<double>(tn) : nullptr;
    evd = ev_dev ? evals : ar.take<double>(k);
    eqd = q_dev ? evecs : ar.take<double>(P * (int64_t)k);
    split = ar.take<char>(kSplitBytes);
  };
  Arena ar;
  plan(ar);
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  plan(ar);
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  cudaStream_t s = h->stream;
  HM_TRY(load_inputs(net, N, in_dbl, x_dev, y_dev, X, Y, in, s));
  const T* omega = dbl ? (const T*)h->omega64 : (const T*)h->omega32;
  HM_TRY(forward_backward(net, omega, (const T*)in.xt, (const T*)in.yt, c, s));

  const uint64_t key = 0x48455353ull;  // start and restart draws
  const double hflops = hvp_flops(net, N);
  double flops = 0.0;
  HM_CUDA(cudaMemsetAsync(alpha, 0, (mcap + 1) * sizeof(double), s));
  HM_CUDA(cudaMemsetAsync(beta, 0, (mcap + 1) * sizeof(double), s));
  HM_CUDA(cudaMemsetAsync(stop, 0xff, sizeof(int), s));
  hl_start_kernel<<<1, 1024, 0, s>>>(Q, P, key);
  HM_LAUNCHED();
  const unsigned gsub = (unsigned)(cdiv(P, 256) < 4096 ? cdiv(P, 256) : 4096);
  const size_t sub_smem = (size_t)ldp * sizeof(double);
  if (sub_smem > (size_t)48 << 10) {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
      e = cudaFuncSetAttribute(hl_sub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
    });
    if (e != cudaSuccess) return set_error(HESS_ERR_CUDA, "Lanczos kernel attribute: %s", cudaGetErrorString(e));
  }
  // two Gram-Schmidt passes of w against q_0 .. q_{cnt-1}; coefficients to co
  auto cgs = [&](int cnt, int self, double* co) -> hess_status {
    dim3 gc((unsigned)cdiv(cnt + 1, 8), kHlChunks);
    hl_coef_kernel<<<gc, 256, 0, s>>>(Q, w, P, cnt, self, pc, part, ldp, stop);
    HM_LAUNCHED();
    hl_sub_kernel<<<gsub, 256, sub_smem, s>>>(Q, part, ldp, kHlChunks, cnt, self, P, w, co, stop);
    HM_LAUNCHED();
    return HESS_OK;
  };
  int m = 0;
  int64_t target = (int64_t)2 * k + 32;
  if (target > mcap) target = mcap;
  bool converged = false;
  double* hp = h->host_pinned;
  while (true) {
    {
      Tick t(h, HESS_K_HLANCZOS, 0.0, 0.0);
      double f = 0.0;
      for (int j = m; j < (int)target; ++j) {
        // w = H q_j
        const double* qj = Q + (int64_t)j * P;
        if (dbl) {
          HM_TRY(hvp_block(net, omega, c, (const T*)qj, P, 1, r, (T*)w, P, s));
        } else {
          d2f_kernel<<<grid_for(P), 256, 0, s>>>(qj, (float*)vt, P);
          HM_LAUNCHED();
          HM_TRY(hvp_block(net, omega, c, (const T*)vt, P, 1, r, ht, P, s));
          f2d_kernel<<<grid_for(P), 256, 0, s>>>((const float*)ht, w, P);
          HM_LAUNCHED();
        }
        HM_TRY(cgs(j + 1, 1, c1));
        HM_TRY(cgs(j + 1, 0, c2));
        hl_next_kernel<<<1, 1024, 0, s>>>(w, P, c1, c2, j, alpha, beta, Q + (int64_t)(j + 1) * P, stop);
        HM_LAUNCHED();
        f += hflops + 8.0 * (j + 1) * (double)P + 4.0 * P;
      }
      t.set_work(f, 0.0);
      flops += f;
    }
    const int mt = (int)target;
    HM_TRY(tridiag_topk(alpha, beta, mt, k, theta, cstart, Y_, mcap, beta + mt - 1, rr, mx, key + 11, tri, s));
    hl_tnorm_kernel<<<1, 32, 0, s>>>(alpha, beta, mt, mx + 2);
    HM_LAUNCHED();
    HM_CUDA(cudaMemcpyAsync(hp, mx, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(hp + 3), stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    const int stopped = reinterpret_cast<int*>(hp + 3)[0];
    if (stopped >= 0) {
      // breakdown at step `stopped`: T_{stopped+1} is complete and decoupled
      m = stopped + 1;
      if (m >= P) {
        // the whole space is spanned: the Ritz pairs are exact
        HM_TRY(tridiag_topk(alpha, beta, m, k, theta, cstart, Y_, mcap, beta + m - 1, rr, mx, key + 11, tri, s));
        converged = true;
        break;
      }
      if (m >= mcap) break;
      // continue from a random vector orthogonal to q_0 .. q_{m-1}
      hl_fill_kernel<<<gsub, 256, 0, s>>>(w, P, key + 7, m);
      HM_LAUNCHED();
      HM_CUDA(cudaMemsetAsync(stop, 0xff, sizeof(int), s));
      HM_TRY(cgs(m, 0, c2));
      HM_TRY(cgs(m, 0, c2));
      hl_store_kernel<<<1, 1024, 0, s>>>(w, P, Q + (int64_t)m * P, stop);
      HM_LAUNCHED();
      target = m + step > (int64_t)k ? m + step : (int64_t)k;
      if (target > mcap) target = mcap;
      continue;
    }
    m = mt;
    if (hp[0] <= 1e-10 * hp[2] || m >= P) {
      converged = true;
      break;
    }
    if (m >= mcap) break;
    target = m + step;
    if (target > mcap) target = mcap;
  }
  if (steps_out) *steps_out = m;
  // Ritz vectors: evecs row c = sum_j Y[c][j] q_j
  {
    Tick t(h, HESS_K_HLANCZOS, 2.0 * P * (double)m * k, 0.0);
    Gemm<double> g;
    g.M = (int)P;
    g.N = k;
    g.K = m;
    g.A = Q;
    g.sam = 1;
    g.sak = P;
    g.B = Y_;
    g.sbk = 1;
    g.sbn = mcap;
    g.C = eqd;
    g.scm = 1;
    g.scn = P;
    HM_TRY(gemm(g, s));
    hl_finalize_kernel<<<k, 256, 0, s>>>(eqd, P, theta, evd);
    HM_LAUNCHED();
  }
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evals, evd, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(evecs, eqd, P * k * sizeof(double), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  HM_TRY(take_sticky_error(h));
  if (!converged) return set_error(HESS_ERR_NOT_CONVERGED, "Hessian Lanczos did not converge in %d steps", m);
  return HESS_OK;
}

hess_status check_inputs(hess_mlp* h, const void* X, const void* Y, int64_t N) {
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (!X || !Y) return set_error(HESS_ERR_INVALID_ARG, "X and Y must be non-NULL");
  if (N < 1 || N > (1ll << 31) - 1) return set_error(HESS_ERR_INVALID_ARG, "N must be in 1 .. 2^31 - 1");
  return take_sticky_error(h);
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hess_status hessian_vector_products(hess_mlp* h, const void* X, const void* Y, int64_t N,
                                               hess_precision prec, const void* V, int b, void* HV) {
  clear_error();
  HM_TRY(check_inputs(h, X, Y, N));
  if (!V || !HV) return set_error(HESS_ERR_INVALID_ARG, "V and HV must be non-NULL");
  if (b < 1) return set_error(HESS_ERR_INVALID_ARG, "b must be >= 1 (got %d)", b);
  if (prec != HESS_FP64 && prec != HESS_FP32)
    return set_error(prec == HESS_BF16 || prec == HESS_BF16X3 ? HESS_ERR_UNSUPPORTED : HESS_ERR_INVALID_ARG,
                     "Hessian-vector products run in FP64 or FP32 (precision %d)", (int)prec);
  Guard g(h->device);
  if (prec == HESS_FP64) return run_hvp<double>(h, X, Y, N, V, b, HV);
  return run_hvp<float>(h, X, Y, N, V, b, HV);
}

extern "C" hess_status hessian_topk_eig(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                        hess_precision prec, double* evals, double* evecs, int* steps) {
  clear_error();
  HM_TRY(check_inputs(h, X, Y, N));
  if (k < 1 || k > h->net.P)
    return set_error(HESS_ERR_INVALID_ARG, "need 1 <= k <= P (k = %d, P = %lld)", k, (long long)h->net.P);
  if (!evals || !evecs) return set_error(HESS_ERR_INVALID_ARG, "evals and evecs must be non-NULL");
  if (prec != HESS_FP64 && prec != HESS_FP32)
    return set_error(prec == HESS_BF16 || prec == HESS_BF16X3 ? HESS_ERR_UNSUPPORTED : HESS_ERR_INVALID_ARG,
                     "the Hessian products of the eigensolver run in FP64 or FP32 (precision %d)", (int)prec);
  Guard g(h->device);
  if (prec == HESS_FP64) return run_heig<double>(h, X, Y, N, true, k, evals, evecs, steps);
  return run_heig<float>(h, X, Y, N, false, k, evals, evecs, steps);
}
