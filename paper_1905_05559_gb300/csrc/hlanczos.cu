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

constexpr int kHlChunks = 32;  // slices of the vector length in the coefficient kernel

// The recurrence's step index j lives in device memory (jd), so that one
// captured step replays for every j.  qcur holds q_j, the direction of the
// next product.

// q_0 = qcur = a random unit vector (counter-based draws), one block.
__global__ void hl_start_kernel(double* q, double* qcur, int64_t P, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double v = rnd_sym(key, (uint64_t)i);
    q[i] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    q[i] *= inv;
    qcur[i] = q[i];
  }
}

__global__ void hl_setj_kernel(int* jd, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *jd = v;
}

// Coefficients c_i = q_i . w for i < cnt = *jd + 1 and (self) c_cnt = w . w.
// One warp per vector and slice of the vector length (blockIdx.y = slice)
// writes a partial; the last block to finish adds the partials in slice
// order (the same order on every run) into c.  Does nothing once the
// recurrence has stopped.
__global__ void hl_coef_kernel(const double* Q, const double* w, int64_t P, const int* jd, int self, int64_t pc,
                               double* part, int ldp, double* c, unsigned* counter, const int* stop) {
  __shared__ int s_last;
  if (*stop >= 0) return;
  const int cnt = *jd + 1;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int ctot = cnt + (self ? 1 : 0);
  if (i < ctot) {
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
    const double sum = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) {
      part[(int64_t)blockIdx.y * ldp + i] = sum;
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    s_last = t == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nch = gridDim.y;
  for (int ii = threadIdx.x; ii < ctot; ii += blockDim.x) {
    double v0 = 0.0, v1 = 0.0;
    int ch = 0;
    for (; ch + 1 < nch; ch += 2) {
      v0 += __ldcg(part + (int64_t)ch * ldp + ii);
      v1 += __ldcg(part + (int64_t)(ch + 1) * ldp + ii);
    }
    if (ch < nch) v0 += __ldcg(part + (int64_t)ch * ldp + ii);
    c[ii] = v0 + v1;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// w -= sum_{i<cnt} c_i q_i (cnt = *jd + 1).  A block of 8 warps owns 32
// consecutive entries (one per lane; grid-stride over such chunks); its
// warps take every 8th i and their sums meet in shared memory in warp order.
// npart (may be null): per-block sums of the updated w_p^2.
__global__ void __launch_bounds__(256) hl_sub_kernel(const double* Q, const double* c, const int* jd, int64_t P,
                                                     double* w, double* npart, const int* stop) {
  extern __shared__ double cs[];
  __shared__ double red[8][33];
  __shared__ double sh[32];
  if (*stop >= 0) return;
  const int cnt = *jd + 1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double nn = 0.0;
  for (int64_t p0 = (int64_t)blockIdx.x * 32; p0 < P; p0 += (int64_t)gridDim.x * 32) {
    const int64_t p = p0 + lane;
    double s0 = 0.0, s1 = 0.0;
    if (p < P) {
      int i = warp;
      for (; i + 8 < cnt; i += 16) {
        s0 = fma(cs[i], Q[(int64_t)i * P + p], s0);
        s1 = fma(cs[i + 8], Q[(int64_t)(i + 8) * P + p], s1);
      }
      if (i < cnt) s0 = fma(cs[i], Q[(int64_t)i * P + p], s0);
    }
    red[warp][lane] = s0 + s1;
    __syncthreads();
    if (warp == 0 && p < P) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += red[q][lane];
      const double v = w[p] - t;
      w[p] = v;
      nn = fma(v, v, nn);
    }
    __syncthreads();
  }
  if (npart) {
    nn = block_sum(nn, sh);
    if (threadIdx.x == 0) npart[blockIdx.x] = nn;
  }
}

// End of step j = *jd: alpha_j = c1_j + c2_j (both passes' coefficient of
// q_j), beta_j = ||w|| (from the nparts block sums of the second pass, added
// in the same order by every block), q_{j+1} = qcur = w / beta_j.  A
// breakdown (||w|| below 1e-8 of ||H q_j||, or zero) sets beta_j = 0 and
// stop = j instead.
__global__ void hl_next_kernel(const double* w, int64_t P, const double* npart, int nparts, const double* c1,
                               const double* c2, const int* jd, double* alpha, double* beta, double* Q,
                               double* qcur, int* stop) {
  __shared__ double s_n2;
  if (*stop >= 0) return;
  const int j = *jd;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nparts; b += 32) t += npart[b];
    t = warp_sum(t);
    if (threadIdx.x == 0) s_n2 = t;
  }
  __syncthreads();
  const double nrm = sqrt(s_n2);
  const double nrm0 = sqrt(fmax(c1[j + 1], 0.0));
  const bool brk = !(nrm > 1e-8 * nrm0) || !(nrm > 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha[j] = c1[j] + c2[j];
    beta[j] = brk ? 0.0 : nrm;
    if (brk) *stop = j;
  }
  if (brk) return;
  const double inv = 1.0 / nrm;
  double* qn = Q + (int64_t)(j + 1) * P;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[p] * inv;
    qn[p] = v;
    qcur[p] = v;
  }
}

// j <- j + 1 unless the recurrence has stopped.
__global__ void hl_advance_kernel(int* jd, const int* stop) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *stop < 0) *jd += 1;
}

// Restart after a breakdown at step j - 1: w = a fresh random vector (the
// same counter-based draw on every run).
__global__ void hl_fill_kernel(double* w, int64_t P, uint64_t key, int j) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    w[p] = rnd_sym(key, (uint64_t)j * 0x100000000ull + (uint64_t)p);
}

// q = qcur = w / ||w|| and clear the stop flag (one block).
__global__ void hl_store_kernel(const double* w, int64_t P, double* q, double* qcur, int* stop) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s = fma(w[p], w[p], s);
  s = block_sum(s, sh);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) {
    const double v = w[p] * inv;
    q[p] = v;
    qcur[p] = v;
  }
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
  double *Q, *w, *qcur, *part, *npart, *c1, *c2, *alpha, *beta, *theta, *Y_, *rr, *mx, *evd, *eqd, *tri;
  T *vt = nullptr, *ht = nullptr;  // FP32 products: the direction and result in T
  int *stop, *cstart, *jd;
  unsigned* counter;
  char* split = nullptr;
  auto plan = [&](Arena& ar) {
    plan_inputs(ar, net, N, in_dbl, x_dev, y_dev, X, Y, in);
    plan_caches(ar, net, N, c);
    plan_rop(ar, net, N, 1, 1, r);
    Q = ar.take<double>((mcap + 1) * P);
    w = ar.take<double>(P);
    qcur = ar.take<double>(P);
    if (!dbl) {
      vt = ar.take<T>(P);
      ht = ar.take<T>(P);
    }
    part = ar.take<double>((int64_t)kHlChunks * ldp);
    npart = ar.take<double>(4096);
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
    jd = ar.take<int>(1);
    counter = ar.take<unsigned>(1);
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
  HM_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  HM_TRY(fill(r.ones, N, T(1), s));
  r.ones_ready = true;
  hl_start_kernel<<<1, 1024, 0, s>>>(Q, qcur, P, key);
  HM_LAUNCHED();
  const unsigned gsub = (unsigned)(cdiv(P, 32) < 4096 ? cdiv(P, 32) : 4096);
  const unsigned gnext = (unsigned)(cdiv(P, 256) < 4096 ? cdiv(P, 256) : 4096);
  const size_t sub_smem = (size_t)ldp * sizeof(double);
  if (sub_smem > (size_t)48 << 10) {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
      e = cudaFuncSetAttribute(hl_sub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
    });
    if (e != cudaSuccess) return set_error(HESS_ERR_CUDA, "Lanczos kernel attribute: %s", cudaGetErrorString(e));
  }
  // a Gram-Schmidt pass of w against q_0 .. q_{*jd}; coefficients to co;
  // the coefficient grid has a warp for each of up to cnt_max vectors and
  // for the self product
  auto cgs = [&](int cnt_max, int self, double* co, double* np, cudaStream_t st) -> hess_status {
    dim3 gc((unsigned)cdiv(cnt_max + 1, 8), kHlChunks);
    hl_coef_kernel<<<gc, 256, 0, st>>>(Q, w, P, jd, self, pc, part, ldp, co, counter, stop);
    HM_LAUNCHED();
    hl_sub_kernel<<<gsub, 256, sub_smem, st>>>(Q, co, jd, P, w, np, stop);
    HM_LAUNCHED();
    return HESS_OK;
  };
  // one Lanczos step j = *jd (j <= jmax): w = H q_j, two passes, q_{j+1}
  auto one_step = [&](int jmax, cudaStream_t st) -> hess_status {
    if (dbl) {
      HM_TRY(hvp_block(net, omega, c, (const T*)qcur, P, 1, r, (T*)w, P, st));
    } else {
      d2f_kernel<<<grid_for(P), 256, 0, st>>>(qcur, (float*)vt, P);
      HM_LAUNCHED();
      HM_TRY(hvp_block(net, omega, c, (const T*)vt, P, 1, r, ht, P, st));
      f2d_kernel<<<grid_for(P), 256, 0, st>>>((const float*)ht, w, P);
      HM_LAUNCHED();
    }
    HM_TRY(cgs(jmax + 1, 1, c1, nullptr, st));
    HM_TRY(cgs(jmax + 1, 0, c2, npart, st));
    hl_next_kernel<<<gnext, 256, 0, st>>>(w, P, npart, (int)gsub, c1, c2, jd, alpha, beta, Q, qcur, stop);
    HM_LAUNCHED();
    hl_advance_kernel<<<1, 32, 0, st>>>(jd, stop);
    HM_LAUNCHED();
    return HESS_OK;
  };
  // steps m .. target-1: one step captured as a CUDA graph on a private
  // stream and replayed (launch-bound short kernels), or launched directly
  // when the capture is not possible
  cudaStream_t cs = nullptr;
  HM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      if (s) cudaStreamDestroy(s);
    }
  } csg{cs};
  auto run_steps = [&](int m0, int m1) -> hess_status {
    hl_setj_kernel<<<1, 32, 0, s>>>(jd, m0);
    HM_LAUNCHED();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t l0 = g_launches.load();
    bool captured = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (captured) {
      const hess_status st = one_step(m1 - 1, cs);
      const bool ended = cudaStreamEndCapture(cs, &graph) == cudaSuccess;
      captured = st == HESS_OK && ended && graph &&
                 cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      if (!captured) clear_error();
    }
    const int64_t nodes = g_launches.load() - l0;
    g_launches -= nodes;
    if (captured) {
      for (int j = m0; j < m1; ++j) {
        const cudaError_t e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) {
          cudaGraphExecDestroy(exec);
          cudaGraphDestroy(graph);
          return set_error(HESS_ERR_CUDA, "Lanczos step graph: %s", cudaGetErrorString(e));
        }
        g_launches += nodes;
      }
      // launches already queued keep their resources until they finish
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      return HESS_OK;
    }
    if (graph) cudaGraphDestroy(graph);
    for (int j = m0; j < m1; ++j) HM_TRY(one_step(m1 - 1, s));
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
      HM_TRY(run_steps(m, (int)target));
      double f = 0.0;
      for (int j = m; j < (int)target; ++j) f += hflops + 8.0 * (j + 1) * (double)P + 4.0 * P;
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
      hl_fill_kernel<<<gnext, 256, 0, s>>>(w, P, key + 7, m);
      HM_LAUNCHED();
      HM_CUDA(cudaMemsetAsync(stop, 0xff, sizeof(int), s));
      hl_setj_kernel<<<1, 32, 0, s>>>(jd, m - 1);
      HM_LAUNCHED();
      HM_TRY(cgs(m, 0, c2, nullptr, s));
      HM_TRY(cgs(m, 0, c2, nullptr, s));
      hl_store_kernel<<<1, 1024, 0, s>>>(w, P, Q + (int64_t)m * P, qcur, stop);
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
