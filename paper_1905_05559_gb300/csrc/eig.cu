// FP64 top-k eigenpairs of the OPG through the N x N Gram matrix
// M = G G^T / N (Sec. 5.4, Eq. J: the OPG eigenvectors are the right singular
// vectors of G, the eigenvalues the squared singular values over N).
//
//   1. M in factored form: g_n . g_m = sum_l (delta_n . delta_m)(a_n . a_m + 1)
//   2. Lanczos on M with full (two-pass classical Gram-Schmidt)
//      reorthogonalisation; a breakdown restarts from a fresh random vector
//   3. top-k eigenvalues of the tridiagonal T_m by Sturm-sequence bisection,
//      eigenvectors by inverse iteration (orthogonalised against the earlier
//      ones), residual bound |beta_m y_m| for convergence
//   4. Ritz vectors U = Q_m Y, back-projection q = G^T u / sqrt(N mu)
#include <cfloat>

#include "internal.h"

namespace hm {

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// SplitMix64 in counter mode: uniform in [-1, 1)
__device__ __forceinline__ double rnd_sym(uint64_t key, uint64_t i) {
  uint64_t z = mix64(key + (i + 1) * 0x9E3779B97F4A7C15ull);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over a block of up to 1024 threads
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ Gram matrix
__global__ void gram_acc_kernel(double* M, const double* DD, const double* AA, int64_t n2,
                                double invN) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    M[i] += DD[i] * (AA[i] + 1.0) * invN;
}

// ---------------------------------------------------------------- BLAS-2
// y[r] = sum_c A[r*lda + c] x[c]; one warp per row.  cond: skip unless *cond.
__global__ void gemv_rows_kernel(const double* A, int64_t lda, int rows, int64_t cols,
                                 const double* x, double* y, const int* cond) {
  if (cond && !*cond) return;
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const double* a = A + (int64_t)r * lda;
  double s = 0.0;
  for (int64_t c = threadIdx.x & 31; c < cols; c += 32) s = fma(a[c], x[c], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) y[r] = s;
}

// w[n] -= sum_i Q[i*ldq + n] h[i]
__global__ void gemv_sub_kernel(const double* Q, int64_t ldq, int nvec, int64_t N, const double* h,
                                double* w, const int* cond) {
  if (cond && !*cond) return;
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s = 0.0;
  for (int i = 0; i < nvec; ++i) s = fma(Q[(int64_t)i * ldq + n], h[i], s);
  w[n] -= s;
}

// ---------------------------------------------------------------- Lanczos
// After the two reorthogonalisation passes: alpha_j = h1[j] + h2[j],
// beta_j = ||w||; q_{j+1} = w / beta_j, or on breakdown a random vector that
// the gated kernels then orthonormalise (flag = 1) with beta_j = 0.
__global__ void lanczos_norm_kernel(const double* w, double* qn, int64_t N, int j,
                                    const double* h1, const double* h2, double* alpha,
                                    double* beta, int* flag, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s = fma(w[n], w[n], s);
  s = block_sum(s, sh);
  double nrm = sqrt(s);
  double a = h1[j] + h2[j];
  // scale of T so far
  double scale = fabs(a);
  for (int i = threadIdx.x; i < j; i += blockDim.x) scale = fmax(scale, fmax(fabs(alpha[i]), beta[i]));
  __shared__ double shm[32];
  {
    double v = scale;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmax(m, shm[i]);
      shm[0] = m;
    }
    __syncthreads();
    scale = shm[0];
  }
  bool breakdown = !(nrm > 1e-12 * scale) || scale == 0.0;
  if (!breakdown) {
    double inv = 1.0 / nrm;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) qn[n] = w[n] * inv;
  } else {
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) qn[n] = rnd_sym(key, (uint64_t)j * 0x100000000ull + n);
  }
  if (threadIdx.x == 0) {
    alpha[j] = a;
    beta[j] = breakdown ? 0.0 : nrm;
    *flag = breakdown ? 1 : 0;
  }
}

// gated: q /= ||q||
__global__ void normalize_gated_kernel(double* q, int64_t N, const int* cond) {
  if (cond && !*cond) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s = fma(q[n], q[n], s);
  s = block_sum(s, sh);
  double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) q[n] *= inv;
}

__global__ void init_start_kernel(double* q, int64_t N, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    double v = rnd_sym(key, n);
    q[n] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  double inv = 1.0 / sqrt(s);
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) q[n] *= inv;
}

// ----------------------------------------------------- tridiagonal eigen
// Number of eigenvalues of T (diag a, off-diagonal b) below x (Sturm count).
__device__ int sturm_count(const double* a, const double* b, int m, double x, double pivmin) {
  int cnt = 0;
  double q = a[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// theta[c] = c-th largest eigenvalue of T_m (bisection to full precision).
__global__ void bisect_kernel(const double* a, const double* b, int m, int k, double* theta) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double lo = DBL_MAX, hi = -DBL_MAX, bmax2 = 0.0;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
    if (i < m - 1) bmax2 = fmax(bmax2, b[i] * b[i]);
  }
  double tnorm = fmax(fabs(lo), fabs(hi));
  double pivmin = DBL_MIN * fmax(1.0, bmax2);
  lo -= 2.0 * DBL_EPSILON * tnorm + pivmin;
  hi += 2.0 * DBL_EPSILON * tnorm + pivmin;
  int t = m - 1 - c;  // index from the smallest
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, m, mid, pivmin) <= t)
      lo = mid;
    else
      hi = mid;
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
  }
  theta[c] = 0.5 * (lo + hi);
}

// Eigenvectors of T_m for theta[0..k-1] by inverse iteration with a
// partially pivoted tridiagonal LU of (T - theta I).  One block; thread 0 runs
// the O(m) recurrences, all threads share the orthogonalisation against the
// vectors already found.  Y: k rows of length ldy.  res[c] = |beta_m y_c[m-1]|.
__global__ void inviter_kernel(const double* a, const double* b, int m, int k, const double* theta,
                               double* Y, int64_t ldy, double* scratch, double beta_m,
                               double* res, uint64_t key) {
  __shared__ double sh[32];
  double* d = scratch;
  double* du = scratch + m;
  double* dl = scratch + 2 * m;
  double* du2 = scratch + 3 * m;
  int* piv = reinterpret_cast<int*>(scratch + 4 * m);
  double tnorm = 0.0;
  for (int i = 0; i < m; ++i)
    tnorm = fmax(tnorm, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0));
  double tiny = DBL_EPSILON * fmax(tnorm, DBL_MIN);
  for (int c = 0; c < k; ++c) {
    double th = theta[c];
    double* y = Y + (int64_t)c * ldy;
    if (threadIdx.x == 0) {
      for (int i = 0; i < m; ++i) {
        d[i] = a[i] - th;
        if (i < m - 1) {
          du[i] = b[i];
          dl[i] = b[i];
        }
        du2[i] = 0.0;
      }
      for (int i = 0; i < m - 1; ++i) {
        if (fabs(d[i]) >= fabs(dl[i])) {
          piv[i] = 0;
          if (fabs(d[i]) < tiny) d[i] = d[i] < 0 ? -tiny : tiny;
          double f = dl[i] / d[i];
          dl[i] = f;
          d[i + 1] -= f * du[i];
        } else {
          piv[i] = 1;
          double f = d[i] / dl[i];
          d[i] = dl[i];
          dl[i] = f;
          double tmp = du[i];
          du[i] = d[i + 1];
          d[i + 1] = tmp - f * d[i + 1];
          if (i < m - 2) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du[i + 1];
          }
        }
      }
      if (fabs(d[m - 1]) < tiny) d[m - 1] = d[m - 1] < 0 ? -tiny : tiny;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = 1.0 + 0.25 * rnd_sym(key + c, i);
    __syncthreads();
    for (int it = 0; it < 4; ++it) {
      if (threadIdx.x == 0) {
        for (int i = 0; i < m - 1; ++i) {
          if (piv[i]) {
            double t = y[i];
            y[i] = y[i + 1];
            y[i + 1] = t;
          }
          y[i + 1] -= dl[i] * y[i];
        }
        y[m - 1] /= d[m - 1];
        if (m >= 2) y[m - 2] = (y[m - 2] - du[m - 2] * y[m - 1]) / d[m - 2];
        for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
      }
      __syncthreads();
      // scale to avoid overflow, then orthogonalise against earlier vectors (twice)
      double s = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) s = fmax(s, fabs(y[i]));
      {
        double v = s;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
          double mm = 0.0;
          for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) mm = fmax(mm, sh[i]);
          sh[0] = mm;
        }
        __syncthreads();
        s = sh[0];
        __syncthreads();
      }
      double inv = s > 0.0 ? 1.0 / s : 1.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= inv;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int p = 0; p < c; ++p) {
          const double* yp = Y + (int64_t)p * ldy;
          double dot = 0.0;
          for (int i = threadIdx.x; i < m; i += blockDim.x) dot = fma(yp[i], y[i], dot);
          dot = block_sum(dot, sh);
          for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] -= dot * yp[i];
          __syncthreads();
        }
      }
      double nn = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) nn = fma(y[i], y[i], nn);
      nn = block_sum(nn, sh);
      double inv2 = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= inv2;
      __syncthreads();
    }
    if (threadIdx.x == 0) res[c] = fabs(beta_m * y[m - 1]);
    __syncthreads();
  }
}

// Final per-column pass: evals, zero null columns, scale 1/sqrt(N mu),
// sign so that the largest-magnitude entry is positive.
__global__ void finalize_kernel(double* evecs, int64_t P, const double* theta, int k, double N,
                                double* evals, int* deficient) {
  __shared__ double shv[32];
  __shared__ int64_t shi[32];
  int c = blockIdx.x;
  double mu = theta[c], mu0 = theta[0];
  double* q = evecs + (int64_t)c * P;
  bool null_dir = !(mu > 1e-13 * mu0) || !(mu > 0.0);
  if (threadIdx.x == 0) {
    evals[c] = mu;
    if (null_dir) atomicExch(deficient, 1);
  }
  if (null_dir) {
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) q[i] = 0.0;
    return;
  }
  double sc = 1.0 / sqrt(N * mu);
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    double v = q[i] * sc;
    q[i] = v;
    if (fabs(v) > best) {
      best = fabs(v);
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, best, o);
    int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
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

__global__ void max_res_kernel(const double* res, int k, const double* theta, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double r = 0.0;
    for (int c = 0; c < k; ++c) r = fmax(r, res[c]);
    out[0] = r;
    out[1] = fabs(theta[0]);
  }
}

}  // namespace

hess_status topk_eig_gram(hess_mlp* h, const Net& net, const Caches<double>& c, int64_t N, int k,
                          double* evals_d, double* evecs_d, Arena& ar, bool dry, EigResult* res) {
  const int64_t P = net.P;
  const int L = net.L;
  int64_t mcap = N < (int64_t)8 * k + 512 ? N : (int64_t)8 * k + 512;
  double* M = ar.take<double>(N * N);
  double* DD = ar.take<double>(N * N);
  double* AA = ar.take<double>(N * N);
  double* G = ar.take<double>(N * P);
  double* Q = AA;  // reused once the Gram matrix is formed (mcap <= N)
  double* w = ar.take<double>(N);
  double* h1 = ar.take<double>(mcap + 1);
  double* h2 = ar.take<double>(mcap + 1);
  double* alpha = ar.take<double>(mcap + 1);
  double* beta = ar.take<double>(mcap + 1);
  double* theta = ar.take<double>(k);
  double* Y = ar.take<double>((int64_t)k * mcap);
  double* U = ar.take<double>(N * k);
  double* scratch = ar.take<double>(5 * (mcap + 1));
  double* rr = ar.take<double>(k);
  double* mx = ar.take<double>(2);
  int* flag = ar.take<int>(2);
  if (dry) return HESS_OK;
  cudaStream_t s = h->stream;

  // 1. Gram matrix, factored by layer
  HM_TRY(fill(M, N * N, 0.0, s));
  for (int wl = 1; wl <= L - 1; ++wl) {
    const int Tin = net.T[wl - 1], Tout = net.T[wl];
    Gemm<double> g;
    g.M = (int)N;
    g.N = (int)N;
    g.K = Tout;
    g.A = c.d[wl];
    g.sam = Tout;
    g.sak = 1;
    g.B = c.d[wl];
    g.sbk = 1;
    g.sbn = Tout;
    g.C = DD;
    g.scm = N;
    g.scn = 1;
    g.upper = 1;
    HM_TRY(gemm(g, s));
    g.K = Tin;
    g.A = c.a[wl - 1];
    g.sam = Tin;
    g.B = c.a[wl - 1];
    g.sbn = Tin;
    g.C = AA;
    HM_TRY(gemm(g, s));
    gram_acc_kernel<<<(unsigned)(cdiv(N * N, 256) < 65536 ? cdiv(N * N, 256) : 65536), 256, 0, s>>>(
        M, DD, AA, N * N, 1.0 / (double)N);
    HM_LAUNCHED();
  }
  HM_TRY(mirror_upper(M, N, N, s));

  // 2-3. Lanczos with full reorthogonalisation, extended until the top-k
  // residual bounds converge
  const uint64_t key = 0x5DEECE66Dull;
  init_start_kernel<<<1, 1024, 0, s>>>(Q, N, key);
  HM_LAUNCHED();
  int m = 0;
  int64_t target = N < (int64_t)2 * k + 32 ? N : (int64_t)2 * k + 32;
  if (target < k) target = k;
  const unsigned rows_blocks_N = (unsigned)cdiv(N, 8);
  const unsigned cols_blocks = (unsigned)cdiv(N, 256);
  bool converged = false;
  double* hp = h->host_pinned;
  while (true) {
    for (; m < target; ++m) {
      double* qj = Q + (int64_t)m * N;
      double* qn = Q + (int64_t)(m + 1) * N;
      gemv_rows_kernel<<<rows_blocks_N, 256, 0, s>>>(M, N, (int)N, N, qj, w, nullptr);
      HM_LAUNCHED();
      double* hs[2] = {h1, h2};
      for (int pass = 0; pass < 2; ++pass) {
        gemv_rows_kernel<<<(unsigned)cdiv(m + 1, 8), 256, 0, s>>>(Q, N, m + 1, N, w, hs[pass],
                                                                 nullptr);
        HM_LAUNCHED();
        gemv_sub_kernel<<<cols_blocks, 256, 0, s>>>(Q, N, m + 1, N, hs[pass], w, nullptr);
        HM_LAUNCHED();
      }
      if (m + 1 < mcap) {
        lanczos_norm_kernel<<<1, 1024, 0, s>>>(w, qn, N, m, h1, h2, alpha, beta, flag, key + 7);
        HM_LAUNCHED();
        for (int pass = 0; pass < 2; ++pass) {
          gemv_rows_kernel<<<(unsigned)cdiv(m + 1, 8), 256, 0, s>>>(Q, N, m + 1, N, qn, h1, flag);
          HM_LAUNCHED();
          gemv_sub_kernel<<<cols_blocks, 256, 0, s>>>(Q, N, m + 1, N, h1, qn, flag);
          HM_LAUNCHED();
        }
        normalize_gated_kernel<<<1, 1024, 0, s>>>(qn, N, flag);
        HM_LAUNCHED();
      } else {
        // last vector of the workspace: only alpha_m and beta_m are needed
        lanczos_norm_kernel<<<1, 1024, 0, s>>>(w, w, N, m, h1, h2, alpha, beta, flag, key + 7);
        HM_LAUNCHED();
      }
    }
    bisect_kernel<<<(unsigned)cdiv(k, 64), 64, 0, s>>>(alpha, beta, m, k, theta);
    HM_LAUNCHED();
    // beta[m-1] couples T_m to the next Lanczos vector
    HM_CUDA(cudaMemcpyAsync(hp, beta + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    double beta_m = hp[0];
    inviter_kernel<<<1, 256, 0, s>>>(alpha, beta, m, k, theta, Y, mcap, scratch, beta_m, rr, key + 11);
    HM_LAUNCHED();
    max_res_kernel<<<1, 32, 0, s>>>(rr, k, theta, mx);
    HM_LAUNCHED();
    HM_CUDA(cudaMemcpyAsync(hp, mx, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (hp[0] <= 1e-11 * hp[1] || m >= N) {
      converged = true;
      break;
    }
    if (m >= mcap) break;
    int64_t step = k > 32 ? k : 32;
    target = m + step;
    if (target > mcap) target = mcap;
    if (target > N) target = N;
  }
  res->lanczos_steps = m;
  res->converged = converged ? 1 : 0;

  // 4. Ritz vectors U = Q_m^T Y (N x k), back-projection through G
  {
    Gemm<double> g;
    g.M = (int)N;
    g.N = k;
    g.K = m;
    g.A = Q;
    g.sam = 1;
    g.sak = N;
    g.B = Y;
    g.sbk = 1;
    g.sbn = mcap;
    g.C = U;
    g.scm = k;
    g.scn = 1;
    HM_TRY(gemm(g, s));
  }
  HM_TRY(write_grads(net, c, G, P, s));
  {
    Gemm<double> g;
    g.M = (int)P;
    g.N = k;
    g.K = (int)N;
    g.A = G;
    g.sam = 1;
    g.sak = P;
    g.B = U;
    g.sbk = k;
    g.sbn = 1;
    g.C = evecs_d;
    g.scm = 1;
    g.scn = P;
    HM_TRY(gemm(g, s));
  }
  HM_CUDA(cudaMemsetAsync(flag + 1, 0, sizeof(int), s));
  finalize_kernel<<<k, 256, 0, s>>>(evecs_d, P, theta, k, (double)N, evals_d, flag + 1);
  HM_LAUNCHED();
  int* hi = reinterpret_cast<int*>(hp);
  HM_CUDA(cudaMemcpyAsync(hi, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  res->rank_deficient = hi[0];
  return HESS_OK;
}

}  // namespace hm
