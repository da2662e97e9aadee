// Top-k OPG eigenpairs in O(k P) device memory: neither the N x P gradient
// matrix, nor the N x N Gram matrix, nor the P x P OPG is ever formed.
//
// Sec. 5.4 reaches the OPG eigenpairs from mini-batches of examples
// (incremental SVD) so that memory stays O(K P) (Sec. 6); here the same
// bound holds for the uncentred OPG of Eq. J, computed exactly rather than by
// a truncated update.  The operator
//
//   v  ->  OPG v = (1/N) sum_chunks G_c^T (G_c v)
//
// is applied to a block of b vectors per pass over the data, chunk by chunk,
// and never with G_c itself: with g_n = [delta_n (x) a_n ; delta_n] per
// weight layer (W^(l-1) rows (i, j) output-major, then the biases),
//
//   (G_c V)[n, c]  = sum_layers sum_i delta[n][i] (sum_j a[n][j] V[(i, j), c] + V[b_i, c])
//   (G_c^T Z)[(i, j), c] = sum_n a[n][j] (delta[n][i] Z[n, c]),   [b_i, c] = sum_n delta[n][i] Z[n, c]
//
// each a GEMM over the layer's inputs (batched over the output units i) and
// a contraction with delta.  The eigenpairs come from a block Krylov method
// with Rayleigh-Ritz extraction and thick restarts: the basis V (m <= s b
// orthonormal vectors) and W = OPG V are kept; each pass appends the
// orthonormalised part of W's newest block outside span(V) (two classical
// Gram-Schmidt passes against V, then the block's columns one by one); the
// projected matrix T = V^T W (m x m) gives Ritz pairs (theta, V y) with
// residuals W y - theta V y, computed without another pass; when the basis
// is full it restarts from its leading Ritz vectors (V <- V Y, W <- W Y,
// T <- diag(theta)).  Memory: V and W (2 m P doubles), one chunk's
// forward/backward caches and two chunk x (T_out b) work arrays.
#include <cfloat>
#include <cmath>
#include <vector>

#include "devmath.cuh"
#include "internal.h"

namespace hm {
namespace {

unsigned blocks_for(int64_t n) {
  int64_t b = cdiv(n, 256);
  if (b > 16384) b = 16384;
  return (unsigned)(b < 1 ? 1 : b);
}

// Z[n][c] (+)= sum_i delta[n][i] (Y[n][i b + c] + Vb[c][i])  for one layer
// (Vb: the bias rows of the block, column c at Vb + c ldv)
template <typename T>
__global__ void lm_contract_kernel(const T* D, const T* Y, const T* Vb, int64_t ldv, int64_t nc, int Tout, int b,
                                   T* Z, int first) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc * b; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / b;
    const int c = (int)(t - n * b);
    const T* d = D + n * Tout;
    const T* y = Y + n * (int64_t)Tout * b + c;
    const T* vb = Vb + (int64_t)c * ldv;
    T acc = first ? (T)0 : Z[t];
    for (int i = 0; i < Tout; ++i) acc += d[i] * (y[(int64_t)i * b] + vb[i]);
    Z[t] = acc;
  }
}

// Bz[n][i b + c] = delta[n][i] Z[n][c]
template <typename T>
__global__ void lm_scale_kernel(const T* D, const T* Z, int64_t nc, int Tout, int b, T* Bz) {
  const int64_t cols = (int64_t)Tout * b;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / cols, r = t - n * cols;
    const int i = (int)(r / b), c = (int)(r - (int64_t)i * b);
    Bz[t] = D[n * Tout + i] * Z[n * b + c];
  }
}

// out[i] = (double) in[i] * s  (the FP64 copy of a block, scaled)
template <typename T>
__global__ void lm_to_f64_kernel(const T* in, double* out, int64_t n, double s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i] * s;
}

__global__ void lm_to_f32_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// Block-reduced squared norm of x (length n) into *out; one launch, many
// blocks, deterministic: partials by block, summed in order by block 0's
// last arrival.
__global__ void lm_norm2_kernel(const double* x, int64_t n, double* part, unsigned* count, double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], x[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += ((volatile double*)part)[b];
    *out = t;
    *count = 0u;
  }
}

// Normalise x given ||x||^2 = *nrm2 (before) and the squared norm *ref2 it
// had before its projections: when less than 1e-20 of it is left (the
// vector lay in the basis), x is replaced by a counter-based random vector
// (projected again by the caller) and *fresh is set.
__global__ void lm_normalise_kernel(double* x, int64_t n, const double* nrm2, const double* ref2, uint64_t key,
                                    int* fresh) {
  const double v = *nrm2, r = *ref2;
  const bool dead = !(v > 1e-20 * r) || !(v > 0.0);
  if (dead) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      x[i] = rnd_sym(key, (uint64_t)i);
    if (blockIdx.x == 0 && threadIdx.x == 0) *fresh = 1;
    return;
  }
  const double inv = 1.0 / sqrt(v);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
}

// x *= 1 / sqrt(*nrm2) (after a random replacement, whose norm is not small)
__global__ void lm_scale_by_norm_kernel(double* x, int64_t n, const double* nrm2) {
  const double v = *nrm2;
  const double inv = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
}

// coef[i] = V[i] . x for rows i < nr (one block per row, length P)
__global__ void lm_rowdots_kernel(const double* V, int64_t P, const double* x, double* coef) {
  __shared__ double sh[32];
  const double* v = V + (int64_t)blockIdx.x * P;
  double s = 0.0;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s = fma(v[p], x[p], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) coef[blockIdx.x] = s;
}

// x[p] -= sum_{i < nr} coef[i] V[i][p]
__global__ void lm_rowaxpy_kernel(const double* V, int64_t P, int nr, const double* coef, double* x) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[p];
    for (int i = 0; i < nr; ++i) acc = fma(-coef[i], V[(int64_t)i * P + p], acc);
    x[p] = acc;
  }
}

// Residual norms of the Ritz pairs: res[c] = ||R[c] - theta_c X[c]|| over
// rows of length P (R = W y_c, X = V y_c); one block per pair.
__global__ void lm_residual_kernel(const double* R, const double* X, const double* theta, int64_t P, double* res) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const double th = theta[c];
  const double* r = R + (int64_t)c * P;
  const double* x = X + (int64_t)c * P;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double d = r[i] - th * x[i];
    s = fma(d, d, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) res[c] = sqrt(s);
}

// Eigenvector output: row c of X to evecs (normalised, largest-magnitude
// entry positive; null when theta_c <= 1e-13 theta_0, as the Gram route).
__global__ void lm_output_kernel(const double* X, const double* theta, int k, int64_t P, double* evecs,
                                 double* evals, int* deficient) {
  __shared__ double sh[32];
  __shared__ double shv[32];
  __shared__ int64_t shi[32];
  const int c = blockIdx.x;
  const double mu = theta[c], mu0 = theta[0];
  const double* x = X + (int64_t)c * P;
  double* q = evecs + (int64_t)c * P;
  const bool null_dir = !(mu > 1e-13 * mu0) || !(mu > 0.0);
  if (threadIdx.x == 0) {
    evals[c] = mu;
    if (null_dir) atomicExch(deficient, 1);
  }
  if (null_dir) {
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) q[i] = 0.0;
    return;
  }
  double s = 0.0, best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double v = x[i];
    s = fma(v, v, s);
    if (fabs(v) > best) {
      best = fabs(v);
      bi = i;
    }
  }
  s = block_sum(s, sh);
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
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (shv[w] > shv[0] || (shv[w] == shv[0] && shi[w] < shi[0])) {
        shv[0] = shv[w];
        shi[0] = shi[w];
      }
  }
  __syncthreads();
  const double sc = (x[shi[0]] < 0.0 ? -1.0 : 1.0) / sqrt(s);
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) q[i] = x[i] * sc;
}

// Tc (r x r, compact) from the projected matrix T (leading dimension ld),
// whose entry (i, j), i <= j, was computed with column j (the block of a
// column holds every earlier row): Tc[i][j] = Tc[j][i] = T[min][max].
__global__ void lm_compact_kernel(const double* T, int64_t ld, int64_t r, double* Tc) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / r, j = t - i * r;
    Tc[t] = i <= j ? T[i * ld + j] : T[j * ld + i];
  }
}

// T = diag(theta_0 .. theta_{keep-1}) (leading dimension ld, ld x ld), after
// a thick restart
__global__ void lm_diag_kernel(double* T, int64_t ld, const double* theta, int keep) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ld * ld; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ld, c = t - r * ld;
    T[t] = (r == c && r < keep) ? theta[r] : 0.0;
  }
}

}  // namespace
}  // namespace hm

namespace hm {
namespace {

// Device buffers of one call (all in the handle's second workspace).
template <typename T>
struct LmBufs {
  int64_t P = 0, chunk = 0, b = 0, mmax = 0, kk = 0;
  double *V = nullptr, *W = nullptr, *NB = nullptr, *Tm = nullptr, *Tc = nullptr, *theta = nullptr, *Yv = nullptr;
  double *X = nullptr, *R = nullptr, *res = nullptr, *coef = nullptr, *scal = nullptr, *part = nullptr;
  double *evs = nullptr, *qs = nullptr;  // output staging (host outputs)
  char* split = nullptr;                 // split-K scratch of the SIMT GEMMs
  unsigned* count = nullptr;
  int* flag = nullptr;
  T *xs = nullptr, *ys = nullptr, *Vt = nullptr, *Wt = nullptr, *Yb = nullptr, *Bz = nullptr, *Zc = nullptr;
  Caches<T> c;
};

constexpr int kNormBlocks = 256;

template <typename T>
void plan_lm(Arena& ar, const Net& net, int64_t chunk, int64_t b, int64_t mmax, int64_t kk, int k, bool stage,
             LmBufs<T>& f) {
  const int64_t P = net.P;
  f.P = P;
  f.chunk = chunk;
  f.b = b;
  f.mmax = mmax;
  f.kk = kk;
  f.V = ar.take<double>(mmax * P);
  f.W = ar.take<double>(mmax * P);
  f.NB = ar.take<double>(b * P);
  f.Tm = ar.take<double>(mmax * mmax);
  f.Tc = ar.take<double>(mmax * mmax);
  f.theta = ar.take<double>(kk);
  f.Yv = ar.take<double>(kk * mmax);
  f.X = ar.take<double>(kk * P);
  f.R = ar.take<double>(kk * P);
  f.res = ar.take<double>(kk);
  f.coef = ar.take<double>(mmax + b);
  f.scal = ar.take<double>(4);
  f.part = ar.take<double>(kNormBlocks);
  f.count = ar.take<unsigned>(1);
  f.flag = ar.take<int>(2);
  f.split = ar.take<char>(kSplitBytes);
  f.evs = stage ? ar.take<double>(k) : nullptr;
  f.qs = stage ? ar.take<double>((int64_t)k * P) : nullptr;
  int maxTout = 0;
  for (int l = 1; l < net.L; ++l) maxTout = net.T[l] > maxTout ? net.T[l] : maxTout;
  f.xs = ar.take<T>(chunk * net.T[0]);
  f.ys = ar.take<T>(chunk * net.T[net.L - 1]);
  f.Vt = sizeof(T) == sizeof(double) ? nullptr : ar.take<T>(b * P);
  f.Wt = sizeof(T) == sizeof(double) ? nullptr : ar.take<T>(b * P);
  f.Yb = ar.take<T>(chunk * maxTout * b);
  f.Bz = ar.take<T>(chunk * maxTout * b);
  f.Zc = ar.take<T>(chunk * b);
  plan_caches(ar, net, chunk, f.c);
}

// Wblk (b rows of P) = OPG Vblk: one pass over the data in chunks; the
// products with G_c are layer GEMMs and contractions with delta (no G_c).
template <typename T>
hess_status lm_apply(hess_mlp* h, const void* X, const void* Y, int x_dev, int y_dev, int64_t N, const double* Vblk,
                     double* Wblk, LmBufs<T>& f, cudaStream_t s) {
  const Net& net = h->net;
  const int64_t P = f.P, b = f.b, T1 = net.T[0], TL = net.T[net.L - 1];
  const bool dbl = sizeof(T) == sizeof(double);
  const T* Vt = dbl ? reinterpret_cast<const T*>(Vblk) : f.Vt;
  T* Wt = dbl ? reinterpret_cast<T*>(Wblk) : f.Wt;
  if (!dbl) {
    lm_to_f32_kernel<<<blocks_for(b * P), 256, 0, s>>>(Vblk, reinterpret_cast<float*>(f.Vt), b * P);
    HM_LAUNCHED();
  }
  HM_CUDA(cudaMemsetAsync(Wt, 0, (size_t)b * P * sizeof(T), s));
  const T* omega = dbl ? reinterpret_cast<const T*>(h->omega64) : reinterpret_cast<const T*>(h->omega32);
  for (int64_t n0 = 0; n0 < N; n0 += f.chunk) {
    const int64_t nc = N - n0 < f.chunk ? N - n0 : f.chunk;
    const T* Xc = reinterpret_cast<const T*>(X) + n0 * T1;
    const T* Yc = reinterpret_cast<const T*>(Y) + n0 * TL;
    if (!x_dev) {
      HM_CUDA(cudaMemcpyAsync(f.xs, Xc, (size_t)nc * T1 * sizeof(T), cudaMemcpyHostToDevice, s));
      Xc = f.xs;
    }
    if (!y_dev) {
      HM_CUDA(cudaMemcpyAsync(f.ys, Yc, (size_t)nc * TL * sizeof(T), cudaMemcpyHostToDevice, s));
      Yc = f.ys;
    }
    Caches<T> c = f.c;
    c.N = nc;
    HM_TRY(forward_backward<T>(net, omega, Xc, Yc, c, s));
    // Z = G_c V (nc x b)
    for (int wl = 1; wl <= net.L - 1; ++wl) {
      const int Tin = net.T[wl - 1], Tout = net.T[wl];
      Gemm<T> g;
      g.M = (int)nc;
      g.N = (int)b;
      g.K = Tin;
      g.A = c.a[wl - 1];
      g.sam = Tin;
      g.sak = 1;
      g.B = Vt + net.woff[wl - 1];
      g.sbk = 1;
      g.sbn = P;
      g.bsb = Tin;
      g.C = f.Yb;
      g.scm = (int64_t)Tout * b;
      g.scn = 1;
      g.bsc = b;
      g.batch = Tout;
      HM_TRY(gemm(g, s));
      lm_contract_kernel<T><<<blocks_for(nc * b), 256, 0, s>>>(c.d[wl], f.Yb, Vt + net.boff[wl - 1], P, nc, Tout,
                                                               (int)b, f.Zc, wl == 1 ? 1 : 0);
      HM_LAUNCHED();
    }
    // W += G_c^T Z
    for (int wl = 1; wl <= net.L - 1; ++wl) {
      const int Tin = net.T[wl - 1], Tout = net.T[wl];
      lm_scale_kernel<T><<<blocks_for(nc * Tout * b), 256, 0, s>>>(c.d[wl], f.Zc, nc, Tout, (int)b, f.Bz);
      HM_LAUNCHED();
      Gemm<T> g;
      g.M = Tin;
      g.N = (int)b;
      g.K = (int)nc;
      g.beta = 1;
      g.A = c.a[wl - 1];
      g.sam = 1;
      g.sak = Tin;
      g.B = f.Bz;
      g.sbk = (int64_t)Tout * b;
      g.sbn = 1;
      g.bsb = b;
      g.C = Wt + net.woff[wl - 1];
      g.scm = 1;
      g.scn = P;
      g.bsc = Tin;
      g.batch = Tout;
      HM_TRY(gemm(g, s));
      Gemm<T> gb;
      gb.M = Tout;
      gb.N = (int)b;
      gb.K = (int)nc;
      gb.beta = 1;
      gb.A = c.d[wl];
      gb.sam = 1;
      gb.sak = Tout;
      gb.B = f.Zc;
      gb.sbk = b;
      gb.sbn = 1;
      gb.C = Wt + net.boff[wl - 1];
      gb.scm = 1;
      gb.scn = P;
      HM_TRY(gemm(gb, s));
    }
  }
  lm_to_f64_kernel<T><<<blocks_for(b * P), 256, 0, s>>>(Wt, Wblk, b * P, 1.0 / (double)N);
  HM_LAUNCHED();
  return HESS_OK;
}

// Rows x_c (c < nrows) of the buffer at Xr (stride P): each orthogonalised
// twice against rows 0 .. r0 + c - 1 of V (which the rows themselves follow
// when Xr == V + r0 P), normalised; a row with nothing left outside the
// span becomes a counter-based random direction, orthogonalised the same way.
hess_status lm_orthonormalise(double* V, int64_t P, int64_t r0, int64_t nrows, double* coef, double* scal,
                              double* part, unsigned* count, int* fresh, uint64_t key, cudaStream_t s) {
  auto project = [&](double* x, int64_t r) -> hess_status {
    if (r == 0) return HESS_OK;
    lm_rowdots_kernel<<<(unsigned)r, 256, 0, s>>>(V, P, x, coef);
    HM_LAUNCHED();
    lm_rowaxpy_kernel<<<blocks_for(P), 256, 0, s>>>(V, P, (int)r, coef, x);
    HM_LAUNCHED();
    return HESS_OK;
  };
  const unsigned nb = blocks_for(P) < (unsigned)kNormBlocks ? blocks_for(P) : (unsigned)kNormBlocks;
  for (int64_t c = 0; c < nrows; ++c) {
    double* x = V + (r0 + c) * P;
    const int64_t r = r0 + c;
    lm_norm2_kernel<<<nb, 256, 0, s>>>(x, P, part, count, scal + 0);
    HM_LAUNCHED();
    HM_TRY(project(x, r));
    HM_TRY(project(x, r));
    lm_norm2_kernel<<<nb, 256, 0, s>>>(x, P, part, count, scal + 1);
    HM_LAUNCHED();
    lm_normalise_kernel<<<nb, 256, 0, s>>>(x, P, scal + 1, scal + 0, key + (uint64_t)r * 0x9E3779B97F4A7C15ull,
                                           fresh);
    HM_LAUNCHED();
    // (a no-op for a row already orthonormal; a random replacement gets its
    // two passes here)
    HM_TRY(project(x, r));
    HM_TRY(project(x, r));
    lm_norm2_kernel<<<nb, 256, 0, s>>>(x, P, part, count, scal + 2);
    HM_LAUNCHED();
    lm_scale_by_norm_kernel<<<nb, 256, 0, s>>>(x, P, scal + 2);
    HM_LAUNCHED();
  }
  return HESS_OK;
}

}  // namespace
}  // namespace hm

namespace hm {
namespace {

template <typename T>
hess_status lowmem_run(hess_mlp* h, const void* X, const void* Y, int x_dev, int y_dev, int64_t N, int k, int64_t b,
                       int64_t mmax, int64_t kk, double tol, int max_passes, int64_t chunk, double* evals, int ev_dev,
                       double* evecs, int q_dev, int* passes_out, int* deficient_out) {
  const Net& net = h->net;
  const int64_t P = net.P;
  cudaStream_t s = h->stream;
  // workspace: the basis and chunk buffers in the second workspace, the
  // projected eigensolver in the first
  Arena a2;
  LmBufs<T> f;
  const bool stage = !ev_dev || !q_dev;
  plan_lm(a2, net, chunk, b, mmax, kk, k, stage, f);
  HM_TRY(ensure_ws2(h, a2.off));
  Arena ae;
  EigResult er;
  HM_TRY(topk_eig_dense(h, nullptr, mmax, (int)kk, nullptr, nullptr, ae, true, &er));
  HM_TRY(ensure_ws(h, ae.off));
  a2 = Arena{h->ws2, 0};
  plan_lm(a2, net, chunk, b, mmax, kk, k, stage, f);
  double* evd = ev_dev ? evals : f.evs;
  double* eqd = q_dev ? evecs : f.qs;
  // the basis products have long K (P) and few output tiles: split K
  SplitGuard sg(f.split, kSplitBytes, h->sm_count);
  const uint64_t key = 0xC0FFEE5EEDull;
  std::vector<double> hv((size_t)(kk > k ? kk : k) + 2);
  double* hp = hv.data();
  HM_CUDA(cudaMemsetAsync(f.count, 0, sizeof(unsigned), s));
  HM_CUDA(cudaMemsetAsync(f.flag, 0, 2 * sizeof(int), s));
  // the first block: counter-based random rows, orthonormalised
  HM_CUDA(cudaMemsetAsync(f.V, 0, (size_t)b * P * sizeof(double), s));
  {
    Tick t0(h, HESS_K_EIG, 0.0, 0.0);
    HM_TRY(lm_orthonormalise(f.V, P, 0, b, f.coef, f.scal, f.part, f.count, f.flag, key, s));
  }
  int64_t r = b;      // rows of the basis
  int64_t cur = 0;    // first row of its newest block
  int passes = 0;
  bool converged = false;
  int64_t kc = 0;     // Ritz pairs of the last extraction
  while (passes < max_passes) {
    {
      Tick t(h, HESS_K_LOWMEM, 4.0 * (double)N * P * b, 0.0);
      HM_TRY(lm_apply<T>(h, X, Y, x_dev, y_dev, N, f.V + cur * P, f.W + cur * P, f, s));
    }
    ++passes;
    Tick te(h, HESS_K_EIG, 2.0 * P * r * b + 4.0 * P * r * kk, 0.0);
    // the new columns of T = V^T W: rows 0..r-1, columns cur..r-1 (leading
    // dimension mmax); then the compact symmetric r x r copy
    {
      Gemm<double> g;
      g.M = (int)r;
      g.N = (int)b;
      g.K = (int)P;
      g.A = f.V;
      g.sam = P;
      g.sak = 1;
      g.B = f.W + cur * P;
      g.sbk = 1;
      g.sbn = P;
      g.C = f.Tm + cur;
      g.scm = mmax;
      g.scn = 1;
      HM_TRY(gemm(g, s));
    }
    lm_compact_kernel<<<blocks_for(r * r), 256, 0, s>>>(f.Tm, mmax, r, f.Tc);
    HM_LAUNCHED();
    kc = kk < r ? kk : r;
    Arena ar{h->ws, 0};
    HM_TRY(topk_eig_dense(h, f.Tc, r, (int)kc, f.theta, f.Yv, ar, false, &er));
    // Ritz vectors X = Y^T V and W Y: the top k for the residuals now, the
    // rest of the kept ones only at a restart
    auto ritz = [&](int64_t c0, int64_t c1) -> hess_status {
      if (c1 <= c0) return HESS_OK;
      for (int w = 0; w < 2; ++w) {
        Gemm<double> g;
        g.M = (int)(c1 - c0);
        g.N = (int)P;
        g.K = (int)r;
        g.A = f.Yv + c0 * r;
        g.sam = r;
        g.sak = 1;
        g.B = w == 0 ? f.V : f.W;
        g.sbk = P;
        g.sbn = 1;
        g.C = (w == 0 ? f.X : f.R) + c0 * P;
        g.scm = P;
        g.scn = 1;
        HM_TRY(gemm(g, s));
      }
      return HESS_OK;
    };
    const int64_t kr = kc < k ? kc : k;
    HM_TRY(ritz(0, kr));
    lm_residual_kernel<<<(unsigned)kr, 256, 0, s>>>(f.R, f.X, f.theta, P, f.res);
    HM_LAUNCHED();
    // (the top k pairs exist once the basis has k vectors)
    HM_CUDA(cudaMemcpyAsync(hp, f.theta, sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(hp + 1, f.res, (size_t)kr * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    te.stop();
    HM_TRY(take_sticky_error(h));
    double worst = 0.0;
    for (int64_t c = 0; c < kr; ++c) worst = hp[1 + c] > worst ? hp[1 + c] : worst;
    if ((kr == k && worst <= tol * hp[0]) || r >= P) {
      converged = true;
      break;
    }
    if (passes >= max_passes) break;
    Tick tb(h, HESS_K_EIG, 0.0, 0.0);
    // the next block: W's newest rows; when the basis is full they are first
    // projected out of the whole basis (twice), so that the block carries the
    // new Krylov directions across the restart that follows
    HM_CUDA(cudaMemcpyAsync(f.NB, f.W + cur * P, (size_t)b * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (r + b > mmax) {
      for (int pass2 = 0; pass2 < 2; ++pass2) {
        // C = V[0:r] NB^T (r x b), NB -= C^T V[0:r]
        Gemm<double> g;
        g.M = (int)r;
        g.N = (int)b;
        g.K = (int)P;
        g.A = f.V;
        g.sam = P;
        g.sak = 1;
        g.B = f.NB;
        g.sbk = 1;
        g.sbn = P;
        g.C = f.Tc;  // (free until the next extraction)
        g.scm = b;
        g.scn = 1;
        HM_TRY(gemm(g, s));
        Gemm<double> u;
        u.M = (int)b;
        u.N = (int)P;
        u.K = (int)r;
        u.alpha = -1.0;
        u.beta = 1.0;
        u.A = f.Tc;
        u.sam = 1;
        u.sak = b;
        u.B = f.V;
        u.sbk = P;
        u.sbn = 1;
        u.C = f.NB;
        u.scm = P;
        u.scn = 1;
        HM_TRY(gemm(u, s));
      }
      // thick restart from the leading Ritz pairs (V <- V Y, W <- W Y,
      // T <- diag(theta)); null Ritz values do not make basis vectors
      HM_CUDA(cudaMemcpyAsync(hp + 1, f.theta, (size_t)kc * sizeof(double), cudaMemcpyDeviceToHost, s));
      HM_CUDA(cudaStreamSynchronize(s));
      int64_t keep = mmax - b < kc ? mmax - b : kc;
      while (keep > 0 && !(hp[1 + keep - 1] > 1e-13 * hp[1])) --keep;
      HM_TRY(ritz(kr, keep));
      HM_CUDA(cudaMemcpyAsync(f.V, f.X, (size_t)keep * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
      HM_CUDA(cudaMemcpyAsync(f.W, f.R, (size_t)keep * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
      lm_diag_kernel<<<blocks_for(mmax * mmax), 256, 0, s>>>(f.Tm, mmax, f.theta, (int)keep);
      HM_LAUNCHED();
      r = keep;
    }
    HM_CUDA(cudaMemcpyAsync(f.V + r * P, f.NB, (size_t)b * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HM_TRY(lm_orthonormalise(f.V, P, r, b, f.coef, f.scal, f.part, f.count, f.flag, key + (uint64_t)passes, s));
    cur = r;
    r += b;
  }
  *passes_out = passes;
  if (!converged) return set_error(HESS_ERR_NOT_CONVERGED, "block Krylov did not converge in %d passes", passes);
  HM_CUDA(cudaMemsetAsync(f.flag + 1, 0, sizeof(int), s));
  lm_output_kernel<<<k, 256, 0, s>>>(f.X, f.theta, k, P, eqd, evd, f.flag + 1);
  HM_LAUNCHED();
  if (!ev_dev) HM_CUDA(cudaMemcpyAsync(evals, evd, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!q_dev) HM_CUDA(cudaMemcpyAsync(evecs, eqd, (size_t)k * P * sizeof(double), cudaMemcpyDeviceToHost, s));
  int defi = 0;
  HM_CUDA(cudaMemcpyAsync(&defi, f.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  *deficient_out = defi;
  return HESS_OK;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" hess_status opg_topk_eig_lowmem(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                           hess_precision prec, int64_t chunk, int block, double* evals,
                                           double* evecs, int* passes) {
  clear_error();
  if (!h) return set_error(HESS_ERR_INVALID_ARG, "handle is NULL");
  if (N < 1 || N > ((int64_t)1 << 40)) return set_error(HESS_ERR_INVALID_ARG, "N must be in 1 .. 2^40");
  if (prec != HESS_FP64 && prec != HESS_FP32)
    return set_error(HESS_ERR_INVALID_ARG, "precision must be HESS_FP64 or HESS_FP32 (got %d)", (int)prec);
  const Net& net = h->net;
  const int64_t P = net.P;
  if (k < 1 || k > N || k > P)
    return set_error(HESS_ERR_INVALID_ARG, "need 1 <= k <= min(N, P) (k = %d, N = %lld, P = %lld)", k, (long long)N,
                     (long long)P);
  if (!X || !Y || !evals || !evecs) return set_error(HESS_ERR_INVALID_ARG, "X, Y, evals and evecs must be non-NULL");
  if (chunk < 1 || chunk > (1ll << 31) - 1)
    return set_error(HESS_ERR_INVALID_ARG, "chunk must be in 1 .. 2^31 - 1 (got %lld)", (long long)chunk);
  if (block < 0) return set_error(HESS_ERR_INVALID_ARG, "block must be >= 0 (0: the default)");
  HM_TRY(take_sticky_error(h));
  Guard g(h->device);
  int x_dev = 0, y_dev = 0, ev_dev = 0, q_dev = 0;
  HM_TRY(locate(h, X, "X", &x_dev));
  HM_TRY(locate(h, Y, "Y", &y_dev));
  HM_TRY(locate(h, evals, "evals", &ev_dev));
  HM_TRY(locate(h, evecs, "evecs", &q_dev));
  if (chunk > N) chunk = N;
  // block size and basis: b vectors per pass, at most mmax in the basis
  // (room for the kept Ritz vectors and one more block); a small P takes
  // the whole space in one block
  int64_t b = block > 0 ? block : (k < 16 ? 16 : (k > 128 ? 128 : k));
  int64_t mmax = 6 * b > k + 3 * b ? 6 * b : k + 3 * b;
  if (P <= mmax || b >= P) {
    b = P;
    mmax = P;
  }
  const int64_t kk = mmax - b > k ? (mmax - b < 2 * k + b ? mmax - b : 2 * k + b) : (mmax < k ? mmax : k);
  const double tol = prec == HESS_FP64 ? 1e-10 : 1e-5;
  const int max_passes = 300;
  int np = 0, deficient = 0;
  const hess_status st =
      prec == HESS_FP64
          ? lowmem_run<double>(h, X, Y, x_dev, y_dev, N, k, b, mmax, kk, tol, max_passes, chunk, evals, ev_dev, evecs,
                               q_dev, &np, &deficient)
          : lowmem_run<float>(h, X, Y, x_dev, y_dev, N, k, b, mmax, kk, tol, max_passes, chunk, evals, ev_dev, evecs,
                              q_dev, &np, &deficient);
  if (passes) *passes = np;
  if (st != HESS_OK) {
    cudaStreamSynchronize(h->stream);
    return st;
  }
  HM_TRY(take_sticky_error(h));
  if (deficient) return set_error(HESS_ERR_RANK_DEFICIENT, "some of the top-%d OPG eigenvalues are null", k);
  return HESS_OK;
}
