// SIMT kernels of the plain FP64 / FP32 path: strided GEMM, the forward and
// backward passes of the MLP, the per-example gradient writer, the batched
// R-operator over blocks of unit directions, and the symmetric scatter that
// places Hessian row blocks and their mirror images; and the double-float
// product of the eigen step's forward pass through a wide layer.
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "devmath.cuh"
#include "internal.h"

namespace hm {

// ====================================================================== GEMM
template <typename T>
struct GemmCfg;
template <>
struct GemmCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct GemmCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
// narrow outputs (<= 32 columns, e.g. the k eigenvector columns, or a layer
// of at most 32 units)
struct GemmCfgNarrow64 {
  static constexpr int BM = 128, BN = 32, BK = 16, TM = 8, TN = 2;
};
// very narrow outputs (<= 16 columns): no idle half tile
struct GemmCfgNarrow16 {
  static constexpr int BM = 128, BN = 16, BK = 16, TM = 8, TN = 1;
};
// tiny outputs (at most 16 x 16, e.g. a contraction over the examples into a
// small weight block): one entry per thread, K split across blocks
struct GemmCfgTiny {
  static constexpr int BM = 16, BN = 16, BK = 16, TM = 1, TN = 1;
};

// Row of the upper-triangular tile enumeration: row r holds nt - r tiles and
// S(r) = r*nt - r*(r-1)/2 tiles come before it.
__device__ __forceinline__ void upper_tile(long long t, int nt, int& tm, int& tn) {
  double b = 2.0 * nt + 1.0;
  int r = (int)floor((b - sqrt(fmax(b * b - 8.0 * (double)t, 0.0))) * 0.5);
  if (r < 0) r = 0;
  if (r > nt - 1) r = nt - 1;
  auto S = [nt](long long rr) { return rr * nt - rr * (rr - 1) / 2; };
  while (r > 0 && S(r) > t) --r;
  while (r + 1 < nt && S(r + 1) <= t) ++r;
  tm = r;
  tn = r + (int)(t - S(r));
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_kernel(Gemm<T> g, int splits, T* part) {
  constexpr int NT = (BM / TM) * (BN / TN);
  static_assert(NT == 256, "256 threads");
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  int tm, tn;
  if (g.upper) {
    upper_tile(blockIdx.x, (g.M + BM - 1) / BM, tm, tn);
  } else {
    tm = blockIdx.x;
    tn = blockIdx.y;
  }
  // blockIdx.z = batch * splits + slice; a slice owns K range [kbeg, kend)
  const int bz = blockIdx.z / splits, slice = blockIdx.z % splits;
  const T* A = g.A + (int64_t)bz * g.bsa;
  const T* B = g.B + (int64_t)bz * g.bsb;
  T* C = g.C + (int64_t)bz * g.bsc;
  const int kchunk = ((g.K + splits - 1) / splits + BK - 1) / BK * BK;
  const int kbeg = slice * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = (int64_t)tm * BM, n0 = (int64_t)tn * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  const bool a_m_fast = (g.sam == 1);
  const bool b_n_fast = (g.sbn == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int it = 0; it < BM * BK / NT; ++it) {
      int e = tid + it * NT;
      int mm, kk;
      if (a_m_fast) {
        mm = e % BM;
        kk = e / BM;
      } else {
        kk = e % BK;
        mm = e / BK;
      }
      int64_t m = m0 + mm;
      int k = k0 + kk;
      As[kk][mm] = (m < g.M && k < kend) ? A[m * g.sam + (int64_t)k * g.sak] : T(0);
    }
#pragma unroll
    for (int it = 0; it < BN * BK / NT; ++it) {
      int e = tid + it * NT;
      int nn, kk;
      if (b_n_fast) {
        nn = e % BN;
        kk = e / BN;
      } else {
        kk = e % BK;
        nn = e / BK;
      }
      int64_t n = n0 + nn;
      int k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < kend) ? B[(int64_t)k * g.sbk + n * g.sbn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (part) {
    // split-K: raw partial sums, [slice][batch][M][N]
    T* pp = part + ((int64_t)slice * (gridDim.z / splits) + bz) * (int64_t)g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int64_t m = m0 + ty + i * (BM / TM);
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int64_t n = n0 + tx + j * (BN / TN);
        if (n < g.N) pp[m * g.N + n] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * (BM / TM);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx + j * (BN / TN);
      if (n >= g.N) continue;
      T* c = C + m * g.scm + n * g.scn;
      T v = g.alpha * acc[i][j];
      if (g.beta != T(0)) v += g.beta * (*c);
      *c = v;
    }
  }
}

// Short K: one thread per output entry, the products accumulated in k order
// (the order of the tiled kernel, so the two give the same bits).
template <typename T>
__global__ void gemm_smallk_kernel(Gemm<T> g) {
  const int64_t mn = (int64_t)g.M * g.N;
  const int64_t total = mn * g.batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bz = idx / mn, r = idx % mn;
    const int64_t m = r / g.N, n = r % g.N;
    const T* A = g.A + bz * g.bsa + m * g.sam;
    const T* B = g.B + bz * g.bsb + n * g.sbn;
    T acc = T(0);
    for (int k = 0; k < g.K; ++k) acc = fma(A[k * g.sak], B[k * g.sbk], acc);
    T* c = g.C + bz * g.bsc + m * g.scm + n * g.scn;
    T v = g.alpha * acc;
    if (g.beta != T(0)) v += g.beta * (*c);
    *c = v;
  }
}

// Sum the split-K partials in slice order and apply alpha / beta: one thread
// per output, or (few outputs) one warp per output with the lanes over the
// slices and a fixed-order warp sum.
template <typename T>
__global__ void splitk_reduce_kernel(Gemm<T> g, int splits, const T* part) {
  const int64_t mn = (int64_t)g.M * g.N;
  const int64_t total = mn * g.batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / mn, r = idx % mn;
    const int64_t m = r / g.N, n = r % g.N;
    T acc = T(0);
    for (int sl = 0; sl < splits; ++sl) acc += part[((int64_t)sl * g.batch + b) * mn + r];
    T* c = g.C + b * g.bsc + m * g.scm + n * g.scn;
    T v = g.alpha * acc;
    if (g.beta != T(0)) v += g.beta * (*c);
    *c = v;
  }
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__global__ void splitk_reduce_warp_kernel(Gemm<T> g, int splits, const T* part) {
  const int64_t mn = (int64_t)g.M * g.N;
  const int64_t total = mn * g.batch;
  const int64_t idx = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= total) return;
  const int64_t b = idx / mn, r = idx % mn;
  const int64_t m = r / g.N, n = r % g.N;
  T a0 = T(0), a1 = T(0);
  int sl = lane;
  for (; sl + 32 < splits; sl += 64) {
    a0 += part[((int64_t)sl * g.batch + b) * mn + r];
    a1 += part[((int64_t)(sl + 32) * g.batch + b) * mn + r];
  }
  if (sl < splits) a0 += part[((int64_t)sl * g.batch + b) * mn + r];
  const T acc = warp_sum_t(a0 + a1);
  if (lane == 0) {
    T* c = g.C + b * g.bsc + m * g.scm + n * g.scn;
    T v = g.alpha * acc;
    if (g.beta != T(0)) v += g.beta * (*c);
    *c = v;
  }
}

thread_local SplitScratch g_split;

// Column sums: block (32 x 32), threadIdx.x over 32 adjacent columns r
// (coalesced), threadIdx.y over 32 slices of n; the slices meet in shared
// memory.
template <typename T>
__global__ void colsum_kernel(const T* A, int64_t lda, int64_t R, int64_t K, T alpha, T* out,
                              int64_t ostride) {
  __shared__ T part[32][33];
  const int64_t r = blockIdx.x * (int64_t)32 + threadIdx.x;
  T a0 = T(0), a1 = T(0);
  if (r < R) {
    int64_t n = threadIdx.y;
    for (; n + 32 < K; n += 64) {
      a0 += A[n * lda + r];
      a1 += A[(n + 32) * lda + r];
    }
    if (n < K) a0 += A[n * lda + r];
  }
  part[threadIdx.y][threadIdx.x] = a0 + a1;
  __syncthreads();
  if (threadIdx.y == 0 && r < R) {
    T acc = T(0);
    for (int y = 0; y < 32; ++y) acc += part[y][threadIdx.x];
    out[r * ostride] = alpha * acc;
  }
}
template <typename T>
hess_status colsum(const T* A, int64_t lda, int64_t R, int64_t K, T alpha, T* out, int64_t ostride,
                   cudaStream_t s) {
  if (R <= 0) return HESS_OK;
  colsum_kernel<T><<<(unsigned)cdiv(R, 32), dim3(32, 32), 0, s>>>(A, lda, R, K, alpha, out, ostride);
  HM_LAUNCHED();
  return HESS_OK;
}
template hess_status colsum<double>(const double*, int64_t, int64_t, int64_t, double, double*,
                                    int64_t, cudaStream_t);
template hess_status colsum<float>(const float*, int64_t, int64_t, int64_t, float, float*, int64_t,
                                   cudaStream_t);

template <typename T, typename Cfg>
static hess_status gemm_cfg(const Gemm<T>& g, cudaStream_t s) {
  if (g.batch > 65535) return set_error(HESS_ERR_INVALID_ARG, "gemm batch %d too large", g.batch);
  int64_t tiles;
  dim3 grid;
  if (g.upper) {
    int64_t nt = cdiv(g.M, Cfg::BM);
    tiles = nt * (nt + 1) / 2;
    grid = dim3((unsigned)tiles, 1, g.batch);
  } else {
    int64_t gy = cdiv(g.N, Cfg::BN);
    if (gy > 65535) return set_error(HESS_ERR_INVALID_ARG, "gemm N %d too large", g.N);
    tiles = cdiv(g.M, Cfg::BM) * gy;
    grid = dim3((unsigned)cdiv(g.M, Cfg::BM), (unsigned)gy, g.batch);
  }
  // split K when the output tiles cannot fill the GPU (deterministic: the
  // partials are summed in slice order by a second kernel)
  int splits = 1;
  const int sms = g_split.sms > 0 ? g_split.sms : 148;
  // (FP64 runs at a small fraction of the FP32 rate, so FP64 products split
  // down to slices of 16; FP32 products on the narrow 128-row tiles, whose
  // blocks carry little work per K step, down to slices of 32)
  constexpr bool narrow = Cfg::BM == 128 && Cfg::BN <= 32;
  const int64_t kmin = std::is_same<T, double>::value ? 64 : (narrow ? 64 : 256);
  const int64_t kslice = std::is_same<T, double>::value ? 16 : (narrow ? 32 : 128);
  if (!g.upper && g_split.p && tiles * g.batch < 2 * sms && g.K >= kmin) {
    int64_t maxs = g.K / kslice;
    int64_t cap = (int64_t)(g_split.bytes / ((size_t)g.M * g.N * g.batch * sizeof(T)));
    if (maxs > cap) maxs = cap;
    if (maxs > 64) maxs = 64;
    if ((int64_t)g.batch * maxs > 65535) maxs = 65535 / g.batch;
    // the split with the least work per SM: waves of blocks times the K
    // range of a block (slices are whole BK steps, so some splits leave
    // empty slices or an idle tail wave)
    int64_t best = 1, best_cost = INT64_MAX;
    for (int64_t sp = 1; sp <= maxs; ++sp) {
      const int64_t kc = cdiv(cdiv(g.K, sp), Cfg::BK) * Cfg::BK;
      const int64_t eff = cdiv(g.K, kc);
      const int64_t cost = cdiv(tiles * g.batch * eff, sms) * kc;
      if (cost < best_cost) {
        best_cost = cost;
        best = sp;
      }
    }
    if (best >= 2) splits = (int)best;
  }
  if (splits > 1) {
    grid.z = g.batch * splits;
    T* part = reinterpret_cast<T*>(g_split.p);
    gemm_kernel<T, Cfg::BM, Cfg::BN, Cfg::BK, Cfg::TM, Cfg::TN><<<grid, 256, 0, s>>>(g, splits, part);
    HM_LAUNCHED();
    int64_t total = (int64_t)g.M * g.N * g.batch;
    if (total <= 8 * sms * 8) {
      splitk_reduce_warp_kernel<T><<<(unsigned)cdiv(total, 8), 256, 0, s>>>(g, splits, part);
    } else {
      int64_t blocks = cdiv(total, 256);
      if (blocks > 65536) blocks = 65536;
      splitk_reduce_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(g, splits, part);
    }
    HM_LAUNCHED();
    return HESS_OK;
  }
  gemm_kernel<T, Cfg::BM, Cfg::BN, Cfg::BK, Cfg::TM, Cfg::TN><<<grid, 256, 0, s>>>(g, 1, nullptr);
  HM_LAUNCHED();
  return HESS_OK;
}
// Shape dispatch.  Skinny problems waste most of a tile (and, in FP64, whose
// rate per SM partition is small, the idle lanes cost as much as busy ones),
// so:
//   K <= 32 and a narrow output     -> one thread per entry
//   M, N <= 16                      -> 16 x 16 tiles (split K)
//   M < 32 <= 4 M <= N              -> the transposed problem C^T = B^T A^T
//   N <= 16 / N <= 32               -> 128 x 16 / 128 x 32 tiles
template <typename T>
hess_status gemm(const Gemm<T>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return HESS_OK;
  if (g.batch > 65535) return set_error(HESS_ERR_INVALID_ARG, "gemm batch %d too large", g.batch);
  const int64_t entries = (int64_t)g.M * g.N;
  if (!g.upper && g.K <= 32 && (g.N <= 32 || entries <= 16384)) {
    int64_t blocks = cdiv(entries * g.batch, 256);
    if (blocks > 65536) blocks = 65536;
    gemm_smallk_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(g);
    HM_LAUNCHED();
    return HESS_OK;
  }
  if (!g.upper && g.M <= 16 && g.N <= 16) return gemm_cfg<T, GemmCfgTiny>(g, s);
  if (!g.upper && g.M < 32 && g.N >= 4 * g.M) {
    Gemm<T> t = g;
    t.M = g.N;
    t.N = g.M;
    t.A = g.B;
    t.sam = g.sbn;
    t.sak = g.sbk;
    t.bsa = g.bsb;
    t.B = g.A;
    t.sbk = g.sak;
    t.sbn = g.sam;
    t.bsb = g.bsa;
    t.scm = g.scn;
    t.scn = g.scm;
    return gemm(t, s);
  }
  if (!g.upper && g.N <= 16) return gemm_cfg<T, GemmCfgNarrow16>(g, s);
  if (!g.upper && g.N <= 32) return gemm_cfg<T, GemmCfgNarrow64>(g, s);
  return gemm_cfg<T, GemmCfg<T>>(g, s);
}
template hess_status gemm<double>(const Gemm<double>&, cudaStream_t);
template hess_status gemm<float>(const Gemm<float>&, cudaStream_t);

// ============================================================= elementwise
template <typename T>
__global__ void fill_kernel(T* p, int64_t n, T v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
template <typename T>
hess_status fill(T* p, int64_t n, T v, cudaStream_t s) {
  if (n <= 0) return HESS_OK;
  int64_t blocks = cdiv(n, 256);
  if (blocks > 65536) blocks = 65536;
  fill_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p, n, v);
  HM_LAUNCHED();
  return HESS_OK;
}
template hess_status fill<double>(double*, int64_t, double, cudaStream_t);
template hess_status fill<float>(float*, int64_t, float, cudaStream_t);

template <typename Ti, typename To>
__global__ void convert_kernel(const Ti* in, To* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}
template <typename Ti, typename To>
hess_status convert(const Ti* in, To* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return HESS_OK;
  int64_t blocks = cdiv(n, 256);
  if (blocks > 65536) blocks = 65536;
  convert_kernel<Ti, To><<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
  HM_LAUNCHED();
  return HESS_OK;
}
template hess_status convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template hess_status convert<float, double>(const float*, double*, int64_t, cudaStream_t);

// =========================================================== activations
// Hidden activation value and its first two derivatives (ReLU: sigma'(0) = 0).
__device__ __forceinline__ void act_eval(int act, double z, double& a, double& d1, double& d2) {
  if (act == HESS_ACT_SIGMOID) {
    double s = 1.0 / (1.0 + exp(-z));
    a = s;
    d1 = s * (1.0 - s);
    d2 = d1 * (1.0 - 2.0 * s);
  } else if (act == HESS_ACT_TANH) {
    double t = tanh(z);
    a = t;
    d1 = 1.0 - t * t;
    d2 = -2.0 * t * d1;
  } else {
    a = z > 0.0 ? z : 0.0;
    d1 = z > 0.0 ? 1.0 : 0.0;
    d2 = 0.0;
  }
}
__device__ __forceinline__ void act_eval(int act, float z, float& a, float& d1, float& d2) {
  if (act == HESS_ACT_SIGMOID) {
    float s = 1.0f / (1.0f + expf(-z));
    a = s;
    d1 = s * (1.0f - s);
    d2 = d1 * (1.0f - 2.0f * s);
  } else if (act == HESS_ACT_TANH) {
    float t = tanhf(z);
    a = t;
    d1 = 1.0f - t * t;
    d2 = -2.0f * t * d1;
  } else {
    a = z > 0.0f ? z : 0.0f;
    d1 = z > 0.0f ? 1.0f : 0.0f;
    d2 = 0.0f;
  }
}

template <typename T>
__global__ void bias_act_kernel(const T* Z, const T* b, int64_t N, int Tn, int act, T* A, T* S1,
                                T* S2) {
  int64_t n_el = N * Tn;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % Tn);
    T a, d1, d2;
    act_eval(act, Z[idx] + b[i], a, d1, d2);
    A[idx] = a;
    S1[idx] = d1;
    S2[idx] = d2;
  }
}

// Softmax output with the log-sum-exp in FP64; delta^(L) = p * sum(y) - y.
// One warp per example, the lanes over the classes; the xor-butterfly sums
// leave the same bits in every lane (IEEE addition commutes).
template <typename T>
__global__ void softmax_kernel(const T* Z, const T* b, const T* Y, int64_t N, int TL, T* Pout,
                               T* D, T* ysum) {
  const int64_t n = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (n >= N) return;  // whole warps
  const T* z = Z + n * TL;
  const T* y = Y + n * TL;
  double m = -INFINITY;
  for (int i = lane; i < TL; i += 32) m = fmax(m, (double)z[i] + (double)b[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  double s = 0.0, ys = 0.0;
  for (int i = lane; i < TL; i += 32) {
    s += exp((double)z[i] + (double)b[i] - m);
    ys += (double)y[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    ys += __shfl_xor_sync(0xffffffffu, ys, o);
  }
  const double lse = m + log(s);
  for (int i = lane; i < TL; i += 32) {
    const double p = exp((double)z[i] + (double)b[i] - lse);
    Pout[n * TL + i] = (T)p;
    D[n * TL + i] = (T)(p * ys - (double)y[i]);
  }
  if (lane == 0) ysum[n] = (T)ys;
}

template <typename T>
__global__ void mul_kernel(const T* a, const T* b, T* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

static unsigned grid1d(int64_t n, int threads = 256) {
  int64_t b = cdiv(n, threads);
  if (b > 1 << 20) b = 1 << 20;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T>
void plan_caches(Arena& ar, const Net& net, int64_t N, Caches<T>& c) {
  const int L = net.L;
  c.N = N;
  int maxT = 0;
  for (int j = 0; j < L; ++j) maxT = net.T[j] > maxT ? net.T[j] : maxT;
  for (int j = 1; j <= L - 2; ++j) {
    c.a[j] = ar.take<T>(N * net.T[j]);
    c.s1[j] = ar.take<T>(N * net.T[j]);
    c.s2[j] = ar.take<T>(N * net.T[j]);
    c.e[j] = ar.take<T>(N * net.T[j]);
  }
  for (int j = 1; j <= L - 1; ++j) c.d[j] = ar.take<T>(N * net.T[j]);
  c.p = ar.take<T>(N * net.T[L - 1]);
  c.ysum = ar.take<T>(N);
  c.z = ar.take<T>(N * maxT);
}
template void plan_caches<double>(Arena&, const Net&, int64_t, Caches<double>&);
template void plan_caches<float>(Arena&, const Net&, int64_t, Caches<float>&);

// Forward pass (Sec. 2, Eq. modelfunc) and per-example back-propagation of
// dC_n/dz^(l) (the per-example errors delta^(l)).
// Z[n][o] = sum_i A[n][i] W[o][i] (A: N x K, W: T x K, Z: N x T, all FP64
// row-major) in double-float arithmetic (devmath.cuh, about 48 significant
// bits, on the FP32 pipe, where this GPU's FP64 rate would make the product
// of a wide layer the longest launch of the pass).  Block (16, 8, 8): 16
// outputs o (x) of 8 examples n (y), the entries of K dealt to z by residue
// mod 8 and the 8 partial sums added at the end in order of z; the 8 rows of
// A and 16 rows of W staged in shared
// memory as hi/lo pairs, kDfgK entries of K at a time (all of K, for the
// layer widths of the workloads), with every load of a stage in flight at
// once.
constexpr int kDfgK = 1024;
size_t gemm_nt_df_smem(int K) {
  const int kc = K < kDfgK ? K : kDfgK;
  return (size_t)24 * (kc + 1) * sizeof(float2);
}
constexpr int kDfgZ = 8;
__global__ void __launch_bounds__(16 * 8 * kDfgZ) gemm_nt_df_kernel(const double* A, int64_t N, int K,
                                                                     const double* W, int T, double* Z) {
  extern __shared__ float2 gsh[];
  __shared__ float2 part[kDfgZ][8][16];
  const int kc = K < kDfgK ? K : kDfgK, ld = kc + 1;  // (odd row stride: no bank conflicts)
  float2* as = gsh;             // 8 x ld
  float2* ws = gsh + 8 * ld;    // 16 x ld
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + 16 * ty + 128 * tz, nthr = 16 * 8 * kDfgZ;
  const int64_t n = (int64_t)blockIdx.x * 8 + ty;
  const int o = blockIdx.y * 16 + tx;
  float s = 0.0f, c = 0.0f;
  for (int k0 = 0; k0 < K; k0 += kc) {
    const int kn = K - k0 < kc ? K - k0 : kc;
    // the 24 rows' entries k0 .. k0 + kn: eight loads in flight per thread
    const int total = 24 * kn;
    for (int e0 = tid; e0 < total; e0 += nthr * 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nthr;
        const int r = e / kn, k = e - r * kn;
        v[u] = 0.0;
        if (e < total) {
          if (r < 8) {
            const int64_t nr = (int64_t)blockIdx.x * 8 + r;
            if (nr < N) v[u] = A[nr * K + k0 + k];
          } else {
            const int orow = blockIdx.y * 16 + (r - 8);
            if (orow < T) v[u] = W[(int64_t)orow * K + k0 + k];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nthr;
        if (e < total) {
          const int r = e / kn, k = e - r * kn;
          gsh[r * ld + k] = df_split_bits(v[u]);  // (as, then ws: rows 8 .. 23)
        }
      }
    }
    __syncthreads();
    const float2* ar = as + ty * ld;
    const float2* wr = ws + tx * ld;
#pragma unroll 4
    for (int k = tz; k < kn; k += kDfgZ) df_mac(ar[k], wr[k], s, c);
    __syncthreads();
  }
  part[tz][ty][tx] = df_norm(s, c);
  __syncthreads();
  if (tz == 0 && n < N && o < T) {
    float ss = 0.0f, cs = 0.0f;
    for (int z = 0; z < kDfgZ; ++z) df_acc(part[z][ty][tx], ss, cs);
    Z[n * T + o] = df_val(df_norm(ss, cs));
  }
}

hess_status gemm_nt_df_attributes() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(gemm_nt_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gemm_nt_df_smem(kDfgK));
  });
  if (e != cudaSuccess) return set_error(HESS_ERR_CUDA, "double-float product attributes: %s", cudaGetErrorString(e));
  return HESS_OK;
}

template <typename T>
hess_status forward_backward(const Net& net, const T* omega, const T* X, const T* Y, Caches<T>& c,
                             cudaStream_t s, bool df_wide) {
  const int L = net.L;
  const int64_t N = c.N;
  c.a[0] = X;
  for (int w = 1; w <= L - 1; ++w) {
    const int Tin = net.T[w - 1], Tout = net.T[w];
    if constexpr (std::is_same<T, double>::value) {
      if (df_wide && Tin >= 128) {
        HM_TRY(gemm_nt_df_attributes());
        const dim3 grid((unsigned)cdiv(N, 8), (unsigned)cdiv(Tout, 16));
        gemm_nt_df_kernel<<<grid, dim3(16, 8, kDfgZ), gemm_nt_df_smem(Tin), s>>>(c.a[w - 1], N, Tin,
                                                                             omega + net.woff[w - 1], Tout, c.z);
        HM_LAUNCHED();
        const T* b = omega + net.boff[w - 1];
        if (w < L - 1) {
          bias_act_kernel<T><<<grid1d(N * Tout), 256, 0, s>>>(c.z, b, N, Tout, net.act[w - 1],
                                                              const_cast<T*>(c.a[w]), c.s1[w], c.s2[w]);
        } else {
          softmax_kernel<T><<<(unsigned)cdiv(N, 8), 256, 0, s>>>(c.z, b, Y, N, Tout, c.p, c.d[w], c.ysum);
        }
        HM_LAUNCHED();
        continue;
      }
    }
    Gemm<T> g;
    g.M = (int)N;
    g.N = Tout;
    g.K = Tin;
    g.A = c.a[w - 1];
    g.sam = Tin;
    g.sak = 1;
    g.B = omega + net.woff[w - 1];
    g.sbk = 1;
    g.sbn = Tin;
    g.C = c.z;
    g.scm = Tout;
    g.scn = 1;
    HM_TRY(gemm(g, s));
    const T* b = omega + net.boff[w - 1];
    if (w < L - 1) {
      bias_act_kernel<T><<<grid1d(N * Tout), 256, 0, s>>>(c.z, b, N, Tout, net.act[w - 1],
                                                          const_cast<T*>(c.a[w]), c.s1[w], c.s2[w]);
      HM_LAUNCHED();
    } else {
      softmax_kernel<T><<<(unsigned)cdiv(N, 8), 256, 0, s>>>(c.z, b, Y, N, Tout, c.p, c.d[w],
                                                                c.ysum);
      HM_LAUNCHED();
    }
  }
  for (int j = L - 2; j >= 1; --j) {
    // e_j = delta_{j+1} W^(j+1)   (W^(j+1) is T[j+1] x T[j])
    Gemm<T> g;
    g.M = (int)N;
    g.N = net.T[j];
    g.K = net.T[j + 1];
    g.A = c.d[j + 1];
    g.sam = net.T[j + 1];
    g.sak = 1;
    g.B = omega + net.woff[j];
    g.sbk = net.T[j];
    g.sbn = 1;
    g.C = c.e[j];
    g.scm = net.T[j];
    g.scn = 1;
    HM_TRY(gemm(g, s));
    mul_kernel<T><<<grid1d(N * net.T[j]), 256, 0, s>>>(c.s1[j], c.e[j], c.d[j], N * net.T[j]);
    HM_LAUNCHED();
  }
  return HESS_OK;
}
template hess_status forward_backward<double>(const Net&, const double*, const double*,
                                              const double*, Caches<double>&, cudaStream_t, bool);
template hess_status forward_backward<float>(const Net&, const float*, const float*, const float*,
                                             Caches<float>&, cudaStream_t, bool);

// ================================================== per-example gradients
// G[n, woff + i*Tin + k] = delta[n,i] a[n,k];  G[n, boff + i] = delta[n,i].
// Block (n, y) writes rows i in [16 y, 16 y + 16) of example n's outer
// product: consecutive threads take consecutive k (coalesced stores, no
// index division), a[n,k] is loaded once per k and delta[n,i] is a broadcast.
constexpr int kGradRows = 16;
template <typename T>
__global__ void write_grads_kernel(const T* D, const T* A, int Tin, int Tout, T* G, int64_t ldg,
                                   int64_t woff, int64_t boff) {
  const int64_t n = blockIdx.x;
  const int i0 = blockIdx.y * kGradRows;
  const int i1 = min(Tout, i0 + kGradRows);
  const T* d = D + n * Tout;
  const T* a = A + n * Tin;
  T* g = G + n * ldg;
  for (int k = threadIdx.x; k < Tin; k += blockDim.x) {
    const T ak = a[k];
    T* gk = g + woff + (int64_t)i0 * Tin + k;
#pragma unroll 4
    for (int i = i0; i < i1; ++i, gk += Tin) *gk = d[i] * ak;
  }
  for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) g[boff + i] = d[i];
}

template <typename T>
hess_status write_grads(const Net& net, const Caches<T>& c, T* G, int64_t ldg, cudaStream_t s) {
  for (int w = 1; w <= net.L - 1; ++w) {
    const int Tin = net.T[w - 1], Tout = net.T[w];
    const int64_t gy = cdiv(Tout, kGradRows);
    if (gy > 65535) return set_error(HESS_ERR_INVALID_ARG, "layer of %d units too wide for the gradient writer", Tout);
    const int threads = Tin >= 256 ? 256 : (Tin >= 128 ? 128 : (Tin >= 64 ? 64 : 32));
    int64_t n0 = 0;
    while (n0 < c.N) {
      int64_t nb = c.N - n0 < 2147483647 ? c.N - n0 : 2147483647;
      write_grads_kernel<T><<<dim3((unsigned)nb, (unsigned)gy), threads, 0, s>>>(
          c.d[w] + n0 * Tout, c.a[w - 1] + n0 * Tin, Tin, Tout, G + n0 * ldg, ldg, net.woff[w - 1],
          net.boff[w - 1]);
      HM_LAUNCHED();
      n0 += nb;
    }
  }
  return HESS_OK;
}
template hess_status write_grads<double>(const Net&, const Caches<double>&, double*, int64_t,
                                         cudaStream_t);
template hess_status write_grads<float>(const Net&, const Caches<float>&, float*, int64_t,
                                        cudaStream_t);

// ======================================================= mirror / scatter
// Copy the strict upper triangle of an n x n matrix onto the lower one,
// through a 32 x 32 shared-memory tile so both sides are coalesced.
template <typename T>
__global__ void mirror_upper_kernel(T* C, int64_t n, int64_t ldc) {
  __shared__ T tile[32][33];
  int64_t ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  int64_t r0 = ti * 32, c0 = tj * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t r = r0 + y, cc = c0 + threadIdx.x;
    if (r < n && cc < n) tile[y][threadIdx.x] = C[r * ldc + cc];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t r = c0 + y, cc = r0 + threadIdx.x;  // destination (r, cc) = source (cc, r)
    if (r < n && cc < n && r > cc) C[r * ldc + cc] = tile[threadIdx.x][y];
  }
}
template <typename T>
hess_status mirror_upper(T* C, int64_t n, int64_t ldc, cudaStream_t s) {
  int64_t nt = cdiv(n, 32);
  if (nt > 65535) return set_error(HESS_ERR_INVALID_ARG, "mirror: n too large");
  mirror_upper_kernel<T><<<dim3((unsigned)nt, (unsigned)nt), dim3(32, 8), 0, s>>>(C, n, ldc);
  HM_LAUNCHED();
  return HESS_OK;
}
template hess_status mirror_upper<double>(double*, int64_t, int64_t, cudaStream_t);
template hess_status mirror_upper<float>(float*, int64_t, int64_t, cudaStream_t);

// tmp is B x cols (row d holds H[d0 + d, c0 .. c0 + cols)).  Entries on or
// above the diagonal (column >= d0 + d) go to row d0 + d; those strictly
// above it are also written to row c (the mirror image), coalesced through a
// shared tile.  Every entry of H is thus written once from one computation
// and once as its mirror, so H is exactly symmetric.
template <typename T>
__global__ void scatter_sym_kernel(const T* tmp, int B, int64_t cols, int64_t c0, int64_t d0, T* H,
                                   int64_t P) {
  __shared__ T tile[32][33];
  int64_t dt = (int64_t)blockIdx.y * 32, ct = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t d = dt + y, cl = ct + threadIdx.x;
    T v = T(0);
    if (d < B && cl < cols) {
      v = tmp[d * cols + cl];
      int64_t c = c0 + cl;
      if (c >= d0 + d) H[(d0 + d) * P + c] = v;
    }
    tile[y][threadIdx.x] = v;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    int64_t cl = ct + y, d = dt + threadIdx.x;
    if (d < B && cl < cols) {
      int64_t c = c0 + cl;
      if (c > d0 + d) H[c * P + d0 + d] = tile[threadIdx.x][y];
    }
  }
}
template <typename T>
hess_status scatter_sym(const T* tmp, int B, int64_t cols, int64_t c0, int64_t d0, T* H, int64_t P,
                        cudaStream_t s) {
  int64_t gx = cdiv(cols, 32), gy = cdiv(B, 32);
  if (gy > 65535) return set_error(HESS_ERR_INVALID_ARG, "scatter: block too large");
  scatter_sym_kernel<T><<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, s>>>(tmp, B, cols, c0,
                                                                                d0, H, P);
  HM_LAUNCHED();
  return HESS_OK;
}
template hess_status scatter_sym<double>(const double*, int, int64_t, int64_t, int64_t, double*,
                                         int64_t, cudaStream_t);
template hess_status scatter_sym<float>(const float*, int, int64_t, int64_t, int64_t, float*,
                                        int64_t, cudaStream_t);

// ============================================================ R-operator
// Layout of every R-quantity: [n][d][t] (example, direction, unit).
//
// Seed: a unit direction inside weight layer jm only moves z at position jm:
//   direction W^(jm)_{pq}:  R{z}[n, d, t] = [t == p] a^(jm-1)[n, q]
//   direction b^(jm+1)_p:   R{z}[n, d, t] = [t == p]
template <typename T>
__global__ void rop_seed_kernel(T* rz, int B, int64_t N, int Tm, int Tin, const T* aprev,
                                int64_t loc0) {
  const int64_t n_el = N * B * Tm;
  const int64_t nW = (int64_t)Tm * Tin;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(idx % Tm);
    int64_t r = idx / Tm;
    int d = (int)(r % B);
    int64_t n = r / B;
    int64_t loc = loc0 + d;
    T v = T(0);
    if (loc < nW) {
      int p = (int)(loc / Tin), q = (int)(loc % Tin);
      if (t == p) v = aprev[n * Tin + q];
    } else if (t == (int)(loc - nW)) {
      v = T(1);
    }
    rz[idx] = v;
  }
}

// R{a} = sigma'(z) R{z}
template <typename T>
__global__ void rop_act_kernel(const T* rz, const T* s1, T* ra, int B, int64_t N, int Tn) {
  const int64_t n_el = N * B * Tn;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(idx % Tn);
    int64_t n = idx / ((int64_t)Tn * B);
    ra[idx] = s1[n * Tn + t] * rz[idx];
  }
}

// Softmax output: R{delta^(L)} = (diag p - p p^T) R{z^(L)} * sum(y).
template <typename T>
__global__ void rop_softmax_kernel(const T* rz, const T* p, const T* ysum, T* rd, int B, int64_t N,
                                   int TL) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= N * B) return;
  int64_t n = r / B;
  const T* z = rz + r * TL;
  const T* pn = p + n * TL;
  T sdot = T(0);
  for (int i = 0; i < TL; ++i) sdot += pn[i] * z[i];
  T ys = ysum[n];
  for (int i = 0; i < TL; ++i) rd[r * TL + i] = pn[i] * (z[i] - sdot) * ys;
}

// R{delta^(l-1)} = sigma''(z) R{z} e + sigma'(z) (W^T R{delta^(l)})
template <typename T>
__global__ void rop_back_kernel(const T* rz, const T* tmp, const T* s1, const T* s2, const T* e,
                                T* rd, int B, int64_t N, int Tn) {
  const int64_t n_el = N * B * Tn;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(idx % Tn);
    int64_t n = idx / ((int64_t)Tn * B);
    int64_t q = n * Tn + t;
    rd[idx] = s2[q] * rz[idx] * e[q] + s1[q] * tmp[idx];
  }
}

template <typename T>
void plan_rop(Arena& ar, const Net& net, int64_t N, int jm, int B, RopBufs<T>& r) {
  const int L = net.L;
  r.B = B;
  r.rz.assign(L, nullptr);
  r.ra.assign(L, nullptr);
  r.rd.assign(L, nullptr);
  int maxT = 0;
  for (int j = jm; j <= L - 1; ++j) {
    r.rz[j] = ar.take<T>(N * B * net.T[j]);
    r.rd[j] = ar.take<T>(N * B * net.T[j]);
    if (j <= L - 2) r.ra[j] = ar.take<T>(N * B * net.T[j]);
    maxT = net.T[j] > maxT ? net.T[j] : maxT;
  }
  r.tmp = ar.take<T>(N * B * maxT);
  r.ones = ar.take<T>(N);
  r.ones_ready = false;
}
template void plan_rop<double>(Arena&, const Net&, int64_t, int, int, RopBufs<double>&);
template void plan_rop<float>(Arena&, const Net&, int64_t, int, int, RopBufs<float>&);

// Forward-over-reverse R-operator for the unit directions d0..d0+B-1 (all in
// weight layer jm).  Only positions >= jm are touched: below the direction's
// layer every R-quantity is zero, and the Hessian columns needed for the upper
// triangle all lie in layers >= jm.
template <typename T>
hess_status rop_block(const Net& net, const T* omega, const Caches<T>& c, int jm, int64_t d0, int B,
                      RopBufs<T>& r, cudaStream_t s) {
  const int L = net.L;
  const int64_t N = c.N;
  {
    const int Tm = net.T[jm], Tin = net.T[jm - 1];
    rop_seed_kernel<T><<<grid1d(N * B * Tm), 256, 0, s>>>(r.rz[jm], B, N, Tm, Tin, c.a[jm - 1],
                                                         d0 - net.woff[jm - 1]);
    HM_LAUNCHED();
  }
  for (int j = jm; j <= L - 2; ++j) {
    const int Tj = net.T[j], Tn = net.T[j + 1];
    rop_act_kernel<T><<<grid1d(N * B * Tj), 256, 0, s>>>(r.rz[j], c.s1[j], r.ra[j], B, N, Tj);
    HM_LAUNCHED();
    // R{z}_{j+1} = R{a}_j W^(j+1)^T  (W^(j+1) is Tn x Tj); V^(j+1) = 0 here
    Gemm<T> g;
    g.M = (int)(N * B);
    g.N = Tn;
    g.K = Tj;
    g.A = r.ra[j];
    g.sam = Tj;
    g.sak = 1;
    g.B = omega + net.woff[j];
    g.sbk = 1;
    g.sbn = Tj;
    g.C = r.rz[j + 1];
    g.scm = Tn;
    g.scn = 1;
    HM_TRY(gemm(g, s));
  }
  {
    const int TL = net.T[L - 1];
    rop_softmax_kernel<T><<<(unsigned)cdiv(N * B, 128), 128, 0, s>>>(r.rz[L - 1], c.p, c.ysum,
                                                                      r.rd[L - 1], B, N, TL);
    HM_LAUNCHED();
  }
  for (int j = L - 2; j >= jm; --j) {
    const int Tj = net.T[j], Tn = net.T[j + 1];
    // tmp = R{delta}_{j+1} W^(j+1)
    Gemm<T> g;
    g.M = (int)(N * B);
    g.N = Tj;
    g.K = Tn;
    g.A = r.rd[j + 1];
    g.sam = Tn;
    g.sak = 1;
    g.B = omega + net.woff[j];
    g.sbk = Tj;
    g.sbn = 1;
    g.C = r.tmp;
    g.scm = Tj;
    g.scn = 1;
    HM_TRY(gemm(g, s));
    rop_back_kernel<T><<<grid1d(N * B * Tj), 256, 0, s>>>(r.rz[j], r.tmp, c.s1[j], c.s2[j], c.e[j],
                                                         r.rd[j], B, N, Tj);
    HM_LAUNCHED();
  }
  return HESS_OK;
}
template hess_status rop_block<double>(const Net&, const double*, const Caches<double>&, int,
                                       int64_t, int, RopBufs<double>&, cudaStream_t);
template hess_status rop_block<float>(const Net&, const float*, const Caches<float>&, int, int64_t,
                                      int, RopBufs<float>&, cudaStream_t);

// Hessian rows d0..d0+B-1 against the columns of weight layer jl:
//   H[d, W(i,k)] = (1/N) sum_n R{delta}[n,d,i] a[n,k] + delta[n,i] R{a}[n,d,k]
//   H[d, b(i)]   = (1/N) sum_n R{delta}[n,d,i]
// (the R-operator applied to dC_n/dW = delta a^T and dC_n/db = delta).
template <typename T>
hess_status contract_layer(const Net& net, const Caches<T>& c, const RopBufs<T>& r, int jm, int jl,
                           int64_t d0, T* tmp, T* H, cudaStream_t s) {
  const int64_t N = c.N;
  const int B = r.B;
  const int Tin = net.T[jl - 1], Tout = net.T[jl];
  const int64_t nW = (int64_t)Tin * Tout;
  T* tmpW = tmp;
  T* tmpB = tmp + (int64_t)B * nW;
  const T invN = T(1) / T(N);
  // W columns all left of the block's first direction lie below the diagonal
  // (their values arrive through the mirror of earlier blocks): skip them
  const bool w_needed = net.woff[jl - 1] + nW > d0;
  if (w_needed) {
    // rows (d, i), columns k
    Gemm<T> g;
    g.M = B * Tout;
    g.N = Tin;
    g.K = (int)N;
    g.alpha = invN;
    g.A = r.rd[jl];
    g.sam = 1;
    g.sak = (int64_t)B * Tout;
    g.B = c.a[jl - 1];
    g.sbk = Tin;
    g.sbn = 1;
    g.C = tmpW;
    g.scm = Tin;
    g.scn = 1;
    HM_TRY(gemm(g, s));
  }
  if (w_needed && jl > jm) {
    // batched over d: rows k, columns i
    Gemm<T> g;
    g.M = Tin;
    g.N = Tout;
    g.K = (int)N;
    g.alpha = invN;
    g.beta = T(1);
    g.A = r.ra[jl - 1];
    g.sam = 1;
    g.sak = (int64_t)B * Tin;
    g.bsa = Tin;
    g.B = c.d[jl];
    g.sbk = Tout;
    g.sbn = 1;
    g.bsb = 0;
    g.C = tmpW;
    g.scm = 1;
    g.scn = Tin;
    g.bsc = nW;
    g.batch = B;
    HM_TRY(gemm(g, s));
  }
  // bias columns: (1/N) sum_n R{delta}[n, d, i]
  HM_TRY(colsum(r.rd[jl], (int64_t)B * Tout, (int64_t)B * Tout, N, invN, tmpB, (int64_t)1, s));
  if (w_needed) HM_TRY(scatter_sym(tmpW, B, nW, net.woff[jl - 1], d0, H, net.P, s));
  HM_TRY(scatter_sym(tmpB, B, (int64_t)Tout, net.boff[jl - 1], d0, H, net.P, s));
  return HESS_OK;
}
template hess_status contract_layer<double>(const Net&, const Caches<double>&,
                                            const RopBufs<double>&, int, int, int64_t, double*,
                                            double*, cudaStream_t);
template hess_status contract_layer<float>(const Net&, const Caches<float>&, const RopBufs<float>&,
                                           int, int, int64_t, float*, float*, cudaStream_t);

// ============================================ Hessian-vector products
// Direction-bias term and activation of the R-forward pass for general
// directions: R{z}[n, d, t] += v_d(b)[t]; hidden positions also get
// R{a} = sigma'(z) R{z}.  Layout [n][d][t].
template <typename T>
__global__ void hvp_bias_act_kernel(T* rz, const T* V, int64_t ldv, int64_t boff, int B, int64_t N, int Tn,
                                    const T* s1, T* ra) {
  const int64_t n_el = N * B * Tn;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_el;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % Tn);
    const int64_t r = idx / Tn;
    const int d = (int)(r % B);
    const int64_t n = r / B;
    const T v = rz[idx] + V[(int64_t)d * ldv + boff + t];
    rz[idx] = v;
    if (ra) ra[idx] = s1[n * Tn + t] * v;
  }
}

// H v_d for B general directions at once (Sec. 5.1; the R-operator of
// Pearlmutter applied to the forward pass and the per-example
// back-propagation, Appendix A):
//   R{z^(j)}  = W^(j) R{a^(j-1)} + V^(j) a^(j-1) + v_b^(j)     (R{a^(0)} = 0)
//   R{a^(j)}  = sigma'(z^(j)) R{z^(j)}
//   R{delta^(L)}   = (diag p - p p^T) R{z^(L)} sum(y)
//   R{delta^(j)}   = sigma''(z^(j)) R{z^(j)} e^(j)
//                    + sigma'(z^(j)) (R{delta^(j+1)} W^(j+1) + delta^(j+1) V^(j+1))
//   (H v)_W^(j) = (1/N) sum_n R{delta^(j)} a^(j-1)^T + delta^(j) R{a^(j-1)}^T
//   (H v)_b^(j) = (1/N) sum_n R{delta^(j)}
// with V^(j), v_b^(j) the direction's slices in the parameter order.  The
// weight GEMMs shared by all directions run once over N B rows; the
// direction-dependent ones are batched over d.
template <typename T>
hess_status hvp_block(const Net& net, const T* omega, const Caches<T>& c, const T* V, int64_t ldv, int B,
                      RopBufs<T>& r, T* HV, int64_t ldh, cudaStream_t s) {
  const int L = net.L;
  const int64_t N = c.N;
  const T invN = T(1) / T(N);
  if (!r.ones_ready) {
    HM_TRY(fill(r.ones, N, T(1), s));
    r.ones_ready = true;
  }
  // forward
  for (int j = 1; j <= L - 1; ++j) {
    const int Tin = net.T[j - 1], Tout = net.T[j];
    if (j > 1) {
      Gemm<T> g;  // R{a}^(j-1) W^(j)^T, W^(j) is Tout x Tin
      g.M = (int)(N * B);
      g.N = Tout;
      g.K = Tin;
      g.A = r.ra[j - 1];
      g.sam = Tin;
      g.sak = 1;
      g.B = omega + net.woff[j - 1];
      g.sbk = 1;
      g.sbn = Tin;
      g.C = r.rz[j];
      g.scm = Tout;
      g.scn = 1;
      HM_TRY(gemm(g, s));
    }
    {
      Gemm<T> g;  // + a^(j-1) V_d^(j)^T, batched over d
      g.M = (int)N;
      g.N = Tout;
      g.K = Tin;
      g.beta = j > 1 ? T(1) : T(0);
      g.A = c.a[j - 1];
      g.sam = Tin;
      g.sak = 1;
      g.bsa = 0;
      g.B = V + net.woff[j - 1];
      g.sbk = 1;
      g.sbn = Tin;
      g.bsb = ldv;
      g.C = r.rz[j];
      g.scm = (int64_t)B * Tout;
      g.scn = 1;
      g.bsc = Tout;
      g.batch = B;
      HM_TRY(gemm(g, s));
    }
    const bool hidden = j <= L - 2;
    hvp_bias_act_kernel<T><<<grid1d(N * B * Tout), 256, 0, s>>>(r.rz[j], V, ldv, net.boff[j - 1], B, N, Tout,
                                                              hidden ? c.s1[j] : nullptr,
                                                              hidden ? r.ra[j] : nullptr);
    HM_LAUNCHED();
  }
  {
    const int TL = net.T[L - 1];
    rop_softmax_kernel<T><<<(unsigned)cdiv(N * B, 128), 128, 0, s>>>(r.rz[L - 1], c.p, c.ysum, r.rd[L - 1], B,
                                                                      N, TL);
    HM_LAUNCHED();
  }
  // backward
  for (int j = L - 2; j >= 1; --j) {
    const int Tj = net.T[j], Tn = net.T[j + 1];
    {
      Gemm<T> g;  // R{delta}^(j+1) W^(j+1)
      g.M = (int)(N * B);
      g.N = Tj;
      g.K = Tn;
      g.A = r.rd[j + 1];
      g.sam = Tn;
      g.sak = 1;
      g.B = omega + net.woff[j];
      g.sbk = Tj;
      g.sbn = 1;
      g.C = r.tmp;
      g.scm = Tj;
      g.scn = 1;
      HM_TRY(gemm(g, s));
    }
    {
      Gemm<T> g;  // + delta^(j+1) V_d^(j+1), batched over d
      g.M = (int)N;
      g.N = Tj;
      g.K = Tn;
      g.beta = T(1);
      g.A = c.d[j + 1];
      g.sam = Tn;
      g.sak = 1;
      g.bsa = 0;
      g.B = V + net.woff[j];
      g.sbk = Tj;
      g.sbn = 1;
      g.bsb = ldv;
      g.C = r.tmp;
      g.scm = (int64_t)B * Tj;
      g.scn = 1;
      g.bsc = Tj;
      g.batch = B;
      HM_TRY(gemm(g, s));
    }
    rop_back_kernel<T><<<grid1d(N * B * Tj), 256, 0, s>>>(r.rz[j], r.tmp, c.s1[j], c.s2[j], c.e[j], r.rd[j], B, N,
                                                         Tj);
    HM_LAUNCHED();
  }
  // contraction with the forward quantities
  for (int j = 1; j <= L - 1; ++j) {
    const int Tin = net.T[j - 1], Tout = net.T[j];
    {
      Gemm<T> g;  // (1/N) R{delta}_d^(j)^T a^(j-1), batched over d
      g.M = Tout;
      g.N = Tin;
      g.K = (int)N;
      g.alpha = invN;
      g.A = r.rd[j];
      g.sam = 1;
      g.sak = (int64_t)B * Tout;
      g.bsa = Tout;
      g.B = c.a[j - 1];
      g.sbk = Tin;
      g.sbn = 1;
      g.bsb = 0;
      g.C = HV + net.woff[j - 1];
      g.scm = Tin;
      g.scn = 1;
      g.bsc = ldh;
      g.batch = B;
      HM_TRY(gemm(g, s));
    }
    if (j > 1) {
      Gemm<T> g;  // + (1/N) delta^(j)^T R{a}_d^(j-1), batched over d
      g.M = Tout;
      g.N = Tin;
      g.K = (int)N;
      g.alpha = invN;
      g.beta = T(1);
      g.A = c.d[j];
      g.sam = 1;
      g.sak = Tout;
      g.bsa = 0;
      g.B = r.ra[j - 1];
      g.sbk = (int64_t)B * Tin;
      g.sbn = 1;
      g.bsb = Tin;
      g.C = HV + net.woff[j - 1];
      g.scm = Tin;
      g.scn = 1;
      g.bsc = ldh;
      g.batch = B;
      HM_TRY(gemm(g, s));
    }
    {
      Gemm<T> g;  // (1/N) sum_n R{delta}_d^(j), batched over d: a product with ones
      g.M = Tout;
      g.N = 1;
      g.K = (int)N;
      g.alpha = invN;
      g.A = r.rd[j];
      g.sam = 1;
      g.sak = (int64_t)B * Tout;
      g.bsa = Tout;
      g.B = r.ones;
      g.sbk = 1;
      g.sbn = 0;
      g.bsb = 0;
      g.C = HV + net.boff[j - 1];
      g.scm = 1;
      g.scn = 0;
      g.bsc = ldh;
      g.batch = B;
      HM_TRY(gemm(g, s));
    }
  }
  return HESS_OK;
}
template hess_status hvp_block<double>(const Net&, const double*, const Caches<double>&, const double*, int64_t,
                                       int, RopBufs<double>&, double*, int64_t, cudaStream_t);
template hess_status hvp_block<float>(const Net&, const float*, const Caches<float>&, const float*, int64_t, int,
                                      RopBufs<float>&, float*, int64_t, cudaStream_t);

}  // namespace hm
