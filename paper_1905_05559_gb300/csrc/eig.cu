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
#include <cooperative_groups.h>

#include <atomic>
#include <cfloat>
#include <climits>
#include <mutex>

#include "devmath.cuh"
#include "internal.h"

namespace hm {

namespace {

// ------------------------------------------------------------ Gram matrix
// M = G G^T / N in factored form (Eq. J, with g_n = [delta_n (x) a_n; delta_n]
// for each weight layer):
//   M[n][m] = (1/N) sum_l (delta_{l,n} . delta_{l,m}) (a_{l,n} . a_{l,m} + 1).
// The dot products are formed in double-float arithmetic (devmath.cuh; FP64
// issues at 1/64 of the FP32 rate on this part) from rows scaled by powers of
// two, a wide layer's a . a from the exact-digit planes of its tensor-core
// product.  With e_D, e_A the exponents of a row's largest delta and
// activation, u_l = e_D + max(e_A, 0) and r_n = max_l u_{l,n}, every layer's
// term of entry (n, m) is 2^(r_n + r_m) times a double-float number of modest
// size: the scaled dots times 2^(p_{A,n} + p_{A,m}) and 2^(p_{D,n} + p_{D,m}),
// p_A = e_D + e_A - r <= 0, p_D = e_D - r <= 0.  (Below 2^-126 a factor counts
// as zero: such a term is under 2^-126 of the larger diagonal entries.)

// The exponent E of max |x| = f 2^E, f in [0.5, 1); 0 for a zero or non-finite
// maximum (the digit split's rule, so that both agree on a wide layer).
__device__ __forceinline__ int row_exp(double mx) {
  int E = 0;
  if (mx > 0.0 && mx <= DBL_MAX) frexp(mx, &E);
  return E;
}
// x 2^e for |e| <= 2100 (two exact power-of-two factors, each in range)
__device__ __forceinline__ double scale2(double x, int e) {
  const int e1 = e / 2, e2 = e - e1;
  return x * __longlong_as_double((long long)(1023 + e1) << 52) * __longlong_as_double((long long)(1023 + e2) << 52);
}
// 2^x as FP32 for x <= 127; 0 below 2^-126
__device__ __forceinline__ float pow2f(int x) { return x < -126 ? 0.0f : __int_as_float((x + 127) << 23); }

struct GramPrepLayer {
  const double* D;  // delta rows, N x Tout
  const double* A;  // activation rows, N x Tin
  int Tout, Tin;
  float2* XD;       // delta rows times 2^-e_D, double-float, N x Tout
  float2* XA;       // activation rows times 2^-e_A, N x Tin (nullptr: a wide layer, not split)
  int *pD, *pA, *eA;  // per row: e_D - r, e_D + e_A - r, e_A
};
struct GramPrepArgs {
  GramPrepLayer l[kMaxLayers];
  int nl;
  int64_t N;
  double invN;
  int* r;
  unsigned long long* maxdiag;  // FP64 bits of max_n M[n][n] (zeroed beforehand)
  float2* q0;                   // when set, the last block writes the Lanczos start vector there
  uint64_t key;
};

// One warp per example row n: exponents, r_n, the FP64 diagonal entry (for the
// scale of the double-float output), and the split rows.
__global__ void gram_prep_kernel(const __grid_constant__ GramPrepArgs g) {
  if (g.q0 && blockIdx.x == gridDim.x - 1) {
    // the Lanczos start vector q_0: a counter-based random unit vector
    // (hi/lo pairs), formed here off the eigen step's critical path
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t n = threadIdx.x; n < g.N; n += blockDim.x) {
      const double v = rnd_sym(g.key, n);
      s = fma(v, v, s);
    }
    s = block_sum(s, sh);
    const double inv = 1.0 / sqrt(s);
    for (int64_t n = threadIdx.x; n < g.N; n += blockDim.x) g.q0[n] = df_split(rnd_sym(g.key, n) * inv);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t n = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (n >= g.N) return;
  int r = INT_MIN;
  double diag = 0.0;
  for (int l = 0; l < g.nl; ++l) {
    const GramPrepLayer& L = g.l[l];
    const double* d = L.D + n * L.Tout;
    const double* a = L.A + n * L.Tin;
    double md = 0.0, ma = 0.0, sd = 0.0, sa = 0.0;
    for (int k = lane; k < L.Tout; k += 32) {
      const double v = d[k];
      md = fmax(md, fabs(v));
      sd = fma(v, v, sd);
    }
#pragma unroll 8
    for (int k = lane; k < L.Tin; k += 32) {
      const double v = a[k];
      ma = fmax(ma, fabs(v));
      sa = fma(v, v, sa);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
      ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    }
    sd = warp_sum(sd);
    sa = warp_sum(sa);
    const int eD = row_exp(md), eA = row_exp(ma);
    const int u = eD + (eA > 0 ? eA : 0);
    r = u > r ? u : r;
    diag = fma(sd, sa + 1.0, diag);
    if (lane == 0) {
      L.pD[n] = eD;  // (relative to r below)
      L.eA[n] = eA;
    }
  }
  if (lane == 0) {
    g.r[n] = r;
    const double v = diag * g.invN;
    if (v > 0.0) atomicMax(g.maxdiag, (unsigned long long)__double_as_longlong(v));
  }
  __syncwarp();
  for (int l = 0; l < g.nl; ++l) {
    const GramPrepLayer& L = g.l[l];
    const int eD = L.pD[n], eA = L.eA[n];
    __syncwarp();
    if (lane == 0) {
      L.pD[n] = eD - r;
      L.pA[n] = eD + eA - r;
    }
    const double* d = L.D + n * L.Tout;
    for (int k = lane; k < L.Tout; k += 32) L.XD[n * L.Tout + k] = df_split(scale2(d[k], -eD));
    if (L.XA) {
      const double* a = L.A + n * L.Tin;
      for (int k = lane; k < L.Tin; k += 32) L.XA[n * L.Tin + k] = df_split(scale2(a[k], -eA));
    }
  }
}

struct GramLayer {
  const float2* D;  // split delta rows (N x Tout)
  const float2* A;  // split activation rows (N x Tin); nullptr: the planes
  const int *pD, *pA, *eA;
  int Tout, Tin;
};
struct GramArgs {
  GramLayer l[kMaxLayers];
  int nl;
  F64SyrkPlanes pl;  // the wide layer's a . a (pl.T set)
  const int* r;
  const unsigned long long* maxdiag;
  int64_t N;
  double invN;
  int accumulate;
  int df_out;   // 1: write 2^-E M as double-float pairs, E = the exponent of max M[n][n]; 0: FP64 M
  int* escale;  // receives E (df_out)
};
constexpr int kGt = 32;

// (s[i], c[i]) = X_{n0 + ty + 8 i} . X_{m0 + tx} over the K columns of the
// split rows X (rows past N count as zero); sr and sc stage 32-column chunks,
// sc transposed so that the lanes read consecutive words.
__device__ __forceinline__ void gram_tile_dot(const float2* X, int K, int64_t N, int64_t n0, int64_t m0,
                                              float2 (*sr)[kGt + 1], float2 (*sc)[kGt + 1], float s[4], float c[4]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) s[i] = c[i] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += kGt) {
    for (int e = threadIdx.x; e < kGt * kGt; e += blockDim.x) {
      const int rr = e >> 5, kk = e & 31;
      const int64_t kg = k0 + kk;
      sr[rr][kk] = (n0 + rr < N && kg < K) ? X[(n0 + rr) * K + kg] : make_float2(0.0f, 0.0f);
      sc[kk][rr] = (m0 + rr < N && kg < K) ? X[(m0 + rr) * K + kg] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const int kc = K - k0 < kGt ? K - k0 : kGt;
    for (int kk = 0; kk < kc; ++kk) {
      const float2 b = sc[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) df_mac(sr[ty + 8 * i][kk], b, s[i], c[i]);
    }
    __syncthreads();
  }
}

// One block per kGt x kGt tile on or above the diagonal, written at (n, m)
// and, through shared memory, at (m, n); a diagonal tile writes its upper
// half and mirrors it, so M is exactly symmetric.
__global__ void __launch_bounds__(256, 3) gram_fused_kernel(const __grid_constant__ GramArgs g, void* Mout) {
  __shared__ float2 sr[kGt][kGt + 1];
  __shared__ float2 sc[kGt][kGt + 1];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  const int64_t N = g.N, n0 = bi * kGt, m0 = bj * kGt;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t m = m0 + tx;
  const bool diag_tile = bi == bj;
  float2 acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.0f, 0.0f);
  for (int l = 0; l < g.nl; ++l) {
    const GramLayer& L = g.l[l];
    float ds[4], dc[4], as[4], ac[4];
    gram_tile_dot(L.D, L.Tout, N, n0, m0, sr, sc, ds, dc);
    if (L.A) {
      gram_tile_dot(L.A, L.Tin, N, n0, m0, sr, sc, as, ac);
    } else {
      // the planes hold the entries (n, m >= n) of the scaled product
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const int64_t n = n0 + ty + 8 * i;
        float S = 0.0f, C = 0.0f;
        if (n < N && m < N && (!diag_tile || n <= m)) {
          const size_t at = (size_t)n * N + m, plane = (size_t)N * N;
          // the planes of one weight 2^(-12 - 7 w) are summed exactly as
          // integers (each below 2^24), then added as a double-float pair;
          // loads in batches of 12
          constexpr int kB = 12;
          int a = 0;
#pragma unroll
          for (int j0 = 0; j0 < kMaxSyrkPlanes; j0 += kB) {
            if (j0 >= g.pl.count) break;
            float v[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j) v[j] = j0 + j < g.pl.count ? g.pl.T[(j0 + j) * plane + at] : 0.0f;
#pragma unroll
            for (int j = 0; j < kB; ++j) {
              const int jj = j0 + j;
              if (jj >= g.pl.count) break;
              a += __float2int_rn(v[j]);
              const int wn = jj + 1 < kMaxSyrkPlanes ? g.pl.wexp[jj + 1] : -1;
              if (jj + 1 == g.pl.count || wn != g.pl.wexp[jj]) {
                const float hi = __int2float_rn(a);
                const float lo = __int2float_rn(a - __float2int_rz(hi));
                const float pw = pow2f(-12 - 7 * g.pl.wexp[jj]);
                float t, e;
                two_sum(S, hi * pw, t, e);
                S = t;
                C += e + lo * pw;
                a = 0;
              }
            }
          }
          if (g.pl.part) {
            // earlier groups of planes, combined in FP64
            const float2 p = df_split(scale2(g.pl.part[n * g.pl.ldp + m], -(L.eA[n] + L.eA[m])));
            float t, e;
            two_sum(S, p.x, t, e);
            S = t;
            C += e + p.y;
          }
        }
        as[i] = S;
        ac[i] = C;
      }
    }
    const int pDm = L.pD[m < N ? m : 0], pAm = L.pA[m < N ? m : 0];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t n = n0 + ty + 8 * i;
      const int pDn = L.pD[n < N ? n : 0], pAn = L.pA[n < N ? n : 0];
      const float pa = pow2f(pAn + pAm), pd = pow2f(pDn + pDm);
      const float2 aa = df_norm(as[i], ac[i]);
      const float2 t = df_add(make_float2(aa.x * pa, aa.y * pa), make_float2(pd, 0.0f));
      acc[i] = df_add(acc[i], df_mul(df_norm(ds[i], dc[i]), t));
    }
  }
  // the tile in shared memory (8-byte entries: a double-float pair or an FP64
  // value), then the direct and the mirrored stores
  unsigned long long(*so)[kGt + 1] = reinterpret_cast<unsigned long long(*)[kGt + 1]>(sr);
  const float2 invN = df_split(g.invN);
  int E = 0;
  if (g.df_out) {
    E = row_exp(__longlong_as_double((long long)*g.maxdiag));
    if (bi == 0 && bj == 0 && threadIdx.x == 0) *g.escale = E;
  }
  const int rm = g.r[m < N ? m : 0];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = ty + 8 * i;
    const int64_t n = n0 + rr;
    const int rn = g.r[n < N ? n : 0];
    const float2 v = df_mul(acc[i], invN);
    unsigned long long bits;
    if (g.df_out) {
      // |2^-E M[n][m]| < 1: a large exponent comes with a tiny v
      int x = rn + rm - E;
      x = x < -250 ? -250 : (x > 250 ? 250 : x);
      const float p1 = pow2f(x / 2), p2 = pow2f(x - x / 2);
      const float2 o = make_float2(v.x * p1 * p2, v.y * p1 * p2);
      bits = (unsigned long long)__double_as_longlong(*reinterpret_cast<const double*>(&o));
    } else {
      bits = (unsigned long long)__double_as_longlong(scale2(df_val(v), rn + rm));
    }
    so[rr][tx] = bits;
  }
  __syncthreads();
  auto store = [&](int64_t row, int64_t col, unsigned long long bits) {
    if (g.df_out) {
      float2* o = reinterpret_cast<float2*>(Mout) + row * N + col;
      const float2 v = *reinterpret_cast<const float2*>(&bits);
      *o = g.accumulate ? df_add(*o, v) : v;
    } else {
      double* o = reinterpret_cast<double*>(Mout) + row * N + col;
      const double v = __longlong_as_double((long long)bits);
      *o = g.accumulate ? *o + v : v;
    }
  };
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = ty + 8 * i;
    const int64_t n = n0 + rr;
    if (n < N && m < N && (!diag_tile || rr <= tx)) store(n, m, so[rr][tx]);
    // mirrored: row m0 + rr, column n0 + tx holds entry (n0 + tx, m0 + rr)
    const int64_t mm = m0 + rr, nn = n0 + tx;
    if (mm < N && nn < N && (!diag_tile || tx < rr)) store(mm, nn, so[tx][rr]);
  }
}

// ------------------------------------------------ cooperative Lanczos
// All Lanczos steps of one extension run in a single cooperative launch (all
// blocks co-resident).  Block b owns the entries [b E, (b + 1) E) of every
// vector: it computes them, and keeps its rows of M and its slice of the
// Lanczos vectors in shared memory when they fit.  A step is four phases
// separated by grid barriers:
//   A  beta_{j-1} = ||w||, q_j = w / beta (owned slice), M q_j on the owned
//      rows (stored in MQ_j), first-pass coefficients h_i = (M q_i) . q_j for
//      i < j (one warp each, over full rows) and block partials of
//      h_j = q_j . (M q_j)
//   B  w' = M q_j - sum_{i<=j} h_i q_i (owned slice)
//   C  second-pass dot products d_i = q_i . w' (i <= j), as chunk partials
//   D  alpha_j = h_j + d_j, w = w' - sum_{i<=j} d_i q_i (owned slice), block
//      partials of ||w||^2
// (classical Gram-Schmidt applied twice against every earlier vector).  At a
// breakdown (||w|| ~ 0) the kernel stops; restart_* below draw a random vector
// orthogonal to the basis and the next launch resumes.  Barrier waits are
// bounded: on timeout the kernel raises *err and returns.
struct LzArgs {
  const double* M;
  int64_t N;
  double* Q;     // Lanczos vectors, rows of length N (mcap rows)
  double* MQ;    // M q_i, rows of length N
  double* w;     // current residual vector
  double* wt;    // w' of the step
  double* h;     // first-pass coefficients (mcap)
  double* dpart; // [mcap][nchunk] partial dot products
  double* npart; // [gridDim] partial squared norms of w
  double* apart; // [gridDim] partial sums of q_j . (M q_j)
  double* alpha;
  double* beta;
  unsigned* bar;  // arrival counter (zero at launch)
  int* err;
  int m0, m1, mcap, nchunk;
  int E;          // entries owned per block
  int cache_m;    // the block's rows of M in shared memory
  int cache_q;    // the block's slice of Q in shared memory
  int cache_w;    // a copy of w in shared memory for the owned rows of M w
  int* stop;      // set to j when step j meets a breakdown (the kernel returns)
  int resumed;    // m0 follows a restart: beta_{m0-1} = 0 is already set
  uint64_t key;
  long long bar_limit;  // clock cycles a grid-barrier wait may take
};

constexpr long long BAR_TIMEOUT = 4000000000ll;
// test hook: a shorter grid-barrier limit (0 = BAR_TIMEOUT)
std::atomic<long long> g_bar_limit{0};

__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: thread 0 of every block adds to one counter, block 0 adding
// 2^31 - (gridDim.x - 1) and the others 1, so that the counter's top bit
// flips exactly when the last block arrives; each block waits (bounded) for
// the flip from the value it saw on arrival.  The add is a release at GPU
// scope (after the block barrier, it publishes every thread's writes) and the
// polling load an acquire (the block barrier after it passes the other
// blocks' writes on to every thread).
__device__ bool grid_barrier_at(unsigned* bar, int* err, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    const unsigned old = atom_add_release_gpu(bar, add);
    const long long t0 = clock64();
    while (((old ^ ld_acquire_gpu(bar)) & 0x80000000u) == 0u) {
      if (clock64() - t0 > limit || *(volatile int*)err) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}
__device__ bool grid_barrier(const LzArgs& a, unsigned& epoch) {
  ++epoch;
  return grid_barrier_at(a.bar, a.err, a.bar_limit);
}

// sum_c x[c] y[c] over one warp for c in [n0, n1); x in global memory, y in
// shared or global memory; sixteen loads per lane in flight
__device__ __forceinline__ double warp_dot(const double* x, const double* y, int64_t n0, int64_t n1) {
  const int lane = threadIdx.x & 31;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t c = n0 + lane;
  for (; c + 15 * 32 < n1; c += 16 * 32) {
    double xv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) xv[u] = x[c + u * 32];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u & 7] = fma(xv[u], y[c + u * 32], acc[u & 7]);
  }
  for (; c + 3 * 32 < n1; c += 4 * 32) {
    double xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = x[c + u * 32];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(xv[u], y[c + u * 32], acc[u]);
  }
  for (; c < n1; c += 32) acc[4] = fma(x[c], y[c], acc[4]);
  const double s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  return warp_sum(s);
}

// For the block's owned entries e < ne (global n0 + e):
//   out[e] = base[e] - sum_{i < nv} coef[i] Q[i][e]
// in 32-entry chunks: lanes along the entries, the block's warps split the i
// range, partial sums meet in shared memory.  Q[i][e] comes from the block's
// shared slice (stride E) or from global rows.  Writes out to shared memory
// and to out_g[n0 + e]; returns (in warp 0) the sum of out[e]^2.
__device__ double combine_slice(const LzArgs& a, const double* Qsh, const double* coef, int nv,
                                const double* base, double* out, double* out_g, int64_t n0, int ne,
                                double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double nn = 0.0;
  if (a.cache_q && ne <= nwarp) {
    // few owned entries: one warp per entry, lanes along i (an FP64 warp
    // instruction costs the same with 7 lanes active as with 32)
    if (warp < ne) {
      const int e = warp;
      double s0 = 0.0, s1 = 0.0;
      int i = lane;
      for (; i + 32 < nv; i += 64) {
        s0 = fma(Qsh[(int64_t)i * a.E + e], coef[i], s0);
        s1 = fma(Qsh[(int64_t)(i + 32) * a.E + e], coef[i + 32], s1);
      }
      if (i < nv) s0 = fma(Qsh[(int64_t)i * a.E + e], coef[i], s0);
      const double t = warp_sum(s0 + s1);
      if (lane == 0) {
        const double v = base[e] - t;
        out[e] = v;
        out_g[n0 + e] = v;
        red[e] = v * v;
      }
    }
    __syncthreads();
    if (warp == 0) {
      for (int e = lane; e < ne; e += 32) nn += red[e];
    }
    __syncthreads();
    return nn;  // warp 0 lanes hold partial sums of squares
  }
  for (int c0 = 0; c0 < ne; c0 += 32) {
    const int e = c0 + lane;
    double s0 = 0.0, s1 = 0.0;
    if (e < ne) {
      if (a.cache_q) {
        for (int i = warp; i < nv; i += nwarp) s0 = fma(Qsh[(int64_t)i * a.E + e], coef[i], s0);
      } else {
        const double* q = a.Q + n0 + e;
        int i = warp;
        for (; i + nwarp < nv; i += 2 * nwarp) {
          s0 = fma(q[(int64_t)i * a.N], coef[i], s0);
          s1 = fma(q[(int64_t)(i + nwarp) * a.N], coef[i + nwarp], s1);
        }
        if (i < nv) s0 = fma(q[(int64_t)i * a.N], coef[i], s0);
      }
    }
    red[warp * 32 + lane] = s0 + s1;
    // pairwise tree over the warps' partial sums (nwarp is a power of two)
    for (int half = nwarp >> 1; half > 0; half >>= 1) {
      __syncthreads();
      if (warp < half) red[warp * 32 + lane] += red[(warp + half) * 32 + lane];
    }
    __syncthreads();
    if (warp == 0 && e < ne) {
      const double t = red[lane];
      const double v = base[e] - t;
      out[e] = v;
      out_g[n0 + e] = v;
      nn = fma(v, v, nn);
    }
    __syncthreads();
  }
  return nn;
}

// sum_b part[b] by warp 0 of the block (same order in every block); every
// lane issues its loads before adding
__device__ double sum_partials(const double* part, int n, double* out_sh) {
  if (threadIdx.x < 32) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = threadIdx.x + 32 * u;
      v[u] = b < n ? part[b] : 0.0;
    }
    double s = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    for (int b = threadIdx.x + 256; b < n; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x == 0) *out_sh = s;
  }
  __syncthreads();
  return *out_sh;
}

__global__ void __launch_bounds__(512, 1) lanczos_coop_kernel(LzArgs a) {
  extern __shared__ double dyn[];
  const int64_t N = a.N;
  const int E = a.E;
  double* d_sh = dyn;                  // coefficients, mcap + 1
  double* wsh_s = d_sh + (a.mcap + 1);                // full w, N (cache_w)
  double* ysh = wsh_s + (a.cache_w ? N : 0);          // owned slice of M q_j, E
  double* wps = ysh + E;               // owned slice of w', E
  double* wsl = wps + E;               // owned slice of w, E
  double* Msh = wsl + E;               // owned rows of M, E x N (cache_m)
  double* Qsh = Msh + (a.cache_m ? (int64_t)E * N : 0);  // owned slice of Q, mcap x E (cache_q)
  const int64_t n0 = (int64_t)blockIdx.x * E;
  const int ne = (int)(N - n0 < E ? (N - n0 > 0 ? N - n0 : 0) : E);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // warp-level tasks over the whole grid, dealt block-major and starting from
  // each block's last warp (the first warps carry the owned rows)
  const int wI = (nwarp - 1 - warp) * gridDim.x + blockIdx.x;
  const int nW = nwarp * gridDim.x;
  const int64_t chunk = (N + a.nchunk - 1) / a.nchunk;
  __shared__ double s_tmp, s_scale, s_rs, s_b;
  __shared__ int s_brk;
  __shared__ double red_sh[16 * 32];
  unsigned epoch = 0;  // meaningful in thread 0 only
  if (a.cache_m)
    for (int e = 0; e < ne; ++e)
      for (int64_t n = threadIdx.x; n < N; n += blockDim.x) Msh[(int64_t)e * N + n] = a.M[(n0 + e) * N + n];
  if (a.cache_q)
    for (int i = warp; i < a.m0; i += nwarp)
      for (int e = lane; e < ne; e += 32) Qsh[(int64_t)i * E + e] = a.Q[(int64_t)i * N + n0 + e];
  for (int e = threadIdx.x; e < ne; e += blockDim.x) wsl[e] = a.w[n0 + e];
  // running scale of T (max |alpha_i|, beta_i so far), kept per block
  if (threadIdx.x == 0) {
    double sc = 0.0;
    for (int i = 0; i < a.m0; ++i)
      sc = fmax(sc, fmax(fabs(a.alpha[i]), i + 1 < a.m0 ? a.beta[i] : 0.0));
    s_scale = sc;
  }
  __syncthreads();
  for (int j = a.m0; j < a.m1; ++j) {
    // ---- A
    // full w for the owned rows of M w (warps 1..) while warp 0 sums the
    // norm partials
    if (a.cache_w && warp > 0)
      for (int64_t n = threadIdx.x - 32; n < N; n += blockDim.x - 32) wsh_s[n] = a.w[n];
    // An FP64 instruction occupies its SM partition for many cycles per
    // warp, so block-wide scalars are computed once, by thread 0, and read
    // from shared memory by the others.
    double nsum = sum_partials(a.npart, gridDim.x, &s_tmp);
    if (threadIdx.x == 0) {
      const double r = nsum > 0.0 ? rsqrt64(nsum) : 0.0;  // 1 / ||w||
      s_rs = r;
      s_b = nsum * r;
      s_brk = j > 0 && !(a.resumed && j == a.m0) && (!(nsum * r > 1e-12 * s_scale) || s_scale == 0.0);
    }
    __syncthreads();
    // breakdown (||w|| ~ 0): stop here; the host draws a new direction
    // orthogonal to q_0..q_{j-1} and resumes at step j.  (Kept out of the
    // loop: code on this path slows every step.)
    if (s_brk) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *a.stop = j;
      return;
    }
    const double rs = s_rs;
    const double bprev = s_b;
    if (j > 0 && !(a.resumed && j == a.m0) && blockIdx.x == 0 && threadIdx.x == 0) a.beta[j - 1] = bprev;
    __syncthreads();  // every thread has read s_rs, s_b
    if (threadIdx.x == 0 && j > 0 && !(a.resumed && j == a.m0)) s_scale = fmax(s_scale, bprev);
    const double inv = rs;  // 0 when ||w|| = 0
    // owned slice of q_j
    const double* wsh = a.cache_w ? wsh_s : a.w;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const double q = wsl[e] * inv;
      a.Q[(int64_t)j * N + n0 + e] = q;
      if (a.cache_q) Qsh[(int64_t)j * E + e] = q;
    }
    __syncthreads();
    double* mqj = a.MQ + (int64_t)j * N;
    for (int e = warp; e < ne; e += nwarp) {
      const double* row = a.cache_m ? Msh + (int64_t)e * N : a.M + (n0 + e) * N;
      double acc = 0.0;
      if (a.cache_m) {
        double c4[4] = {0.0, 0.0, 0.0, 0.0};
        int64_t n = lane;
        for (; n + 96 < N; n += 128) {
#pragma unroll
          for (int u = 0; u < 4; ++u) c4[u] = fma(row[n + 32 * u], wsh[n + 32 * u], c4[u]);
        }
        for (; n < N; n += 32) c4[0] = fma(row[n], wsh[n], c4[0]);
        acc = warp_sum((c4[0] + c4[1]) + (c4[2] + c4[3]));
      } else {
        acc = warp_dot(row, wsh, 0, N);
      }
      if (lane == 0) {
        ysh[e] = acc * inv;
        mqj[n0 + e] = acc * inv;
      }
    }
    for (int i = wI; i < j; i += nW) {
      const double sr = warp_dot(a.MQ + (int64_t)i * N, wsh, 0, N) * inv;
      if (lane == 0) a.h[i] = sr;
    }
    __syncthreads();
    if (warp == 0) {
      double v = 0.0;
      for (int e = lane; e < ne; e += 32) v = fma(wsl[e] * inv, ysh[e], v);
      v = warp_sum(v);
      if (lane == 0) a.apart[blockIdx.x] = v;
    }
    if (!grid_barrier(a, epoch)) return;
    // ---- B: w' = M q_j - sum_{i<=j} h_i q_i on the owned slice (warps 1..
    // fetch h_i while warp 0 sums the partials of h_j)
    if (warp > 0)
      for (int i = threadIdx.x - 32; i < j; i += blockDim.x - 32) d_sh[i] = a.h[i];
    const double hj = sum_partials(a.apart, gridDim.x, &s_tmp);
    if (threadIdx.x == 0) d_sh[j] = hj;
    __syncthreads();
    combine_slice(a, Qsh, d_sh, j + 1, ysh, wps, a.wt, n0, ne, red_sh);
    if (!grid_barrier(a, epoch)) return;
    // ---- C: partial dot products q_i . w' over chunks, one warp per (i, chunk)
    for (int task = wI; task < (j + 1) * a.nchunk; task += nW) {
      const int i = task / a.nchunk, ch = task % a.nchunk;
      const int64_t c0 = ch * chunk, c1 = min(N, c0 + chunk);
      const double sr = warp_dot(a.Q + (int64_t)i * N, a.wt, c0, c1);
      if (lane == 0) a.dpart[(int64_t)i * a.nchunk + ch] = sr;
    }
    if (!grid_barrier(a, epoch)) return;
    // ---- D: w = w' - sum_{i<=j} d_i q_i, alpha_j = h_j + d_j
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      double v[8];  // nchunk <= 8
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) v[ch] = ch < a.nchunk ? a.dpart[(int64_t)i * a.nchunk + ch] : 0.0;
      d_sh[i] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    __syncthreads();
    double sn = combine_slice(a, Qsh, d_sh, j + 1, wps, wsl, a.w, n0, ne, red_sh);
    if (warp == 0) {
      sn = warp_sum(sn);  // the slice's sum of squares lives in warp 0
      if (lane == 0) {
        a.npart[blockIdx.x] = sn;
        const double al = hj + d_sh[j];
        if (blockIdx.x == 0) a.alpha[j] = al;
        s_scale = fmax(s_scale, fabs(al));
      }
    }
    if (!grid_barrier(a, epoch)) return;
  }
}

// Start vector: w = random unit vector, npart = (1, 0, 0, ...) so that the
// first step reads ||w|| = 1.
__global__ void init_start_kernel(double* w, double* npart, int nparts, int64_t N, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    double v = rnd_sym(key, n);
    w[n] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  double inv = 1.0 / sqrt(s);
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) w[n] *= inv;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) npart[b] = b == 0 ? 1.0 : 0.0;
}

// Restart after a breakdown at step j: w = a random vector (the same
// counter-based draw on every run), beta_{j-1} = 0.
__global__ void restart_fill_kernel(double* w, int64_t N, uint64_t key, int j, double* beta) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    w[n] = rnd_sym(key, (uint64_t)j * 0x100000000ull + (uint64_t)n);
  if (blockIdx.x == 0 && threadIdx.x == 0) beta[j - 1] = 0.0;
}

// c_i = q_i . w for i < j, one warp per i
__global__ void restart_coef_kernel(const double* Q, const double* w, int64_t N, int j, double* c) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= j) return;
  double s = 0.0;
  for (int64_t n = lane; n < N; n += 32) s = fma(Q[(int64_t)i * N + n], w[n], s);
  s = warp_sum(s);
  if (lane == 0) c[i] = s;
}

// w -= sum_{i<j} c_i q_i
__global__ void restart_sub_kernel(const double* Q, const double* c, int64_t N, int j, double* w) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < j; ++i) s = fma(Q[(int64_t)i * N + n], c[i], s);
    w[n] -= s;
  }
}

// npart = (||w||^2, 0, 0, ...) for the resumed launch
__global__ void restart_norm_kernel(const double* w, int64_t N, double* npart, int nparts) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s = fma(w[n], w[n], s);
  s = block_sum(s, sh);
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) npart[b] = b == 0 ? s : 0.0;
}

// beta of the last completed step (the coupling of T_m to the next vector)
__global__ void last_beta_kernel(const double* npart, int nparts, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += npart[b];
    *out = sqrt(s);
  }
}

// ------------------------------------------ double-float Lanczos kernel ----
// The same Lanczos process with full reorthogonalisation, for Gram matrices
// whose rows fit the blocks' shared memory, in double-float arithmetic
// (devmath.cuh: about 48 significant bits, all on the FP32 pipe), with one
// grid-wide reduction and two grid barriers per step j.  The second
// Gram-Schmidt pass of each vector is taken one step late, in the next
// step's reduction (classical Gram-Schmidt twice, the second pass lagged):
// the vector handed from step j-1 to step j is w = q~_j, orthogonalised once
// and not normalised.
//   1  gather q~_j; u~ = M q~_j on the owned rows; chunk partials of
//      c_i = q_i . q~_j and g_i = (M q_i) . q~_j for i < j (a warp per
//      coefficient and chunk of kDfChunk entries, over the stored rows q_i and
//      M q_i); block partials of nu = ||q~_j||^2 and a~ = q~_j . u~; barrier
//   2  c, g, nu and a~ from the partials (every block sums them in the same
//      order, so every block gets the same bits);
//      r^2 = nu - ||c||^2 (Pythagoras: q~_j - Q c is orthogonal to Q c; when
//      ||c||^2 exceeds a quarter of nu the subtraction would lose digits, and
//      ||q~_j - Q c||^2 is summed directly, one barrier more); r = beta_{j-1};
//      with Q^T M Q = T_j (the tridiagonal matrix so far): alpha_j =
//      q_j . M q_j = (a~ - 2 c.g + c.T_j c) / r^2 and the first pass
//      h = Q^T M q_j = (g - T_j c) / r; then, in one pass over the owned
//      slices of Q and MQ, q_j = (q~_j - Q c) / r, M q_j = (u~ - (MQ) c) / r
//      (column j of the slices, rows j of Q and MQ) and w = M q_j - Q h -
//      alpha_j q_j = (u~ - alpha_j q~_j - (MQ) c - Q (r h - alpha_j c)) / r,
//      written as row j+1 of Q (q~_{j+1}); barrier.
// A launch over steps m0 .. m1-1 ends with a half step m1 (1 without the
// product, then r) that gives beta_{m1-1} and leaves q~_{m1} in row m1 of Q,
// where the next launch resumes.  M arrives scaled by 2^-e (e from the
// largest diagonal entry, which bounds every entry of a positive
// semidefinite matrix) as hi/lo pairs; alpha and beta are stored unscaled in
// FP64.  A breakdown (beta_{j-1} <= 1e-12 of the largest alpha or beta so
// far) stores beta_{j-1} = 0, records stop = j and ends the kernel; the host
// restarts from a new direction (row j of Q), and the first step of a launch
// leaves beta_{m0-1} as stored.
struct DfArgs {
  const float2* M;    // N x N, scaled, hi/lo pairs
  int64_t N;
  float2* Q;          // rows q_i (mcap + 1 rows; row j holds q~_j until step j)
  float2* MQ;         // rows M q_i
  float2* hc;         // chunk partials of c ([mcap + 2][nch])
  float2* hg;         // chunk partials of g
  float2* apart;      // [gridDim][4] block partials: nu, a~, ||q~ - Q c||^2
  double* alpha;
  double* beta;
  const int* escale;  // M was scaled by 2^-escale
  unsigned* bar;
  int* err;
  int* stop;
  int m0, m1, mcap, E, qcap;
  int nch;  // chunks per coefficient
  long long bar_limit;
};

constexpr int kDfThreads = 512;
constexpr int kDfMaxGrid = 256;
constexpr int kDfChunk = 256;     // entries per coefficient task
constexpr int kDfMaxChunks = 8;   // so N <= 2048
constexpr int kDfWarps = kDfThreads / 32;
constexpr int kDfRed = 1024;  // float2 scratch entries per block

// out[e] = base[e] - sum_{i < nv} coef[i] Qs[e][i] for the owned entries:
// a warp per entry (warps w0 .. w0 + nw - 1 of the block), lanes over i
__device__ __forceinline__ void df_combine(const float2* Qs, int qcap, const float2* coef, int nv,
                                           const float2* base, float2* out, int ne, int w0 = 0,
                                           int nw = kDfWarps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = warp - w0; e < ne; e += nw) {
    const float2* q = Qs + (int64_t)e * qcap;
    float s = 0.0f, c = 0.0f;
    for (int i = lane; i < nv; i += 32) df_mac(coef[i], q[i], s, c);
    const float2 t = df_warp_sum(s, c);
    if (lane == 0) out[e] = df_sub(base[e], t);
  }
}

// sum over the blocks' partials part[b * 4 + f] in block order, by one warp
// (the same bits in every block)
__device__ __forceinline__ float2 df_block_sum(const float2* part, int f, int G) {
  const int lane = threadIdx.x & 31;
  float s = 0.0f, c = 0.0f;
  for (int b = lane; b < G; b += 32) df_acc(part[(int64_t)b * 4 + f], s, c);
  return df_warp_sum(s, c);
}

__global__ void __launch_bounds__(kDfThreads, 1) lanczos_df_kernel(DfArgs a) {
  extern __shared__ float2 dfsh[];
  const int64_t N = a.N;
  const int E = a.E, qcap = a.qcap;
  float2* Msh = dfsh;                      // owned rows of M, E x N
  float2* qf = Msh + (int64_t)E * N;       // q~_j, N
  float2* Qs = qf + N;                     // owned slices of q_i, entry-major, E x qcap
  float2* MQs = Qs + (int64_t)E * qcap;    // owned slices of M q_i, E x qcap
  float2* us = MQs + (int64_t)E * qcap;    // owned slice of u~, E
  float2* qn = us + E;                     // owned slice of q~ - Q c (the rare direct norm), E
  float2* cc = qn + E;                     // c, qcap + 1
  float2* cg = cc + (qcap + 1);            // g, qcap + 1
  float2* ch = cg + (qcap + 1);            // T_j c, then d = r h - alpha_j c, qcap + 1
  float2* Ta = ch + (qcap + 1);            // alpha_i (scaled), qcap + 1
  float2* Tb = Ta + (qcap + 1);            // beta_i (scaled), qcap + 1
  float2* red = Tb + (qcap + 1);           // scratch, kDfRed
  const int64_t n0 = (int64_t)blockIdx.x * E;
  const int ne = (int)(N - n0 < E ? (N - n0 > 0 ? N - n0 : 0) : E);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = (int)gridDim.x;
  __shared__ float2 s_nu, s_at, s_cc, s_cgd, s_ctc, s_r2, s_rinv, s_al;
  __shared__ int s_brk, s_direct;
  __shared__ float s_scale;  // largest |alpha|, beta so far (scaled units)
  const double unscale = ldexp(1.0, *a.escale);
  const double rescale = 1.0 / unscale;
  for (int e = 0; e < ne; ++e)
    for (int64_t n = tid; n < N; n += kDfThreads) Msh[(int64_t)e * N + n] = a.M[(n0 + e) * N + n];
  for (int e = warp; e < ne; e += kDfWarps)
    for (int i = lane; i < a.m0 && i < qcap; i += 32) {
      Qs[(int64_t)e * qcap + i] = a.Q[(int64_t)i * N + n0 + e];
      MQs[(int64_t)e * qcap + i] = a.MQ[(int64_t)i * N + n0 + e];
    }
  for (int i = tid; i < a.m0 && i <= qcap; i += kDfThreads) {
    Ta[i] = df_split(a.alpha[i] * rescale);
    Tb[i] = df_split(a.beta[i] * rescale);
  }
  if (tid == 0) {
    float sc = 0.0f;
    for (int i = 0; i < a.m0; ++i)
      sc = fmaxf(sc, fmaxf(fabsf((float)(a.alpha[i] * rescale)), (float)(a.beta[i] * rescale)));
    s_scale = sc;
  }
  // wpr warps share one owned row of the product
  int wpr = 1;
  while (wpr < 8 && 2 * wpr * (ne > 0 ? ne : 1) <= kDfWarps) wpr *= 2;
  const int rows_per_pass = kDfWarps / wpr;
  __syncthreads();
  for (int j = a.m0; j <= a.m1; ++j) {
    const bool full = j < a.m1;  // the last pass is the half step
    // ---- 1: u~ = M q~_j (owned rows); chunk partials of c and g.  The
    // tasks are a warp per coefficient and chunk (the chunks are summed
    // after the barrier); each warp's first task has its loads issued with
    // those of q~_j, before the product.
    const int ntc = j * a.nch, ntask = full ? 2 * ntc : ntc;
    const int task0 = (kDfWarps - 1 - warp) * G + (int)blockIdx.x;
    float2 pv[kDfChunk / 32];
    if (task0 < ntask) {
      const bool isg = task0 >= ntc;
      const int tt = isg ? task0 - ntc : task0;
      const int i = tt / a.nch, chn = tt - i * a.nch;
      const float2* src = (isg ? a.MQ : a.Q) + (int64_t)i * N + (int64_t)chn * kDfChunk + lane;
      const int64_t rem = N - (int64_t)chn * kDfChunk - lane;
#pragma unroll
      for (int u = 0; u < kDfChunk / 32; ++u) pv[u] = u * 32 < rem ? src[u * 32] : make_float2(0.0f, 0.0f);
    }
    for (int64_t n = tid; n < N; n += kDfThreads) qf[n] = a.Q[(int64_t)j * N + n];
    __syncthreads();
    if (full) {
      for (int r = warp / wpr; r < ne; r += rows_per_pass) {
        const float2* row = Msh + (int64_t)r * N;
        // two independent running sums per lane
        float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
        const int st = wpr * 32;
        int64_t n = (warp % wpr) * 32 + lane;
#pragma unroll 2
        for (; n + st < N; n += 2 * st) {
          df_mac(row[n], qf[n], s0, c0);
          df_mac(row[n + st], qf[n + st], s1, c1);
        }
        if (n < N) df_mac(row[n], qf[n], s0, c0);
        float sx, ex;
        two_sum(s0, s1, sx, ex);
        const float2 t = df_warp_sum(sx, (c0 + c1) + ex);
        if (lane == 0) red[r * wpr + warp % wpr] = t;
      }
    }
    for (int t = task0; t < ntask; t += kDfWarps * G) {
      const bool isg = t >= ntc;
      const int tt = isg ? t - ntc : t;
      const int i = tt / a.nch, chn = tt - i * a.nch;
      const int64_t c0 = (int64_t)chn * kDfChunk + lane;
      const float2* src = (isg ? a.MQ : a.Q) + (int64_t)i * N;
      float2 v[kDfChunk / 32];
      if (t == task0) {
#pragma unroll
        for (int u = 0; u < kDfChunk / 32; ++u) v[u] = pv[u];
      } else {
#pragma unroll
        for (int u = 0; u < kDfChunk / 32; ++u) {
          const int64_t n = c0 + u * 32;
          v[u] = n < N ? src[n] : make_float2(0.0f, 0.0f);
        }
      }
      float s = 0.0f, c = 0.0f;
#pragma unroll
      for (int u = 0; u < kDfChunk / 32; ++u) {
        const int64_t n = c0 + u * 32;
        if (n < N) df_mac(v[u], qf[n], s, c);
      }
      const float2 r2 = df_warp_sum(s, c);
      if (lane == 0) (isg ? a.hg : a.hc)[(int64_t)i * a.nch + chn] = r2;
    }
    __syncthreads();
    if (full && tid < ne) {
      float s = 0.0f, c = 0.0f;
      for (int p = 0; p < wpr; ++p) df_acc(red[tid * wpr + p], s, c);
      us[tid] = df_norm(s, c);
    }
    __syncthreads();
    if (warp == 0) {
      float s = 0.0f, c = 0.0f;
      for (int e = lane; e < ne; e += 32) df_mac(qf[n0 + e], qf[n0 + e], s, c);
      const float2 t = df_warp_sum(s, c);
      if (lane == 0) a.apart[(int64_t)blockIdx.x * 4 + 0] = t;
    } else if (warp == 1 && full) {
      float s = 0.0f, c = 0.0f;
      for (int e = lane; e < ne; e += 32) df_mac(qf[n0 + e], us[e], s, c);
      const float2 t = df_warp_sum(s, c);
      if (lane == 0) a.apart[(int64_t)blockIdx.x * 4 + 1] = t;
    }
    if (!grid_barrier_at(a.bar, a.err, a.bar_limit)) return;
    // ---- 2: the coefficients and norms; q_j, u, alpha_j, h and w
    for (int i = tid; i < j; i += kDfThreads) {
      float2 vc[kDfMaxChunks], vg[kDfMaxChunks];
#pragma unroll
      for (int chn = 0; chn < kDfMaxChunks; ++chn) {
        vc[chn] = chn < a.nch ? a.hc[(int64_t)i * a.nch + chn] : make_float2(0.0f, 0.0f);
        vg[chn] = full && chn < a.nch ? a.hg[(int64_t)i * a.nch + chn] : make_float2(0.0f, 0.0f);
      }
      float s = 0.0f, c = 0.0f, s2 = 0.0f, c2 = 0.0f;
#pragma unroll
      for (int chn = 0; chn < kDfMaxChunks; ++chn) {
        df_acc(vc[chn], s, c);
        df_acc(vg[chn], s2, c2);
      }
      cc[i] = df_norm(s, c);
      cg[i] = df_norm(s2, c2);
    }
    if (warp == kDfWarps - 1) {
      const float2 t = df_block_sum(a.apart, 0, G);
      if (lane == 0) s_nu = t;
    } else if (warp == kDfWarps - 2 && full) {
      const float2 t = df_block_sum(a.apart, 1, G);
      if (lane == 0) s_at = t;
    }
    __syncthreads();
    // T_j c and the sums ||c||^2, c.g, c.T_j c (three warps)
    if (warp < 3) {
      float s = 0.0f, c = 0.0f;
      for (int i = lane; i < j; i += 32) {
        const float2 ci = cc[i];
        if (warp == 0) {
          df_mac(ci, ci, s, c);
        } else if (warp == 1) {
          df_mac(ci, cg[i], s, c);
        } else {
          // (T_j c)_i over the entries of T_j (indices below j)
          float ts = 0.0f, tcr = 0.0f;
          df_mac(Ta[i], ci, ts, tcr);
          if (i > 0) df_mac(Tb[i - 1], cc[i - 1], ts, tcr);
          if (i + 1 < j) df_mac(Tb[i], cc[i + 1], ts, tcr);
          const float2 tci = df_norm(ts, tcr);
          ch[i] = tci;
          df_mac(ci, tci, s, c);
        }
      }
      const float2 t = df_warp_sum(s, c);
      if (lane == 0) {
        if (warp == 0) s_cc = t;
        else if (warp == 1) s_cgd = t;
        else s_ctc = t;
      }
    }
    __syncthreads();
    if (tid == 0) {
      const float2 nu = s_nu, c2 = s_cc;
      s_direct = c2.x > 0.25f * nu.x;  // the same decision in every block
      s_r2 = df_sub(nu, c2);
    }
    __syncthreads();
    if (s_direct) {
      // ||q~_j - Q c||^2 summed directly, one barrier more
      df_combine(Qs, qcap, cc, j, qf + n0, qn, ne);
      __syncthreads();
      if (warp == 0) {
        float s = 0.0f, c = 0.0f;
        for (int e = lane; e < ne; e += 32) df_mac(qn[e], qn[e], s, c);
        const float2 t = df_warp_sum(s, c);
        if (lane == 0) a.apart[(int64_t)blockIdx.x * 4 + 2] = t;
      }
      if (!grid_barrier_at(a.bar, a.err, a.bar_limit)) return;
      if (warp == 0) {
        const float2 t = df_block_sum(a.apart, 2, G);
        if (lane == 0) s_r2 = t;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const float2 r = df_sqrt(s_r2);
      float sc = s_scale;
      int brk = 0;
      if (j > a.m0) {
        // r = beta_{j-1}
        brk = !(r.x > 1e-12f * sc) || sc == 0.0f;
        if (!brk) {
          sc = fmaxf(sc, r.x);
          Tb[j - 1] = r;
        }
        if (blockIdx.x == 0) {
          a.beta[j - 1] = brk ? 0.0 : df_val(r) * unscale;
          if (brk) *a.stop = j;
        }
      }
      s_brk = brk;
      s_rinv = r.x > 0.0f ? df_rcp(r) : make_float2(0.0f, 0.0f);
      if (full && !brk) {
        // alpha_j = (a~ - 2 c.g + c.T_j c) / r^2
        const float2 ri = s_rinv;
        const float2 num = df_add(df_sub(s_at, df_add(s_cgd, s_cgd)), s_ctc);
        const float2 al = df_mul(df_mul(num, ri), ri);
        sc = fmaxf(sc, fabsf(al.x));
        Ta[j] = al;
        s_al = al;
        if (blockIdx.x == 0) a.alpha[j] = df_val(al) * unscale;
      }
      s_scale = sc;
    }
    __syncthreads();
    if (s_brk || !full) return;  // the same decision in every block
    const float2 rinv = s_rinv, al = s_al;
    // d = (g - T_j c) - alpha_j c = r h - alpha_j c, so that
    // r w = u~ - alpha_j q~_j - (MQ) c - Q d
    for (int i = tid; i < j; i += kDfThreads) ch[i] = df_sub(df_sub(cg[i], ch[i]), df_mul(al, cc[i]));
    __syncthreads();
    // q_j = (q~_j - Q c) / r, M q_j = (u~ - (MQ) c) / r and w on the owned
    // slice in one pass over the basis (a warp per entry, lanes over i)
    for (int e = warp; e < ne; e += kDfWarps) {
      const float2* qe = Qs + (int64_t)e * qcap;
      const float2* me = MQs + (int64_t)e * qcap;
      float s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f, s3 = 0.0f, c3 = 0.0f;
      for (int i = lane; i < j; i += 32) {
        const float2 qi = qe[i], ci = cc[i];
        df_mac(ci, qi, s1, c1);
        df_mac(ci, me[i], s2, c2);
        df_mac(ch[i], qi, s3, c3);
      }
      const float2 t1 = df_warp_sum(s1, c1), t2 = df_warp_sum(s2, c2), t3 = df_warp_sum(s3, c3);
      if (lane == 0) {
        const float2 qt = qf[n0 + e], ut = us[e];
        const float2 q = df_mul(df_sub(qt, t1), rinv);
        const float2 u = df_mul(df_sub(ut, t2), rinv);
        const float2 w = df_mul(df_sub(df_sub(df_sub(ut, df_mul(al, qt)), t2), t3), rinv);
        Qs[(int64_t)e * qcap + j] = q;
        MQs[(int64_t)e * qcap + j] = u;
        a.Q[(int64_t)j * N + n0 + e] = q;
        a.MQ[(int64_t)j * N + n0 + e] = u;
        a.Q[(int64_t)(j + 1) * N + n0 + e] = w;  // q~_{j+1}
      }
    }
    if (!grid_barrier_at(a.bar, a.err, a.bar_limit)) return;
  }
}

// 2^e >= the largest diagonal entry of the n x n matrix M (one block)
__global__ void df_scale_kernel(const double* M, int64_t n, int* escale) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(M[i * n + i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sh[w]);
    mx = fmax(mx, sh[0]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx < 2^e
    *escale = e;
  }
}

// M (FP64) -> 2^-e M as hi/lo pairs, in place (the same 8 bytes per entry)
__global__ void df_split_kernel(double* M, int64_t n2, const int* escale) {
  const double sc = ldexp(1.0, -*escale);
  float2* out = reinterpret_cast<float2*>(M);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df_split(M[i] * sc);
}

// q_0: a counter-based random unit vector (hi/lo pairs)
__global__ void df_start_kernel(float2* q, int64_t N, uint64_t key) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const double v = rnd_sym(key, n);
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) q[n] = df_split(rnd_sym(key, n) * inv);
}

// Restart after a breakdown that ended step m - 1: q_m = a counter-based
// random vector orthogonalised twice against q_0 .. q_{m-1}, normalised (one
// block, FP64, w in shared memory; a rare path)
__global__ void df_restart_kernel(float2* Q, int64_t N, int m, uint64_t key) {
  extern __shared__ double rsh[];
  double* w = rsh;      // N
  double* c = rsh + N;  // m
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) w[n] = rnd_sym(key + (uint64_t)m * 0x9E3779B97F4A7C15ull, n);
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = warp; i < m; i += nwarp) {
      const float2* q = Q + (int64_t)i * N;
      double s = 0.0;
      for (int64_t n = lane; n < N; n += 32) s = fma(df_val(q[n]), w[n], s);
      s = warp_sum(s);
      if (lane == 0) c[i] = s;
    }
    __syncthreads();
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
      double v = w[n];
      for (int i = 0; i < m; ++i) v = fma(-c[i], df_val(Q[(int64_t)i * N + n]), v);
      w[n] = v;
    }
    __syncthreads();
  }
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s = fma(w[n], w[n], s);
  s = block_sum(s, sh);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) Q[(int64_t)m * N + n] = df_split(w[n] * inv);
}

// ------------------------------------------------------ back-projection ----
// B[n][i k + c] = delta[n][i] u[n][c]  (N x Tout k), or its transpose
// B[i k + c][n] (trans: the rows that the digit split reads along n)
__global__ void bp_build_kernel(const double* D, const double* U, int64_t N, int Tout, int k, double* B, int trans) {
  const int64_t cols = (int64_t)Tout * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t n, r;
    if (trans) {
      r = t / N;
      n = t - r * N;
    } else {
      n = t / cols;
      r = t - n * cols;
    }
    const int i = (int)(r / k), c = (int)(r - (int64_t)i * k);
    B[t] = D[n * Tout + i] * U[n * k + c];
  }
}

// evecs[c][woff + i Tin + j] = R[j][i k + c], evecs[c][boff + i] = Rb[i][c]
__global__ void bp_scatter_kernel(const double* R, const double* Rb, int Tin, int Tout, int k, double* evecs,
                                  int64_t P, int64_t woff, int64_t boff) {
  const int64_t per = (int64_t)(Tin + 1) * Tout;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < per * k;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / per);
    const int64_t p = t - (int64_t)c * per;
    if (p < (int64_t)Tin * Tout) {
      const int64_t i = p / Tin, j = p - i * Tin;
      evecs[(int64_t)c * P + woff + p] = R[j * Tout * (int64_t)k + i * k + c];
    } else {
      const int64_t i = p - (int64_t)Tin * Tout;
      evecs[(int64_t)c * P + boff + i] = Rb[i * k + c];
    }
  }
}

// Cluster boundaries of the Ritz values (descending): eigenvalues closer
// than ortol to their predecessor share a cluster whose eigenvectors are
// orthogonalised against each other during inverse iteration.
__global__ void clusters_kernel(const double* theta, int k, double rel, int* start) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double ortol = rel * fabs(theta[0]);
  int s = 0;
  for (int c = 0; c < k; ++c) {
    if (c > 0 && theta[c - 1] - theta[c] > ortol) s = c;
    start[c] = s;
  }
}

// ----------------------------------------------------- tridiagonal eigen
// Number of eigenvalues of T below x (Sturm count) from the signs of the
// leading principal minors p_i = det(T_i - x I):
//   p_0 = 1,  p_1 = a_0 - x,  p_{i+1} = (a_i - x) p_i - b_{i-1}^2 p_{i-1},
// the count being the number of sign changes along p_0 .. p_m (Sturm
// sequence property).  The recurrence needs no division: its dependent
// chain is one FMA per step (b^2 p_{i-1} is ready a step early), which
// matters where an FP64 operation waits tens of cycles for its inputs.
// Every 8 steps the pair (p_i, p_{i-1}) is rescaled by a power of two (exact,
// signs unchanged); a and b2 arrive scaled so that ||T|| <= 1.  A minor that
// comes out exactly zero is replaced by a tiny value of the opposite sign of
// its predecessor (it counts as one change).
__device__ int sturm_count(const double* a, const double* b2, int m, double x) {
  double pm1 = 1.0;
  double p = a[0] - x;
  int cnt = 0;
  unsigned long long sprev = 0ull;  // sign bit of p_0
  auto step_sign = [&](double& v) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    if ((bits & 0x7fffffffffffffffull) == 0ull) {
      bits = 0x0010000000000000ull | ((sprev ^ 1ull) << 63);  // +-DBL_MIN
      v = __longlong_as_double((long long)bits);
    }
    const unsigned long long sb = bits >> 63;
    cnt += (int)(sb ^ sprev);
    sprev = sb;
  };
  step_sign(p);
#pragma unroll 8
  for (int i = 1; i < m; ++i) {
    const double t = b2[i - 1] * pm1;
    double pn = fma(a[i] - x, p, -t);
    step_sign(pn);
    pm1 = p;
    p = pn;
    if ((i & 7) == 0) {
      const int ep = (int)(((unsigned long long)__double_as_longlong(p) >> 52) & 0x7ff);
      const int eq = (int)(((unsigned long long)__double_as_longlong(pm1) >> 52) & 0x7ff);
      const int e = ep > eq ? ep : eq;
      if (e > 1023 + 256 || e < 1023 - 256) {
        const double sc = __longlong_as_double((long long)(2046 - e) << 52);  // 2^(1023 - e)
        p *= sc;
        pm1 *= sc;
      }
    }
  }
  return cnt;
}

// The same count in FP32 (rescaled every 4 steps), for coarse brackets.
__device__ int sturm_count_f32(const float* a, const float* b2, int m, float x) {
  float pm1 = 1.0f;
  float p = a[0] - x;
  int cnt = 0;
  unsigned sprev = 0u;
  auto step_sign = [&](float& v) {
    unsigned bits = __float_as_uint(v);
    if ((bits & 0x7fffffffu) == 0u) {
      bits = 0x00800000u | ((sprev ^ 1u) << 31);  // +-FLT_MIN
      v = __uint_as_float(bits);
    }
    const unsigned sb = bits >> 31;
    cnt += (int)(sb ^ sprev);
    sprev = sb;
  };
  step_sign(p);
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    const float t = b2[i - 1] * pm1;
    float pn = fmaf(a[i] - x, p, -t);
    step_sign(pn);
    pm1 = p;
    p = pn;
    if ((i & 3) == 0) {
      const int ep = (int)((__float_as_uint(p) >> 23) & 0xff);
      const int eq = (int)((__float_as_uint(pm1) >> 23) & 0xff);
      const int e = ep > eq ? ep : eq;
      if (e > 127 + 40 || e < 127 - 40) {
        const float sc = __uint_as_float((unsigned)(254 - e) << 23);  // 2^(127 - e)
        p *= sc;
        pm1 *= sc;
      }
    }
  }
  return cnt;
}

// The same count in double-float (devmath.cuh), rescaled every 4 steps: on
// the FP32 pipe, resolving eigenvalues to about 1e-13 ||T|| between the FP32
// sweeps and the FP64 ones.
__device__ int sturm_count_df(const float2* a, const float2* b2, int m, float2 x) {
  float2 pm1 = make_float2(1.0f, 0.0f);
  float2 p = df_sub(a[0], x);
  int cnt = 0;
  unsigned sprev = 0u;
  auto step_sign = [&](float2& v) {
    unsigned bits = __float_as_uint(v.x);
    if ((bits & 0x7fffffffu) == 0u) {
      bits = 0x00800000u | ((sprev ^ 1u) << 31);  // +-FLT_MIN
      v = make_float2(__uint_as_float(bits), 0.0f);
    }
    const unsigned sb = bits >> 31;
    cnt += (int)(sb ^ sprev);
    sprev = sb;
  };
  step_sign(p);
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    const float2 t = df_mul(b2[i - 1], pm1);
    float2 pn = df_sub(df_mul(df_sub(a[i], x), p), t);
    step_sign(pn);
    pm1 = p;
    p = pn;
    if ((i & 3) == 0) {
      const int ep = (int)((__float_as_uint(p.x) >> 23) & 0xff);
      const int eq = (int)((__float_as_uint(pm1.x) >> 23) & 0xff);
      const int e = ep > eq ? ep : eq;
      if (e > 127 + 40 || e < 127 - 40) {
        const float sc = __uint_as_float((unsigned)(254 - e) << 23);  // 2^(127 - e)
        p = make_float2(p.x * sc, p.y * sc);
        pm1 = make_float2(pm1.x * sc, pm1.y * sc);
      }
    }
  }
  return cnt;
}

// Smallest thread index of the block whose predicate holds (blockDim.x if
// none); every thread gets the answer.
__device__ int block_first(bool pred, int* s4) {
  const unsigned bal = __ballot_sync(0xffffffffu, pred);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s4[warp] = bal ? warp * 32 + __ffs(bal) - 1 : (int)blockDim.x;
  __syncthreads();
  int f = (int)blockDim.x;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) f = min(f, s4[w]);
  __syncthreads();
  return f;
}

// theta[c] = c-th largest eigenvalue of T_m, one block of 128 threads per
// eigenvalue (one warp per SM partition): each sweep evaluates the Sturm
// count at 128 interior points of the bracket (multisection), shrinking it
// 129-fold.  T is staged in shared memory, scaled by a power of two so that
// ||T|| <= 1.  Two coarse sweeps run in FP32; their bracket is widened by
// 4e-6 (well above the FP32 backward error of the count, a few float ulps of
// ||T||) before the FP64 sweeps take it down to a few ulps.
__global__ void bisect_kernel(const double* a, const double* b, int m, int k, double* theta, double* gscratch) {
  extern __shared__ double tsh_s[];
  // T's copies in shared memory, or (when 3 m doubles exceed it) in a global
  // scratch of 3 m doubles per block
  double* tsh = gscratch ? gscratch + (int64_t)blockIdx.x * 3 * m : tsh_s;
  double* sa = tsh;
  double* sb2 = tsh + m;
  float* fa = reinterpret_cast<float*>(tsh + 2 * m);
  float* fb2 = fa + m;
  __shared__ double s_lo, s_hi, s_sc;
  __shared__ int s4[32];
  const int c = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (c >= k) return;
  if (tid < 32) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = tid; i < m; i += 32) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (tid == 0) {
      const double tnorm = fmax(fabs(lo), fabs(hi));
      int E = 0;
      if (tnorm > 0.0) frexp(tnorm, &E);
      const double sc = ldexp(1.0, -E);  // 2^-E with 2^E >= tnorm: exact
      s_sc = sc;
      s_lo = lo * sc - (2.0 * DBL_EPSILON + 4.0 * DBL_MIN);
      s_hi = hi * sc + (2.0 * DBL_EPSILON + 4.0 * DBL_MIN);
    }
  }
  __syncthreads();
  const double sc = s_sc;
  for (int i = tid; i < m; i += nt) {
    const double ai = a[i] * sc;
    const double bi = i < m - 1 ? b[i] * sc : 0.0;
    sa[i] = ai;
    sb2[i] = bi * bi;
    fa[i] = (float)ai;
    fb2[i] = (float)(bi * bi);
  }
  __syncthreads();
  const int t = m - 1 - c;  // index from the smallest
  double lo = s_lo, hi = s_hi;
  const double lo0 = lo, hi0 = hi;
  const double inv_n = 1.0 / (double)(nt + 1);
  // coarse FP32 sweeps
  for (int it = 0; it < 2; ++it) {
    const float xf = (float)(lo + (hi - lo) * (double)(tid + 1) * inv_n);
    const int f = block_first(sturm_count_f32(fa, fb2, m, xf) > t, s4);
    const double nhi = f < nt ? lo + (hi - lo) * (double)(f + 1) * inv_n : hi;
    const double nlo = f > 0 ? lo + (hi - lo) * (double)f * inv_n : lo;
    lo = nlo;
    hi = nhi;
  }
  lo = fmax(lo0, lo - 4e-6);
  hi = fmin(hi0, hi + 4e-6);
  // down to a few ulps of the eigenvalue, or to 4 eps ||T|| (the accuracy of
  // any backward-stable symmetric eigensolver) for eigenvalues much smaller
  // than ||T||
  const double tiny = 4.0 * DBL_MIN;
  const double tol_abs = 4.0 * DBL_EPSILON * fmax(fabs(lo0), fabs(hi0));
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= fmax(2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)), tol_abs) + tiny) break;
    const double x = lo + (hi - lo) * (double)(tid + 1) * inv_n;
    const int f = block_first(sturm_count(sa, sb2, m, x) > t, s4);
    const double nhi = f < nt ? lo + (hi - lo) * (double)(f + 1) * inv_n : hi;
    const double nlo = f > 0 ? lo + (hi - lo) * (double)f * inv_n : lo;
    if (!(nlo < nhi)) break;
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) theta[c] = 0.5 * (lo + hi) / sc;
}

// The same multisection with a cluster of kBisCta CTAs per eigenvalue: each
// CTA evaluates 128 of the kBisCta * 128 points of a sweep (the bracket
// shrinks (kBisCta * 128 + 1)-fold), the CTAs exchange their first crossing
// through distributed shared memory, and all of them take the same new
// bracket, so they make the same number of cluster barriers.  Two FP32
// sweeps, then double-float sweeps down to 2^-40 ||T||: the eigenvalue to
// about 1e-12 ||T||, which the inverse iteration's Rayleigh quotient takes to
// FP64 rounding (FP64 Sturm counts, bound by this GPU's FP64 rate, are left
// out).
constexpr int kBisCta = 4;
__global__ void bisect_cluster_kernel(const double* a, const double* b, int m, int k, double* theta) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double tsh_c[];
  float* fa = reinterpret_cast<float*>(tsh_c);
  float* fb2 = fa + m;
  float2* da = reinterpret_cast<float2*>(tsh_c + m);
  float2* db2 = da + m;
  __shared__ double s_lo, s_hi, s_sc;
  __shared__ int s4[32];
  __shared__ int s_first;  // this CTA's first crossing in the current sweep (128: none)
  const int c = blockIdx.x / kBisCta;
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;  // nt = 128
  // c is the same for the whole cluster, so a cluster leaves together
  if (c >= k) return;
  if (tid < 32) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = tid; i < m; i += 32) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (tid == 0) {
      const double tnorm = fmax(fabs(lo), fabs(hi));
      int E = 0;
      if (tnorm > 0.0) frexp(tnorm, &E);
      const double sc = ldexp(1.0, -E);
      s_sc = sc;
      s_lo = lo * sc - (2.0 * DBL_EPSILON + 4.0 * DBL_MIN);
      s_hi = hi * sc + (2.0 * DBL_EPSILON + 4.0 * DBL_MIN);
    }
  }
  __syncthreads();
  const double sc = s_sc;
  for (int i = tid; i < m; i += nt) {
    const double ai = a[i] * sc;
    const double bi = i < m - 1 ? b[i] * sc : 0.0;
    fa[i] = (float)ai;
    fb2[i] = (float)(bi * bi);
    da[i] = df_split(ai);
    db2[i] = df_split(bi * bi);
  }
  __syncthreads();
  const int t = m - 1 - c;  // index from the smallest
  const int np = kBisCta * nt;  // points per sweep
  const double inv_n = 1.0 / (double)(np + 1);
  const int g = rank * nt + tid;  // this thread's point
  double lo = s_lo, hi = s_hi;
  const double lo0 = lo, hi0 = hi;
  // the cluster's first crossing of a sweep, from every CTA's own
  auto cluster_first = [&](bool pred) -> int {
    const int f = block_first(pred, s4);
    if (tid == 0) s_first = f;
    cluster.sync();
    int F = np;
    for (int r = 0; r < kBisCta; ++r) {
      const int fr = *cluster.map_shared_rank(&s_first, r);
      if (fr < nt) {
        F = r * nt + fr;
        break;
      }
    }
    cluster.sync();  // every CTA has read s_first before the next sweep writes it
    return F;
  };
  // coarse FP32 sweeps
  for (int it = 0; it < 2; ++it) {
    const float xf = (float)(lo + (hi - lo) * (double)(g + 1) * inv_n);
    const int F = cluster_first(sturm_count_f32(fa, fb2, m, xf) > t);
    const double nhi = F < np ? lo + (hi - lo) * (double)(F + 1) * inv_n : hi;
    const double nlo = F > 0 ? lo + (hi - lo) * (double)F * inv_n : lo;
    lo = nlo;
    hi = nhi;
  }
  lo = fmax(lo0, lo - 4e-6);
  hi = fmin(hi0, hi + 4e-6);
  // double-float sweeps down to 2^-40 of ||T|| (<= 1 here): the midpoint is
  // then within about 1e-12 ||T|| of the eigenvalue, the double-float count's
  // error included
  for (int it = 0; it < 8; ++it) {
    if (hi - lo <= 9.1e-13) break;
    const double x = lo + (hi - lo) * (double)(g + 1) * inv_n;
    const int F = cluster_first(sturm_count_df(da, db2, m, df_split(x)) > t);
    const double nhi = F < np ? lo + (hi - lo) * (double)(F + 1) * inv_n : hi;
    const double nlo = F > 0 ? lo + (hi - lo) * (double)F * inv_n : lo;
    if (!(nlo < nhi)) break;
    lo = nlo;
    hi = nhi;
  }
  // (the inverse iteration refines the eigenvalue to FP64 rounding by the
  // Rayleigh quotient of its vector)
  if (rank == 0 && tid == 0) theta[c] = 0.5 * (lo + hi) / sc;
}

// Eigenvectors of T_m for theta[0..k-1] by inverse iteration with a
// partially pivoted tridiagonal LU of (T - theta I).  One block per cluster
// (block c works only if c starts a cluster); inside a cluster the vectors
// are found in order, each orthogonalised against the earlier ones at every
// iteration.  Thread 0 runs the O(m) recurrences (elimination and solves);
// the fill, the reciprocal pivots and the norms are spread over the block.
// Y: k rows of length ldy.
// res[c] = |beta_m y_c[m-1]| bounds the residual of Ritz pair c.
__global__ void inviter_kernel(const double* a, const double* b, int m, int k, double* theta,
                               const int* cstart, double* Y, int64_t ldy, const double* beta_last,
                               double* res, uint64_t key, double* gscratch) {
  const int c0 = blockIdx.x;
  if (cstart[c0] != c0) return;
  __shared__ double sh[32];
  __shared__ double sdot[1024];
  // the O(m) recurrences run on copies in shared memory (5 m doubles + m
  // ints), or in a global scratch of 6 m doubles per block when too large
  extern __shared__ double ish_s[];
  double* ish = gscratch ? gscratch + (int64_t)blockIdx.x * 6 * m : ish_s;
  double* d = ish;
  double* du = ish + m;
  double* dl = ish + 2 * m;
  double* du2 = ish + 3 * m;
  double* ys = ish + 4 * m;
  int* piv = reinterpret_cast<int*>(ish + 5 * m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // block-wide FP64 scalars are computed by one warp (an FP64 instruction
  // occupies its SM partition for many cycles) and shared
  __shared__ double s_tiny, s_inv;
  if (warp == 0) {
    double tn = 0.0;
    for (int i = lane; i < m; i += 32)
      tn = fmax(tn, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    if (lane == 0) s_tiny = DBL_EPSILON * fmax(tn, DBL_MIN);
  }
  __syncthreads();
  const double tiny = s_tiny;
  const double beta_m = *beta_last;
  for (int c = c0; c < k && cstart[c] == c0; ++c) {
    const double th = theta[c];
    double* y = ys;
    // T - theta I by all threads; the elimination below is sequential
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      d[i] = a[i] - th;
      if (i < m - 1) {
        du[i] = b[i];
        dl[i] = b[i];
      }
      du2[i] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < m - 1; ++i) {
        if (fabs(d[i]) >= fabs(dl[i])) {
          piv[i] = 0;
          if (fabs(d[i]) < tiny) d[i] = d[i] < 0 ? -tiny : tiny;
          const double f = dl[i] * rcp64(d[i]);
          dl[i] = f;
          d[i + 1] -= f * du[i];
        } else {
          piv[i] = 1;
          const double f = d[i] * rcp64(dl[i]);
          d[i] = dl[i];
          dl[i] = f;
          const double tmp = du[i];
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
    __syncthreads();
    // the solves multiply by the reciprocal pivots
    for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = rcp64(d[i]);
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = 1.0 + 0.25 * rnd_sym(key + c, i);
    __syncthreads();
    // two solves: with a shift accurate to a few ulps the first leaves an
    // error of about eps ||T|| / gap, the second removes it
    for (int it = 0; it < 2; ++it) {
      if (warp == 0) {
        if (lane == 0) {
          for (int i = 0; i < m - 1; ++i) {
            if (piv[i]) {
              const double t = y[i];
              y[i] = y[i + 1];
              y[i + 1] = t;
            }
            y[i + 1] -= dl[i] * y[i];
          }
          y[m - 1] *= d[m - 1];
          if (m >= 2) y[m - 2] = (y[m - 2] - du[m - 2] * y[m - 1]) * d[m - 2];
          for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * d[i];
        }
        __syncwarp();
        // max |y_i| over the warp (exact in any order)
        double mx = 0.0;
        for (int i = lane; i < m; i += 32) mx = fmax(mx, fabs(y[i]));
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) sh[0] = mx > 0.0 ? 1.0 / mx : 1.0;
      }
      __syncthreads();
      const double inv = sh[0];
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= inv;
      __syncthreads();
      // orthogonalise against the cluster's earlier vectors (twice)
      const int nprev = c - c0;
      for (int pass = 0; pass < 2 && nprev > 0; ++pass) {
        for (int pb = 0; pb < nprev; pb += 1024) {
          const int cnt = nprev - pb < 1024 ? nprev - pb : 1024;
          for (int pi = warp; pi < cnt; pi += nwarp) {
            const double* yp = Y + (int64_t)(c0 + pb + pi) * ldy;
            double dot = 0.0;
            for (int i = lane; i < m; i += 32) dot = fma(yp[i], y[i], dot);
            dot = warp_sum(dot);
            if (lane == 0) sdot[pi] = dot;
          }
          __syncthreads();
          for (int i = threadIdx.x; i < m; i += blockDim.x) {
            double s = 0.0;
            for (int pi = 0; pi < cnt; ++pi) s = fma(sdot[pi], Y[(int64_t)(c0 + pb + pi) * ldy + i], s);
            y[i] -= s;
          }
          __syncthreads();
        }
      }
      double nn = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) nn = fma(y[i], y[i], nn);
      nn = block_sum(nn, sh);
      if (threadIdx.x == 0) s_inv = nn > 0.0 ? rsqrt64(nn) : 0.0;
      __syncthreads();
      const double inv2 = s_inv;
      for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= inv2;
      __syncthreads();
    }
    if (threadIdx.x == 0) res[c] = fabs(beta_m * y[m - 1]);
    for (int i = threadIdx.x; i < m; i += blockDim.x) Y[(int64_t)c * ldy + i] = y[i];
    // theta_c = y^T T y (unit y): the eigenvalue to FP64 rounding (its error
    // is quadratic in the vector's)
    double rq = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      rq = fma(y[i], fma(a[i], y[i], i + 1 < m ? 2.0 * b[i] * y[i + 1] : 0.0), rq);
    rq = block_sum(rq, sh);
    if (threadIdx.x == 0) theta[c] = rq;
    __syncthreads();
  }
}

// The same inverse iteration with the O(m) recurrences (elimination and the
// two solves, one thread's dependent chains) in double-float on T scaled by
// a power of two (||T|| < 1; the eigenvector does not change): a dependent
// step costs a few FP32 latencies instead of several FP64 ones.  The
// normalisation and the orthogonalisation within a cluster stay FP64, on an
// FP64 copy of the vector.  Needs 7 m doubles of shared memory.
__global__ void inviter_df_kernel(const double* a, const double* b, int m, int k, double* theta,
                                  const int* cstart, double* Y, int64_t ldy, const double* beta_last, double* res,
                                  uint64_t key) {
  const int c0 = blockIdx.x;
  if (cstart[c0] != c0) return;
  __shared__ double sh[32];
  __shared__ double sdot[1024];
  extern __shared__ double idf_s[];
  float2* d = reinterpret_cast<float2*>(idf_s);
  float2* du = d + m;
  float2* dl = du + m;
  float2* du2 = dl + m;
  float2* y = du2 + m;
  double* y64 = idf_s + 5 * m;
  int* piv = reinterpret_cast<int*>(idf_s + 6 * m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  __shared__ double s_sc, s_inv;
  __shared__ float s_tiny;
  if (warp == 0) {
    double tn = 0.0;
    for (int i = lane; i < m; i += 32)
      tn = fmax(tn, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    if (lane == 0) {
      int E = 0;
      if (tn > 0.0) frexp(tn, &E);
      const double sc = ldexp(1.0, -E);  // exact
      s_sc = sc;
      s_tiny = (float)(DBL_EPSILON * fmax(tn * sc, DBL_MIN));
    }
  }
  __syncthreads();
  const double sc = s_sc;
  const float tiny = s_tiny;
  const double beta_m = *beta_last;
  for (int c = c0; c < k && cstart[c] == c0; ++c) {
    const double th = theta[c] * sc;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      d[i] = df_split(a[i] * sc - th);
      if (i < m - 1) {
        du[i] = df_split(b[i] * sc);
        dl[i] = du[i];
      }
      du2[i] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    if (c == c0 && (c + 1 >= k || cstart[c + 1] != c0)) {
      // a cluster of one: the eigenvector from a twisted factorization of
      // T - theta I (the pivots d+ from the top and d- from the bottom, one
      // thread each; the twist r where gamma_r = d+_r + d-_r - (a_r - theta)
      // is smallest in magnitude; then z_r = 1 and the products outward,
      // z_i = -(b_i / d+_i) z_{i+1} above r, z_i = -(b_{i-1} / d-_i) z_{i-1}
      // below), with no iteration
      float2* dp = du2;
      float2* dm = y;
      if (threadIdx.x == 0) {
        float2 p = d[0];
        if (fabsf(p.x) < tiny) p = make_float2(p.x < 0.0f ? -tiny : tiny, 0.0f);
        dp[0] = p;
        for (int i = 1; i < m; ++i) {
          p = df_sub(d[i], df_mul(df_mul(du[i - 1], du[i - 1]), df_rcp(p)));
          if (fabsf(p.x) < tiny) p = make_float2(p.x < 0.0f ? -tiny : tiny, 0.0f);
          dp[i] = p;
        }
      } else if (threadIdx.x == 32) {
        float2 q = d[m - 1];
        if (fabsf(q.x) < tiny) q = make_float2(q.x < 0.0f ? -tiny : tiny, 0.0f);
        dm[m - 1] = q;
        for (int i = m - 2; i >= 0; --i) {
          q = df_sub(d[i], df_mul(df_mul(du[i], du[i]), df_rcp(q)));
          if (fabsf(q.x) < tiny) q = make_float2(q.x < 0.0f ? -tiny : tiny, 0.0f);
          dm[i] = q;
        }
      }
      __syncthreads();
      float gmin = FLT_MAX;
      int gidx = m;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float g = fabsf(df_sub(df_add(dp[i], dm[i]), d[i]).x);
        if (g < gmin) {
          gmin = g;
          gidx = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float g2 = __shfl_xor_sync(0xffffffffu, gmin, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, gidx, o);
        if (g2 < gmin || (g2 == gmin && i2 < gidx)) {
          gmin = g2;
          gidx = i2;
        }
      }
      if (lane == 0) {
        sdot[2 * warp] = (double)gmin;
        sdot[2 * warp + 1] = (double)gidx;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double bg = sdot[0];
        int bi = (int)sdot[1];
        for (int w = 1; w < nwarp; ++w)
          if (sdot[2 * w] < bg) {
            bg = sdot[2 * w];
            bi = (int)sdot[2 * w + 1];
          }
        piv[0] = bi;
      }
      __syncthreads();
      const int r = piv[0];
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < r)
          y64[i] = -df_val(df_mul(du[i], df_rcp(dp[i])));
        else if (i > r)
          y64[i] = -df_val(df_mul(du[i - 1], df_rcp(dm[i])));
        else
          y64[i] = 1.0;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int i = r - 1; i >= 0; --i) y64[i] *= y64[i + 1];
      } else if (threadIdx.x == 32) {
        for (int i = r + 1; i < m; ++i) y64[i] *= y64[i - 1];
      }
      __syncthreads();
      double nn = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) nn = fma(y64[i], y64[i], nn);
      nn = block_sum(nn, sh);
      if (threadIdx.x == 0) s_inv = nn > 0.0 ? rsqrt64(nn) : 0.0;
      __syncthreads();
      const double inv2 = s_inv;
      for (int i = threadIdx.x; i < m; i += blockDim.x) y64[i] *= inv2;
      __syncthreads();
    } else {
      if (threadIdx.x == 0) {
        for (int i = 0; i < m - 1; ++i) {
          if (fabsf(d[i].x) >= fabsf(dl[i].x)) {
            piv[i] = 0;
            if (fabsf(d[i].x) < tiny) d[i] = make_float2(d[i].x < 0.0f ? -tiny : tiny, 0.0f);
            const float2 f = df_mul(dl[i], df_rcp(d[i]));
            dl[i] = f;
            d[i + 1] = df_sub(d[i + 1], df_mul(f, du[i]));
          } else {
            piv[i] = 1;
            const float2 f = df_mul(d[i], df_rcp(dl[i]));
            d[i] = dl[i];
            dl[i] = f;
            const float2 tmp = du[i];
            du[i] = d[i + 1];
            d[i + 1] = df_sub(tmp, df_mul(f, d[i + 1]));
            if (i < m - 2) {
              du2[i] = du[i + 1];
              du[i + 1] = df_mul(make_float2(-f.x, -f.y), du[i + 1]);
            }
          }
        }
        if (fabsf(d[m - 1].x) < tiny) d[m - 1] = make_float2(d[m - 1].x < 0.0f ? -tiny : tiny, 0.0f);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = df_rcp(d[i]);
      for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = df_split(1.0 + 0.25 * rnd_sym(key + c, i));
      __syncthreads();
      for (int it = 0; it < 2; ++it) {
        if (threadIdx.x == 0) {
          for (int i = 0; i < m - 1; ++i) {
            if (piv[i]) {
              const float2 t = y[i];
              y[i] = y[i + 1];
              y[i + 1] = t;
            }
            y[i + 1] = df_sub(y[i + 1], df_mul(dl[i], y[i]));
          }
          y[m - 1] = df_mul(y[m - 1], d[m - 1]);
          if (m >= 2) y[m - 2] = df_mul(df_sub(y[m - 2], df_mul(du[m - 2], y[m - 1])), d[m - 2]);
          for (int i = m - 3; i >= 0; --i)
            y[i] = df_mul(df_sub(df_sub(y[i], df_mul(du[i], y[i + 1])), df_mul(du2[i], y[i + 2])), d[i]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) y64[i] = df_val(y[i]);
        __syncthreads();
        if (warp == 0) {
          double mx = 0.0;
          for (int i = lane; i < m; i += 32) mx = fmax(mx, fabs(y64[i]));
          for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (lane == 0) sh[0] = mx > 0.0 ? 1.0 / mx : 1.0;
        }
        __syncthreads();
        const double inv = sh[0];
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) y64[i] *= inv;
        __syncthreads();
        // orthogonalise against the cluster's earlier vectors (twice)
        const int nprev = c - c0;
        for (int pass = 0; pass < 2 && nprev > 0; ++pass) {
          for (int pb = 0; pb < nprev; pb += 1024) {
            const int cnt = nprev - pb < 1024 ? nprev - pb : 1024;
            for (int pi = warp; pi < cnt; pi += nwarp) {
              const double* yp = Y + (int64_t)(c0 + pb + pi) * ldy;
              double dot = 0.0;
              for (int i = lane; i < m; i += 32) dot = fma(yp[i], y64[i], dot);
              dot = warp_sum(dot);
              if (lane == 0) sdot[pi] = dot;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
              double sacc = 0.0;
              for (int pi = 0; pi < cnt; ++pi) sacc = fma(sdot[pi], Y[(int64_t)(c0 + pb + pi) * ldy + i], sacc);
              y64[i] -= sacc;
            }
            __syncthreads();
          }
        }
        double nn = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) nn = fma(y64[i], y64[i], nn);
        nn = block_sum(nn, sh);
        if (threadIdx.x == 0) s_inv = nn > 0.0 ? rsqrt64(nn) : 0.0;
        __syncthreads();
        const double inv2 = s_inv;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          y64[i] *= inv2;
          y[i] = df_split(y64[i]);
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) res[c] = fabs(beta_m * y64[m - 1]);
    for (int i = threadIdx.x; i < m; i += blockDim.x) Y[(int64_t)c * ldy + i] = y64[i];
    // theta_c = y^T T y (unit y, T unscaled): the eigenvalue to FP64
    // rounding (its error is quadratic in the vector's)
    double rq = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      rq = fma(y64[i], fma(a[i], y64[i], i + 1 < m ? 2.0 * b[i] * y64[i + 1] : 0.0), rq);
    rq = block_sum(rq, sh);
    if (threadIdx.x == 0) theta[c] = rq;
    __syncthreads();
  }
}


// U[n][c] = sum_j q_j[n] Y[c][j]: the Ritz vectors in the example space from
// the double-float Lanczos basis (rows q_j), in double-float, written in
// FP64.  Block (32, 4): 32 adjacent examples, the steps j in 4 interleaved
// slices (summed through shared memory at the end), 8 columns c; Y's 8 rows
// split into shared memory (8 m pairs).
constexpr int kRitzC = 8;
__global__ void ritz_df_kernel(const float2* Q, int64_t N, int m, const double* Y, int64_t ldy, int k, double* U) {
  extern __shared__ float2 ys[];  // kRitzC x m, then the slice sums
  const int c0 = blockIdx.y * kRitzC;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int e = tid; e < kRitzC * m; e += 128) {
    const int cc = e / m, j = e - cc * m;
    ys[e] = c0 + cc < k ? df_split(Y[(int64_t)(c0 + cc) * ldy + j]) : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  const int64_t n = blockIdx.x * (int64_t)32 + threadIdx.x;
  float s[kRitzC], c[kRitzC];
#pragma unroll
  for (int cc = 0; cc < kRitzC; ++cc) s[cc] = c[cc] = 0.0f;
  if (n < N) {
    // eight basis rows in flight per batch
    for (int j0 = threadIdx.y; j0 < m; j0 += 32) {
      float2 q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + 4 * u;
        q[u] = j < m ? Q[(int64_t)j * N + n] : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + 4 * u;
        if (j < m)
#pragma unroll
          for (int cc = 0; cc < kRitzC; ++cc) df_mac(q[u], ys[cc * m + j], s[cc], c[cc]);
      }
    }
  }
  float2* red = ys + kRitzC * m;  // 4 x kRitzC x 32
#pragma unroll
  for (int cc = 0; cc < kRitzC; ++cc) red[(threadIdx.y * kRitzC + cc) * 32 + threadIdx.x] = make_float2(s[cc], c[cc]);
  __syncthreads();
  if (threadIdx.y != 0 || n >= N) return;
#pragma unroll
  for (int cc = 0; cc < kRitzC; ++cc) {
    float2 v = df_norm(red[cc * 32 + threadIdx.x].x, red[cc * 32 + threadIdx.x].y);
    for (int y = 1; y < 4; ++y) {
      const float2 w = red[(y * kRitzC + cc) * 32 + threadIdx.x];
      v = df_add(v, df_norm(w.x, w.y));
    }
    if (c0 + cc < k) U[n * k + c0 + cc] = df_val(v);
  }
}

// A narrow weight layer's block of G^T U and its bias rows without forming G
// or B: R[j][i k + c] = sum_n a1[n][j] delta[n][i] u[n][c] with a1 = [a | 1]
// (j = Tin: the bias rows), in double-float.  Block (32, 8) for 32 columns
// (i, c) and up to kBpRows rows j, over the examples of its slice
// (blockIdx.z) in batches of 32 staged in shared memory; the slices' partial
// sums go to part[slice][j][col] for bp_small_reduce_kernel.
constexpr int kBpRows = 32;
__global__ void bp_small_kernel(const double* A, int Tin, const double* D, int Tout, const double* U, int k,
                                int64_t N, int64_t nper, float2* part) {
  __shared__ float2 sa[32][kBpRows + 1];
  __shared__ float2 sb[32][33];
  const int cols = Tout * k;
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int j0 = blockIdx.y * kBpRows;
  const int64_t nb = (int64_t)blockIdx.z * nper, ne = nb + nper < N ? nb + nper : N;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  float s[kBpRows / 8], c[kBpRows / 8];
#pragma unroll
  for (int t = 0; t < kBpRows / 8; ++t) s[t] = c[t] = 0.0f;
  for (int64_t b0 = nb; b0 < ne; b0 += 32) {
    for (int e = tid; e < 32 * kBpRows; e += 256) {
      const int nn = e / kBpRows, jj = e - nn * kBpRows;
      const int64_t n = b0 + nn;
      const int j = j0 + jj;
      double v = 0.0;
      if (n < ne && j <= Tin) v = j < Tin ? A[n * Tin + j] : 1.0;
      sa[nn][jj] = df_split(v);
    }
    for (int e = tid; e < 32 * 32; e += 256) {
      const int nn = e >> 5, cc = e & 31;
      const int64_t n = b0 + nn;
      const int cl = blockIdx.x * 32 + cc;
      double v = 0.0;
      if (n < ne && cl < cols) {
        const int i = cl / k, ci = cl - i * k;
        v = D[n * Tout + i] * U[n * k + ci];
      }
      sb[nn][cc] = df_split(v);
    }
    __syncthreads();
    const int nc = ne - b0 < 32 ? (int)(ne - b0) : 32;
    for (int nn = 0; nn < nc; ++nn) {
      const float2 b = sb[nn][threadIdx.x];
#pragma unroll
      for (int t = 0; t < kBpRows / 8; ++t) df_mac(sa[nn][threadIdx.y + 8 * t], b, s[t], c[t]);
    }
    __syncthreads();
  }
  if (col >= cols) return;
#pragma unroll
  for (int t = 0; t < kBpRows / 8; ++t) {
    const int j = j0 + threadIdx.y + 8 * t;
    if (j <= Tin) part[((int64_t)blockIdx.z * (Tin + 1) + j) * cols + col] = make_float2(s[t], c[t]);
  }
}

// R[j][col] (FP64) = the sum over the slices of part
__global__ void bp_small_reduce_kernel(const float2* part, int slices, int64_t rows_cols, double* R) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows_cols) return;
  float2 v = make_float2(0.0f, 0.0f);
#pragma unroll 8
  for (int z = 0; z < slices; ++z) {
    const float2 w = part[(int64_t)z * rows_cols + t];
    v = df_add(v, df_norm(w.x, w.y));
  }
  R[t] = df_val(v);
}

// The output pass over the k eigenvectors (P entries each), in slices of
// blockIdx.y: evals; null directions (mu <= 1e-13 mu_1) zeroed and flagged;
// the others scaled by 1/sqrt(N mu) (N = 0: left as they are); each slice
// reports its entry of largest magnitude (FP64 bits of |v|; 2 index + 1 if
// v < 0; ties to the smaller index) for the sign pass.
__global__ void finalize_scale_kernel(double* evecs, int64_t P, const double* theta, int k, double N,
                                      double* evals, int* deficient, unsigned long long* best) {
  __shared__ unsigned long long shv[32];
  __shared__ int64_t shi[32];
  const int c = blockIdx.x, S = gridDim.y, sl = blockIdx.y;
  const int64_t chunk = (P + S - 1) / S, i0 = sl * chunk, i1 = i0 + chunk < P ? i0 + chunk : P;
  const double mu = theta[c], mu0 = theta[0];
  double* q = evecs + (int64_t)c * P;
  const bool null_dir = !(mu > 1e-13 * mu0) || !(mu > 0.0);
  if (sl == 0 && threadIdx.x == 0) {
    evals[c] = mu;
    if (null_dir) atomicExch(deficient, 1);
  }
  unsigned long long bv = 0ull;
  int64_t bi = i0;
  bool neg = false;
  if (null_dir) {
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) q[i] = 0.0;
  } else {
    const double sc = N > 0.0 ? 1.0 / sqrt(N * mu) : 1.0;
#pragma unroll 4
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double v = q[i] * sc;
      q[i] = v;
      const unsigned long long a = (unsigned long long)__double_as_longlong(fabs(v));
      if (a > bv) {
        bv = a;
        bi = i;
        neg = v < 0.0;
      }
    }
  }
  int64_t bx = 2 * bi + (neg ? 1 : 0);  // index and sign
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int64_t ox = __shfl_xor_sync(0xffffffffu, bx, o);
    if (ov > bv || (ov == bv && (ox >> 1) < (bx >> 1))) {
      bv = ov;
      bx = ox;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    shv[threadIdx.x >> 5] = bv;
    shi[threadIdx.x >> 5] = bx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bv = shv[0];
    bx = shi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (shv[w] > bv || (shv[w] == bv && (shi[w] >> 1) < (bx >> 1))) {
        bv = shv[w];
        bx = shi[w];
      }
    best[((int64_t)c * S + sl) * 2] = bv;
    best[((int64_t)c * S + sl) * 2 + 1] = (unsigned long long)bx;
  }
}

// The sign pass: each slice finds its vector's entry of largest magnitude
// from the slices' reports (not from the vector, which other slices may be
// negating) and negates its own entries when that entry is negative.
__global__ void finalize_sign_kernel(double* evecs, int64_t P, const unsigned long long* best) {
  const int c = blockIdx.x, S = gridDim.y, sl = blockIdx.y;
  const int64_t chunk = (P + S - 1) / S, i0 = sl * chunk, i1 = i0 + chunk < P ? i0 + chunk : P;
  unsigned long long bv = 0ull;
  int64_t bx = 2 * P;
  for (int z = 0; z < S; ++z) {
    const unsigned long long v = best[((int64_t)c * S + z) * 2];
    const int64_t x = (int64_t)best[((int64_t)c * S + z) * 2 + 1];
    if (v > bv || (v == bv && (x >> 1) < (bx >> 1))) {
      bv = v;
      bx = x;
    }
  }
  if (!(bx & 1)) return;
  double* q = evecs + (int64_t)c * P;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) q[i] = -q[i];
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

// Dynamic shared memory the eigen kernels may use (their attribute is set
// once to this, so that concurrent calls with different sizes do not race).
constexpr size_t kEigSmemCap = (size_t)208 << 10;

hess_status eig_kernel_attributes() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(lanczos_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bisect_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(inviter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lanczos_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(inviter_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ritz_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemCap);
  });
  if (e != cudaSuccess) return set_error(HESS_ERR_CUDA, "eigen kernel attributes: %s", cudaGetErrorString(e));
  return HESS_OK;
}

// The output pass (finalize_scale_kernel, then finalize_sign_kernel) over
// slices of about 2048 entries; best holds 2 k finalize_slices(P) words.
int finalize_slices(int64_t P) {
  const int64_t S = cdiv(P, 2048);
  return (int)(S < 1 ? 1 : (S > 64 ? 64 : S));
}
hess_status finalize_vectors(double* evecs, int64_t P, const double* theta, int k, double N, double* evals,
                             int* deficient, unsigned long long* best, cudaStream_t s) {
  const dim3 grid((unsigned)k, (unsigned)finalize_slices(P));
  finalize_scale_kernel<<<grid, 256, 0, s>>>(evecs, P, theta, k, N, evals, deficient, best);
  HM_LAUNCHED();
  finalize_sign_kernel<<<grid, 256, 0, s>>>(evecs, P, best);
  HM_LAUNCHED();
  return HESS_OK;
}

int64_t tridiag_scratch_doubles(int64_t mcap, int k) {
  const bool need = (size_t)6 * mcap * sizeof(double) > kEigSmemCap;
  return need ? (int64_t)k * 6 * (mcap + 1) : 0;
}

hess_status tridiag_topk(const double* a, const double* b, int m, int k, double* theta, int* cstart, double* Y,
                         int64_t ldy, const double* beta_last, double* res, double* mx, uint64_t key,
                         double* scratch, cudaStream_t s) {
  HM_TRY(eig_kernel_attributes());
  const bool inv_g = (size_t)6 * m * sizeof(double) > kEigSmemCap;
  const bool bis_g = (size_t)3 * m * sizeof(double) > kEigSmemCap;
  if ((inv_g || bis_g) && !scratch) return set_error(HESS_ERR_INVALID_ARG, "tridiagonal scratch missing");
  // a cluster of CTAs per eigenvalue (T in each CTA's shared memory), or,
  // when T does not fit shared memory, one block per eigenvalue over global
  // scratch
  if (!bis_g) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kBisCta * k));
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = (size_t)3 * m * sizeof(double);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kBisCta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HM_CUDA(cudaLaunchKernelEx(&cfg, bisect_cluster_kernel, a, b, m, k, theta));
  } else {
    bisect_kernel<<<(unsigned)k, 128, 0, s>>>(a, b, m, k, theta, scratch);
  }
  HM_LAUNCHED();
  // eigenvalues closer than 1e-6 of the largest share a cluster
  clusters_kernel<<<1, 32, 0, s>>>(theta, k, 1e-6, cstart);
  HM_LAUNCHED();
  if ((size_t)7 * m * sizeof(double) <= kEigSmemCap) {
    inviter_df_kernel<<<k, 256, (size_t)7 * m * sizeof(double), s>>>(a, b, m, k, theta, cstart, Y, ldy, beta_last,
                                                                     res, key);
    HM_LAUNCHED();
    max_res_kernel<<<1, 32, 0, s>>>(res, k, theta, mx);
    HM_LAUNCHED();
    return HESS_OK;
  }
  inviter_kernel<<<k, 256, inv_g ? 0 : (size_t)6 * m * sizeof(double), s>>>(a, b, m, k, theta, cstart, Y, ldy,
                                                                           beta_last, res, key,
                                                                           inv_g ? scratch : nullptr);
  HM_LAUNCHED();
  max_res_kernel<<<1, 32, 0, s>>>(res, k, theta, mx);
  HM_LAUNCHED();
  return HESS_OK;
}

// Lanczos buffers of an n x n symmetric problem (Q and MQ: mcap x n; given
// by the caller to reuse its memory, or taken from the arena).
struct LzBufs {
  int64_t n = 0, mcap = 0;
  double *Q = nullptr, *MQ = nullptr, *w = nullptr, *wt = nullptr, *dpart = nullptr, *npart = nullptr,
         *apart = nullptr, *h1 = nullptr, *h2 = nullptr, *alpha = nullptr, *beta = nullptr, *theta = nullptr,
         *Y = nullptr, *rr = nullptr, *mx = nullptr, *tri_scratch = nullptr;
  unsigned* bar = nullptr;
  int *err = nullptr, *cstart = nullptr, *stop = nullptr;
  // double-float kernel: block partials and the scale exponent of M
  float2 *dfapart = nullptr, *dfh = nullptr, *dfg = nullptr;
  int* escale = nullptr;
};

void plan_lz(Arena& ar, int64_t n, int k, LzBufs& b, double* Q, double* MQ) {
  b.n = n;
  b.mcap = n < (int64_t)8 * k + 512 ? n : (int64_t)8 * k + 512;
  const int64_t mcap = b.mcap;
  b.Q = Q ? Q : ar.take<double>((mcap + 1) * n);  // (the double-float kernel's q~ row)
  b.MQ = MQ ? MQ : ar.take<double>(mcap * n);
  b.w = ar.take<double>(n);
  b.wt = ar.take<double>(n);
  b.dpart = ar.take<double>((mcap + 1) * 8);
  b.npart = ar.take<double>(4096);
  b.apart = ar.take<double>(4096);
  b.h1 = ar.take<double>(mcap + 1);
  b.h2 = ar.take<double>(mcap + 1);
  b.alpha = ar.take<double>(mcap + 1);
  b.beta = ar.take<double>(mcap + 1);
  b.theta = ar.take<double>(k);
  b.Y = ar.take<double>((int64_t)k * mcap);
  b.bar = ar.take<unsigned>(64);
  b.err = ar.take<int>(1);
  b.cstart = ar.take<int>(k);
  b.rr = ar.take<double>(k);
  b.mx = ar.take<double>(2);
  b.stop = ar.take<int>(1);
  // global scratch of the tridiagonal kernels when shared memory is too small
  const int64_t tri_n = tridiag_scratch_doubles(mcap, k);
  b.tri_scratch = tri_n ? ar.take<double>(tri_n) : nullptr;
  b.dfapart = ar.take<float2>((int64_t)kDfMaxGrid * 4);
  b.dfh = ar.take<float2>((mcap + 2) * kDfMaxChunks);
  b.dfg = ar.take<float2>((mcap + 2) * kDfMaxChunks);
  b.escale = ar.take<int>(1);
}

// Shared memory of the double-float kernel for grid g on an n x n matrix with
// slices of q_0 .. q_{m1} and M q_0 .. M q_{m1}.
size_t df_smem(int64_t n, int64_t g, int64_t mcap, int64_t m1) {
  (void)mcap;
  const int64_t E = cdiv(n, g), qcap = m1 + 1;
  const int64_t f2 = E * n + n + 2 * E * qcap + 2 * E + 5 * (qcap + 1) + kDfRed;
  return (size_t)f2 * sizeof(float2);
}

// Grid of the double-float kernel for an n x n matrix: the handle's
// lz_blocks when set, else 8/15 of the SMs (the kernel waits on its grid
// barriers far more than it computes, so a grid smaller than the GPU costs
// it little, and the SMs left over run the contractions of the fused call
// beside it: for 1024 examples on 152 SMs, 79 blocks of 13 rows balance the
// two chains better than 86 blocks of 12); 0 when the kernel does not apply
// (n above its chunk table, or the owned rows and slices exceed shared
// memory even with a block on every SM).
int df_grid(hess_mlp* h, int64_t n, int64_t mcap) {
  const int gmax = h->sm_count < kDfMaxGrid ? h->sm_count : kDfMaxGrid;
  if (gmax < 1 || n > (int64_t)kDfChunk * kDfMaxChunks || df_smem(n, gmax, mcap, mcap) > kEigSmemCap) return 0;
  int g = h->lz_blocks > 0 ? h->lz_blocks : (h->sm_count * 8) / 15;
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  if (n < g) g = (int)n;
  return g;
}

int eig_lanczos_blocks(hess_mlp* h, int64_t n, int k) {
  const int64_t mcap = n < (int64_t)8 * k + 512 ? n : (int64_t)8 * k + 512;
  const int g = df_grid(h, n, mcap);
  if (g <= 0) return h->sm_count;  // the FP64 kernel: a block on every SM
  return (int)cdiv(n, cdiv(n, g));
}

// The Lanczos process of run_lz with the double-float kernel.  M is the
// n x n matrix as scaled hi/lo pairs (m_split; otherwise FP64, overwritten by
// its pairs here), q_0 is in row 0 of b.Q already when q0_ready.  On return
// b.Q holds q_0 .. q_{m-1} as hi/lo pairs (rows of n) and b.theta, b.Y the
// top-k eigenpairs of T_m.  Optional hooks: after_launch runs once, right
// after the first Lanczos launch is queued (host work that the launch then
// hides); spec(m) runs as soon as the tridiagonal eigenpairs of T_m are
// queued, before the host reads the convergence flags, and *spec_m receives
// the m of the last such call whose eigenpairs stand (-1 if none: the
// caller repeats its work for the final m); theta_host (k doubles of pinned
// memory) receives the Ritz values with the flags.
constexpr uint64_t kLzKey = 0x5DEECE66Dull;  // the start vector's counter-based draw

hess_status run_lz_df(hess_mlp* h, double* M, int k, LzBufs& b, int grid, int* m_out, bool* converged_out,
                      bool m_split, bool q0_ready, const std::function<hess_status(int)>* spec, int* spec_m,
                      const std::function<hess_status()>* after_launch, double* theta_host) {
  if (spec_m) *spec_m = -1;
  const int64_t N = b.n, mcap = b.mcap;
  cudaStream_t s = h->stream;
  const uint64_t key = kLzKey;
  float2* Q = reinterpret_cast<float2*>(b.Q);
  float2* MQ = reinterpret_cast<float2*>(b.MQ);
  const int max_grid = h->sm_count < kDfMaxGrid ? h->sm_count : kDfMaxGrid;
  HM_TRY(eig_kernel_attributes());
  {
    // (preparation of M and the start vector: counted with the Gram matrix)
    Tick t(h, HESS_K_GRAM, 0.0, 0.0);
    if (!m_split) {
      df_scale_kernel<<<1, 1024, 0, s>>>(M, N, b.escale);
      HM_LAUNCHED();
      const int64_t n2 = N * N;
      df_split_kernel<<<(unsigned)(cdiv(n2, 256) < 4096 ? cdiv(n2, 256) : 4096), 256, 0, s>>>(M, n2, b.escale);
      HM_LAUNCHED();
    }
    if (!q0_ready) {
      df_start_kernel<<<1, 1024, 0, s>>>(Q, N, key);
      HM_LAUNCHED();
    }
  }
  HM_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), s));
  int m = 0;
  int64_t target = N < (int64_t)3 * k + 32 ? N : (int64_t)3 * k + 32;
  if (target < k) target = k;
  if (target > mcap) target = mcap;
  bool converged = false;
  double* hp = h->host_pinned;
  const long long lim = g_bar_limit.load();
  while (true) {
    DfArgs a;
    a.M = reinterpret_cast<const float2*>(M);
    a.N = N;
    a.Q = Q;
    a.MQ = MQ;
    a.hc = b.dfh;
    a.hg = b.dfg;
    a.apart = b.dfapart;
    a.alpha = b.alpha;
    a.beta = b.beta;
    a.escale = b.escale;
    a.bar = b.bar;
    a.err = b.err;
    a.stop = b.stop;
    a.m0 = m;
    a.m1 = (int)target;
    a.mcap = (int)mcap;
    a.qcap = (int)target + 1;
    a.nch = (int)cdiv(N, kDfChunk);
    a.bar_limit = lim > 0 ? lim : BAR_TIMEOUT;
    // this launch's grid: the requested one, or more blocks when the slices
    // of q_0 .. q_target do not fit shared memory (the eligibility check
    // guarantees that the most blocks fit)
    int gl = grid;
    while (gl < max_grid && df_smem(N, gl, mcap, target) > kEigSmemCap) ++gl;
    gl = (int)cdiv(N, cdiv(N, gl));
    a.E = (int)cdiv(N, gl);
    const size_t dyn = df_smem(N, gl, mcap, target);
    void* kargs[] = {&a};
    HM_CUDA(cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), s));
    HM_CUDA(cudaMemsetAsync(b.stop, 0xff, sizeof(int), s));
    {
      double fl = 0.0;
      for (int64_t j = m; j < target; ++j) fl += 2.0 * N * N + 8.0 * N * (j + 1);
      Tick t(h, HESS_K_LANCZOS, fl, 0.0);
      HM_CUDA(cudaLaunchCooperativeKernel((void*)lanczos_df_kernel, gl, kDfThreads, kargs, dyn, s));
      HM_LAUNCHED();
    }
    // the caller's host work that may overlap the first launch
    if (after_launch) {
      HM_TRY((*after_launch)());
      after_launch = nullptr;
    }
    // the tridiagonal eigenpairs of T_target are queued at once and read
    // with the kernel's flags (one host round trip); after a breakdown or a
    // failed barrier they are discarded
    {
      Tick t(h, HESS_K_TRIDIAG, 0.0, 0.0);
      HM_TRY(tridiag_topk(b.alpha, b.beta, target, k, b.theta, b.cstart, b.Y, mcap, b.beta + (target - 1), b.rr,
                          b.mx, key + 11, b.tri_scratch, s));
    }
    // the caller's work on the eigenpairs of T_target, queued before the
    // flags are read (kept if they show convergence at target)
    if (spec) {
      HM_TRY((*spec)((int)target));
      *spec_m = (int)target;
    }
    HM_CUDA(cudaMemcpyAsync(hp, b.mx, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(hp + 2), b.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(hp + 2) + 1, b.stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    // (the Ritz values with them, for the caller's checks)
    if (theta_host) HM_CUDA(cudaMemcpyAsync(theta_host, b.theta, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (*reinterpret_cast<int*>(hp + 2)) return set_error(HESS_ERR_TIMEOUT, "Lanczos grid barrier gave up");
    const int stopped = reinterpret_cast<int*>(hp + 2)[1];
    if (stopped >= 0) {
      // breakdown: beta_{stopped-1} = 0 is stored and T_stopped is complete;
      // a new direction orthogonal to the basis continues it (none exists
      // once the basis spans the whole space)
      m = stopped;
      if (m >= N) {
        converged = true;
        break;
      }
      if (m < mcap) {
        Tick t(h, HESS_K_TRIDIAG, 0.0, 0.0);
        df_restart_kernel<<<1, 1024, (size_t)(N + m) * sizeof(double), s>>>(Q, N, m, key + 7);
        HM_LAUNCHED();
        continue;
      }
    } else {
      m = (int)target;
    }
    if (stopped >= 0) {
      // (reached only when the basis cannot grow: m == mcap) the eigenpairs
      // of the complete T_m
      if (spec_m) *spec_m = -1;
      Tick t(h, HESS_K_TRIDIAG, 0.0, 0.0);
      HM_TRY(tridiag_topk(b.alpha, b.beta, m, k, b.theta, b.cstart, b.Y, mcap, b.beta + (m - 1), b.rr, b.mx,
                          key + 11, b.tri_scratch, s));
      HM_CUDA(cudaMemcpyAsync(hp, b.mx, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      HM_CUDA(cudaStreamSynchronize(s));
    }
    if (hp[0] <= 1e-10 * hp[1] || m >= N) {
      converged = true;
      break;
    }
    if (m >= mcap) break;
    int64_t step = k > 32 ? k : 32;
    target = m + step;
    if (target > mcap) target = mcap;
    if (target > N) target = N;
  }
  if (converged && m >= N) {
    // the tridiagonal eigenpairs of the complete T (after a final breakdown)
    if (spec_m) *spec_m = -1;
    Tick t(h, HESS_K_TRIDIAG, 0.0, 0.0);
    HM_TRY(tridiag_topk(b.alpha, b.beta, m, k, b.theta, b.cstart, b.Y, mcap, b.beta + (m - 1), b.rr, b.mx,
                        key + 11, b.tri_scratch, s));
  }
  *m_out = m;
  *converged_out = converged;
  return HESS_OK;
}

// Steps 2-3 on the resident n x n matrix M: Lanczos with full
// reorthogonalisation, extended until the top-k residual bounds converge;
// on return b.theta and b.Y hold the top-k Ritz values and the eigenvectors
// of T_m (rows of Y, stride mcap), *m_out the Krylov dimension.
hess_status run_lz(hess_mlp* h, const double* M, int k, LzBufs& b, int* m_out, bool* converged_out) {
  const int64_t N = b.n, mcap = b.mcap;
  double *Q = b.Q, *MQ = b.MQ, *w = b.w, *wt = b.wt, *dpart = b.dpart, *npart = b.npart, *apart = b.apart,
         *h1 = b.h1, *h2 = b.h2, *alpha = b.alpha, *beta = b.beta, *theta = b.theta, *Y = b.Y, *rr = b.rr,
         *mx = b.mx, *tri_scratch = b.tri_scratch;
  unsigned* bar = b.bar;
  int *err = b.err, *cstart = b.cstart, *stop = b.stop;
  cudaStream_t s = h->stream;
  const uint64_t key = 0x5DEECE66Dull;
  // ownership: E entries per block over at most one block per SM; shared
  // memory holds the coefficients and the owned slices, then, as far as they
  // fit, w, the owned rows of M and the owned slice of Q
  const int64_t E = cdiv(N, h->sm_count);
  const int grid = (int)cdiv(N, E);
  const size_t cap = kEigSmemCap;
  size_t dyn = ((size_t)(mcap + 1) + 3 * (size_t)E) * sizeof(double);
  int cache_w = 0, cache_m = 0, cache_q = 0;
  if (dyn + (size_t)N * 8 <= cap) {
    cache_w = 1;
    dyn += (size_t)N * 8;
  }
  if (cache_w && dyn + (size_t)E * N * 8 <= cap) {
    cache_m = 1;
    dyn += (size_t)E * N * 8;
  }
  if (dyn + (size_t)mcap * E * 8 <= cap) {
    cache_q = 1;
    dyn += (size_t)mcap * E * 8;
  }
  if (dyn > cap) return set_error(HESS_ERR_UNSUPPORTED, "Lanczos workspace exceeds shared memory (N = %lld)",
                                  (long long)N);
  int per_sm = 0;
  HM_TRY(eig_kernel_attributes());
  HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_coop_kernel, 512, dyn));
  if (per_sm < 1 || grid > per_sm * h->sm_count) return set_error(HESS_ERR_CUDA, "Lanczos kernel cannot be resident");
  init_start_kernel<<<1, 1024, 0, s>>>(w, npart, grid, N, key);
  HM_LAUNCHED();
  HM_CUDA(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), s));
  HM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  const int nchunk = (int)(N < 1024 ? cdiv(N, 128) : 8);
  int m = 0;
  int64_t target = N < (int64_t)3 * k + 32 ? N : (int64_t)3 * k + 32;
  if (target < k) target = k;
  if (target > mcap) target = mcap;
  bool converged = false;
  double* hp = h->host_pinned;
  int resumed = 0;
  while (true) {
    LzArgs la;
    la.M = M;
    la.N = N;
    la.Q = Q;
    la.MQ = MQ;
    la.w = w;
    la.wt = wt;
    la.h = h1;
    la.dpart = dpart;
    la.npart = npart;
    la.apart = apart;
    la.alpha = alpha;
    la.beta = beta;
    la.bar = bar;
    la.err = err;
    la.m0 = m;
    la.m1 = (int)target;
    la.mcap = (int)mcap;
    la.nchunk = nchunk < 1 ? 1 : nchunk;
    la.E = (int)E;
    la.cache_m = cache_m;
    la.cache_q = cache_q;
    la.cache_w = cache_w;
    la.stop = stop;
    la.resumed = resumed;
    la.key = key + 7;
    {
      const long long lim = g_bar_limit.load();
      la.bar_limit = lim > 0 ? lim : BAR_TIMEOUT;
    }
    void* kargs[] = {&la};
    HM_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    HM_CUDA(cudaMemsetAsync(stop, 0xff, sizeof(int), s));
    {
      double fl = 0.0;
      for (int64_t j = m; j < target; ++j) fl += 2.0 * N * N + 8.0 * N * (j + 1);
      Tick t(h, HESS_K_LANCZOS, fl, 0.0);
      HM_CUDA(cudaLaunchCooperativeKernel((void*)lanczos_coop_kernel, grid, 512, kargs, dyn, s));
      HM_LAUNCHED();
    }
    m = (int)target;
    {
      Tick t(h, HESS_K_TRIDIAG, 0.0, 0.0);
      last_beta_kernel<<<1, 32, 0, s>>>(npart, grid, h2);
      HM_LAUNCHED();
      HM_TRY(tridiag_topk(alpha, beta, m, k, theta, cstart, Y, mcap, h2, rr, mx, key + 11, tri_scratch, s));
    }
    HM_CUDA(cudaMemcpyAsync(hp, mx, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(hp + 2), err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(hp + 2) + 1, stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (*reinterpret_cast<int*>(hp + 2))
      return set_error(HESS_ERR_TIMEOUT, "Lanczos grid barrier gave up");
    const int stopped = reinterpret_cast<int*>(hp + 2)[1];
    resumed = 0;
    if (stopped >= 0) {
      // breakdown at step `stopped` (the eigen pass above saw an incomplete
      // T and is discarded): a random vector orthogonalised twice against
      // q_0..q_{stopped-1}, then resume there
      m = stopped;
      const unsigned gb = (unsigned)(cdiv(N, 256) < 4096 ? cdiv(N, 256) : 4096);
      restart_fill_kernel<<<gb, 256, 0, s>>>(w, N, key + 7, m, beta);
      HM_LAUNCHED();
      for (int pass = 0; pass < 2; ++pass) {
        restart_coef_kernel<<<(unsigned)cdiv(m, 8), 256, 0, s>>>(Q, w, N, m, h1);
        HM_LAUNCHED();
        restart_sub_kernel<<<gb, 256, 0, s>>>(Q, h1, N, m, w);
        HM_LAUNCHED();
      }
      restart_norm_kernel<<<1, 1024, 0, s>>>(w, N, npart, grid);
      HM_LAUNCHED();
      resumed = 1;
      continue;
    }
    if (hp[0] <= 1e-10 * hp[1] || m >= N) {
      converged = true;
      break;
    }
    if (m >= mcap) break;
    int64_t step = k > 32 ? k : 32;
    target = m + step;
    if (target > mcap) target = mcap;
    if (target > N) target = N;
  }
  *m_out = m;
  *converged_out = converged;
  return HESS_OK;
}

hess_status topk_eig_gram(hess_mlp* h, const Net& net, const Caches<double>& c, int64_t N, int k,
                          double* evals_d, double* evecs_d, Arena& ar, bool dry, EigResult* res,
                          const std::function<hess_status()>* after_gram, const EigSide* side) {
  const int64_t P = net.P;
  const int L = net.L;
  double* M = ar.take<double>(N * N);
  double* DD = ar.take<double>(N * N);
  double* AA = ar.take<double>(N * N);
  LzBufs lb;
  // M Q reuses DD once the Gram matrix is formed, and so does the basis AA
  // unless the double-float kernel runs (its start vector is formed with
  // the Gram matrix, while AA may still hold a partial product)
  const int64_t mcap0 = N < (int64_t)8 * k + 512 ? N : (int64_t)8 * k + 512;
  const int dfg = df_grid(h, N, mcap0);
  plan_lz(ar, N, k, lb, dfg > 0 ? nullptr : AA, DD);
  const int64_t mcap = lb.mcap;
  double* U = ar.take<double>(N * k);
  int* flag = ar.take<int>(2);
  double* theta = lb.theta;
  double* Y = lb.Y;
  double* Q = lb.Q;
  double* hp = h->host_pinned;
  // wide layer inputs (A A^T over K = T_in >= 128) go to the tensor cores as
  // exact-digit FP64 products
  int64_t ktc = 0;
  for (int wl = 1; wl <= L - 1; ++wl)
    if (f64_syrk_tc_eligible(h, N, net.T[wl - 1]) && net.T[wl - 1] > ktc) ktc = net.T[wl - 1];
  F64SyrkScratch fs;
  if (ktc) plan_f64_syrk(ar, N, ktc, fs);
  // the Gram kernels' split rows and per-row exponents
  GramPrepArgs gp{};
  gp.nl = L - 1;
  gp.N = N;
  gp.invN = 1.0 / (double)N;
  for (int wl = 1; wl <= L - 1; ++wl) {
    const int Tin = net.T[wl - 1], Tout = net.T[wl];
    const bool wide = ktc && Tin >= 128 && Tin <= ktc;
    GramPrepLayer& pl = gp.l[wl - 1];
    pl.D = c.d[wl];
    pl.A = c.a[wl - 1];
    pl.Tout = Tout;
    pl.Tin = Tin;
    pl.XD = ar.take<float2>(N * Tout);
    pl.XA = wide ? nullptr : ar.take<float2>(N * Tin);
    pl.pD = ar.take<int>(N);
    pl.pA = ar.take<int>(N);
    pl.eA = ar.take<int>(N);
  }
  gp.r = ar.take<int>(N);
  gp.maxdiag = ar.take<unsigned long long>(1);
  gp.q0 = dfg > 0 ? reinterpret_cast<float2*>(lb.Q) : nullptr;
  gp.key = kLzKey;
  // and so does the back-projection G^T U (K = N)
  // and so do the back-projection's wide layers: per weight layer,
  // R = A^T B with B[n][(i, c)] = delta[n][i] u[n][c] (K = N)
  // (mode 1: rows of A^T against B in column groups; mode 2, for narrow
  // layers: rows of B^T against A, the transposed product; mode 0: the SIMT
  // FP64 GEMM, for products too small to repay the digit splitting)
  int64_t cols_max = 0, r_max = 0, tout_max = 0;
  F64GemmNeed need;
  int bp_mode[kMaxLayers] = {};
  for (int wl = 1; wl <= L - 1; ++wl) {
    const int64_t Tin = net.T[wl - 1], Tout = net.T[wl], cols = Tout * k;
    const int64_t gw = cols < 256 ? cols : 256;
    cols_max = cols > cols_max ? cols : cols_max;
    r_max = (Tin + 1) * cols > r_max ? (Tin + 1) * cols : r_max;
    tout_max = Tout > tout_max ? Tout : tout_max;
    if (2.0 * N * Tin * cols < 5e7) continue;
    if (f64_gemm_nt_tc_eligible(h, Tin + 1, gw, N, cols)) {
      bp_mode[wl] = 1;
      f64_gemm_nt_need(Tin + 1, gw, N, cols, need);
    } else if (Tin <= 256 && f64_gemm_nt_tc_eligible(h, cols, Tin, N)) {
      bp_mode[wl] = 2;
      f64_gemm_nt_need(cols, Tin, N, Tin, need);
    }
  }
  double* Bf = ar.take<double>(N * cols_max);
  double* Rf = ar.take<double>(r_max);
  double* Rb = ar.take<double>(tout_max * k);
  // the narrow layers' slices of examples (bp_small_kernel)
  const int64_t bp_nper = 64, bp_slices = cdiv(N, bp_nper);
  int64_t part_max = 0;
  for (int wl = 1; wl <= L - 1; ++wl)
    if (!bp_mode[wl]) part_max = std::max<int64_t>(part_max, (int64_t)(net.T[wl - 1] + 1) * net.T[wl] * k);
  float2* bp_part = ar.take<float2>(bp_slices * part_max);
  unsigned long long* best = ar.take<unsigned long long>((int64_t)2 * k * finalize_slices(P));
  F64GemmScratch fb;
  if (need.M) plan_f64_gemm_nt(ar, need, fb);
  // the narrow layers' R when they run on the side stream
  int64_t rs_max = 1;
  for (int wl = 1; wl <= L - 1; ++wl)
    if (!bp_mode[wl]) rs_max = std::max<int64_t>(rs_max, (int64_t)(net.T[wl - 1] + 1) * net.T[wl] * k);
  double* Rs = ar.take<double>(rs_max);
  if (dry) return HESS_OK;
  cudaStream_t s = h->stream;
  // the activations' digit split of the back-projection ahead of time, on
  // the side stream, when exactly one layer's product uses the digit scratch
  int a_pre = 0;
  if (side && side->s) {
    int users = 0;
    for (int wl = 1; wl <= L - 1; ++wl)
      if (bp_mode[wl]) {
        ++users;
        if (bp_mode[wl] == 1) a_pre = wl;
      }
    if (users != 1) a_pre = 0;
    HM_CUDA(cudaEventRecord(side->ev[0], s));  // (the forward pass is done)
  }

  // 1. Gram matrix, factored by layer: the wide layers' activation products
  // as exact-digit tensor-core planes, everything else in double-float in
  // fused launches (one per wide layer), written as the Lanczos kernel's
  // double-float input when that kernel runs
  {
    Tick t(h, HESS_K_GRAM, 0.0, 0.0);
    HM_CUDA(cudaMemsetAsync(gp.maxdiag, 0, sizeof(unsigned long long), s));
    gram_prep_kernel<<<(unsigned)(cdiv(N, 8) + (gp.q0 ? 1 : 0)), 256, 0, s>>>(gp);
    HM_LAUNCHED();
  }
  {
    GramArgs ga{};
    ga.N = N;
    ga.invN = 1.0 / (double)N;
    ga.r = gp.r;
    ga.maxdiag = gp.maxdiag;
    ga.df_out = dfg > 0 ? 1 : 0;
    ga.escale = lb.escale;
    double fl = 0.0;
    int launches = 0;
    auto flush = [&]() -> hess_status {
      Tick t(h, HESS_K_GRAM, fl, 0.0);
      ga.accumulate = launches > 0 ? 1 : 0;
      const unsigned nb = (unsigned)cdiv(N, kGt);
      gram_fused_kernel<<<dim3(nb, nb), 256, 0, s>>>(ga, M);
      HM_LAUNCHED();
      ++launches;
      ga.nl = 0;
      ga.pl = F64SyrkPlanes{};
      fl = 0.0;
      return HESS_OK;
    };
    for (int wl = 1; wl <= L - 1; ++wl) {
      const GramPrepLayer& pl = gp.l[wl - 1];
      const bool wide = pl.XA == nullptr;
      GramLayer gl{pl.XD, pl.XA, pl.pD, pl.pA, pl.eA, pl.Tout, pl.Tin};
      fl += (double)N * (N + 1) * (pl.Tout + (wide ? 0 : pl.Tin));
      if (wide) {
        if (ga.pl.T) HM_TRY(flush());
        HM_TRY(f64_syrk_tc(h, c.a[wl - 1], pl.Tin, pl.Tin, AA, N, fs, s, &ga.pl));
        if (!ga.pl.T) return set_error(HESS_ERR_UNSUPPORTED, "exact-digit Gram term: no planes left to combine");
      }
      ga.l[ga.nl++] = gl;
    }
    HM_TRY(flush());
  }
  if (side && side->gram_done) HM_CUDA(cudaEventRecord(side->gram_done, s));
  // the caller's hook and the side stream's digit split, once the first
  // Lanczos launch is queued
  const std::function<hess_status()> post_launch = [&]() -> hess_status {
    if (after_gram) HM_TRY((*after_gram)());
    if (a_pre) {
      // (on the side stream, behind its earlier work)
      const int64_t Tin = net.T[a_pre - 1], cols = net.T[a_pre] * (int64_t)k;
      F64GemmScratch f2 = fb;
      f2.M = Tin + 1;
      f2.Nn = cols < 256 ? cols : 256;
      HM_CUDA(cudaStreamWaitEvent(side->s, side->ev[0], 0));
      HM_TRY(f64_gemm_nt_split_a(c.a[a_pre - 1], Tin, N, f2, side->s, Tin));
      HM_CUDA(cudaEventRecord(side->ev[3], side->s));
    }
    return HESS_OK;
  };

  // 4. from the eigenpairs of T_m: Ritz vectors U = Q_m^T Y (N x k), the
  // back-projection through G, the scaling and signs (queued by the
  // double-float route as soon as the tridiagonal eigenpairs are, before
  // their convergence is known, and again if they are replaced)
  const bool narrow_side = side && side->s;
  auto tail = [&](int m) -> hess_status {
    if (dfg > 0) {
      Tick t(h, HESS_K_BACKPROJ, 2.0 * N * m * k, 0.0);
      const size_t sm = (size_t)kRitzC * m * sizeof(float2) + (size_t)4 * kRitzC * 32 * sizeof(float2);
      ritz_df_kernel<<<dim3((unsigned)cdiv(N, 32), (unsigned)cdiv(k, kRitzC)), dim3(32, 4), sm, s>>>(
          reinterpret_cast<const float2*>(Q), N, m, Y, mcap, k, U);
      HM_LAUNCHED();
    } else {
      Tick t(h, HESS_K_BACKPROJ, 2.0 * N * m * k, 0.0);
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
    if (narrow_side) {
      HM_CUDA(cudaEventRecord(side->ev[1], s));
      HM_CUDA(cudaStreamWaitEvent(side->s, side->ev[1], 0));
    }
    // q_c = G^T u_c without forming G: the block of weight layer w is
    // R[j][(i, c)] = sum_n a[n][j] (delta[n][i] u[n][c]), its bias rows
    // sum_n delta[n][i] u[n][c] (Eq. J with g_n = [delta_n (x) a_n; delta_n])
    for (int wl = 1; wl <= L - 1; ++wl) {
      const int64_t Tin = net.T[wl - 1], Tout = net.T[wl], cols = Tout * k;
      if (!bp_mode[wl]) {
        // R and its bias row Tin in one pass, without forming B (on the
        // side stream, into its own R, beside the wide layers)
        Tick t(narrow_side ? nullptr : h, HESS_K_BACKPROJ, 2.0 * N * (Tin + 1) * cols, 0.0);
        const cudaStream_t sl = narrow_side ? side->s : s;
        double* R = narrow_side ? Rs : Rf;
        const dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(Tin + 1, kBpRows), (unsigned)bp_slices);
        bp_small_kernel<<<grid, dim3(32, 8), 0, sl>>>(c.a[wl - 1], (int)Tin, c.d[wl], (int)Tout, U, k, N, bp_nper,
                                                      bp_part);
        HM_LAUNCHED();
        const int64_t rc = (Tin + 1) * cols;
        bp_small_reduce_kernel<<<(unsigned)cdiv(rc, 256), 256, 0, sl>>>(bp_part, (int)bp_slices, rc, R);
        HM_LAUNCHED();
        const int64_t per = (Tin + 1) * Tout;
        bp_scatter_kernel<<<(unsigned)(cdiv(per * k, 256) < 65536 ? cdiv(per * k, 256) : 65536), 256, 0, sl>>>(
            R, R + Tin * cols, (int)Tin, (int)Tout, k, evecs_d, P, net.woff[wl - 1], net.boff[wl - 1]);
        HM_LAUNCHED();
        continue;
      }
      Tick t(h, HESS_K_BACKPROJ, 2.0 * N * Tout * k, 0.0);
      bp_build_kernel<<<(unsigned)(cdiv(N * cols, 256) < 65536 ? cdiv(N * cols, 256) : 65536), 256, 0, s>>>(
          c.d[wl], U, N, (int)Tout, k, Bf, bp_mode[wl] == 1 ? 1 : 0);
      HM_LAUNCHED();
      // the bias rows: row Tin of R (a row of ones appended to A^T), or their
      // own product
      const double* Rbl = Rb;
      if (bp_mode[wl] == 1) {
        // (B transposed: the digit split reads its rows along n, coalesced)
        F64GemmScratch f2 = fb;
        f2.M = Tin + 1;
        f2.Nn = cols < 256 ? cols : 256;
        if (wl == a_pre) HM_CUDA(cudaStreamWaitEvent(s, side->ev[3], 0));
        HM_TRY(f64_gemm_nt_tc(h, c.a[wl - 1], Tin, Bf, N, 1, N, Rf, cols, 1, f2, s, cols, Tin, wl == a_pre));
        Rbl = Rf + Tin * cols;
      } else {
        // R^T = B^T A: rows (i, c) of B^T against the Tin rows of A^T
        F64GemmScratch f2 = fb;
        f2.M = cols;
        f2.Nn = Tin;
        HM_TRY(f64_gemm_nt_tc(h, Bf, cols, c.a[wl - 1], 1, Tin, N, Rf, 1, cols, f2, s, Tin));
        Gemm<double> g;
        g.M = (int)Tout;
        g.N = k;
        g.K = (int)N;
        g.A = c.d[wl];
        g.sam = 1;
        g.sak = Tout;
        g.B = U;
        g.sbk = k;
        g.sbn = 1;
        g.C = Rb;
        g.scm = k;
        g.scn = 1;
        HM_TRY(gemm(g, s));
      }
      const int64_t per = (Tin + 1) * Tout;
      bp_scatter_kernel<<<(unsigned)(cdiv(per * k, 256) < 65536 ? cdiv(per * k, 256) : 65536), 256, 0, s>>>(
          Rf, Rbl, (int)Tin, (int)Tout, k, evecs_d, P, net.woff[wl - 1], net.boff[wl - 1]);
      HM_LAUNCHED();
    }
    if (narrow_side) {
      HM_CUDA(cudaEventRecord(side->ev[2], side->s));
      HM_CUDA(cudaStreamWaitEvent(s, side->ev[2], 0));
    }
    Tick t(h, HESS_K_BACKPROJ, 0.0, 0.0);
    HM_CUDA(cudaMemsetAsync(flag + 1, 0, sizeof(int), s));
    HM_TRY(finalize_vectors(evecs_d, P, theta, k, (double)N, evals_d, flag + 1, best, s));
    return HESS_OK;
  };

  int m = 0, spec_m = -1;
  bool converged = false;
  // the Ritz values reach the host with the convergence flags (room for k
  // doubles after the flags in the handle's pinned scratch)
  double* theta_host = k <= 500 ? hp + 4 : nullptr;
  if (dfg > 0) {
    const std::function<hess_status(int)> spec = tail;
    HM_TRY(run_lz_df(h, M, k, lb, dfg, &m, &converged, true, true, &spec, &spec_m, &post_launch, theta_host));
  } else {
    HM_TRY(post_launch());
    HM_TRY(run_lz(h, M, k, lb, &m, &converged));
  }
  res->lanczos_steps = m;
  {
    double f = 0.0;
    for (int wl = 1; wl <= L - 1; ++wl) f += (double)N * (N + 1) * (net.T[wl - 1] + net.T[wl]);
    for (int j = 0; j < m; ++j) f += 2.0 * N * N + 8.0 * N * (j + 1);
    f += 2.0 * N * m * k + 2.0 * P * N * k;
    res->flops = f;
  }
  res->converged = converged ? 1 : 0;
  if (spec_m == m && theta_host) {
    // the tail queued with these Ritz values is the result: the null
    // directions (the output pass's test) are known without waiting for it
    int deficient = 0;
    for (int c = 0; c < k; ++c)
      if (!(theta_host[c] > 1e-13 * theta_host[0]) || !(theta_host[c] > 0.0)) deficient = 1;
    res->rank_deficient = deficient;
    return HESS_OK;
  }
  if (spec_m != m) HM_TRY(tail(m));
  int* hi = reinterpret_cast<int*>(hp);
  HM_CUDA(cudaMemcpyAsync(hi, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  res->rank_deficient = hi[0];
  return HESS_OK;
}

hess_status topk_eig_dense(hess_mlp* h, const double* M, int64_t n, int k, double* evals_d, double* evecs_d,
                           Arena& ar, bool dry, EigResult* res) {
  LzBufs lb;
  plan_lz(ar, n, k, lb, nullptr, nullptr);
  int* flag = ar.take<int>(2);
  unsigned long long* best = ar.take<unsigned long long>((int64_t)2 * k * finalize_slices(n));
  if (dry) return HESS_OK;
  cudaStream_t s = h->stream;
  int m = 0;
  bool converged = false;
  HM_TRY(run_lz(h, M, k, lb, &m, &converged));
  res->lanczos_steps = m;
  {
    double f = 0.0;
    for (int j = 0; j < m; ++j) f += 2.0 * n * n + 8.0 * n * (j + 1);
    f += 2.0 * n * m * k;
    res->flops = f;
  }
  res->converged = converged ? 1 : 0;
  // Ritz vectors: row c of evecs = sum_j Y[c][j] q_j
  Gemm<double> g;
  g.M = (int)n;
  g.N = k;
  g.K = m;
  g.A = lb.Q;
  g.sam = 1;
  g.sak = n;
  g.B = lb.Y;
  g.sbk = 1;
  g.sbn = lb.mcap;
  g.C = evecs_d;
  g.scm = 1;
  g.scn = n;
  HM_TRY(gemm(g, s));
  HM_CUDA(cudaMemsetAsync(flag + 1, 0, sizeof(int), s));
  HM_TRY(finalize_vectors(evecs_d, n, lb.theta, k, 0.0, evals_d, flag + 1, best, s));
  int* hi = reinterpret_cast<int*>(h->host_pinned);
  HM_CUDA(cudaMemcpyAsync(hi, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  res->rank_deficient = hi[0];
  return HESS_OK;
}

}  // namespace hm

extern "C" hess_status hess_debug_set_barrier_limit(int64_t cycles) {
  hm::g_bar_limit.store(cycles > 0 ? (long long)cycles : 0);
  return HESS_OK;
}
