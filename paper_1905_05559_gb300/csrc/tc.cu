// Tensor-core contractions on sm_103a: tcgen05.mma with TMEM accumulators,
// operands staged by TMA (cp.async.bulk.tensor) into 128-byte-swizzled shared
// memory, one persistent CTA per SM with warp-specialised roles:
//   warp 0      TMA producer (one elected thread)
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2-9   epilogue: TMEM -> registers -> global, 32 TMEM lanes and
//               every other 32-column group of the tile each
// The accumulator is double-buffered in TMEM (2 x 256 fp32 columns) so the
// epilogue of one tile overlaps the main loop of the next.
//
// Split-BF16 ("x3") products: one stage holds A_hi, A_lo, B_hi and B_lo of a
// k-block and the MMA thread issues hi*hi, hi*lo and lo*hi from it into the
// same FP32 accumulator.
//
// Both users write a symmetric matrix from row blocks: an entry computed at
// (orow, ocol) is stored directly when ocol >= orow and mirrored to
// (ocol, orow) when ocol > orow, so every entry is written exactly once.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cfloat>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <type_traits>

#include "internal.h"

namespace hm {

namespace tc {

constexpr int BM = 128;  // UMMA M (rows of A per tile = TMEM lanes)
constexpr int BK = 64;   // bf16 elements per 128-byte swizzle row
constexpr int MAXBN = 256;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = MAXBN * BK * 2;
// operand ring: BF16 runs 4 stages of {A, B}; split-BF16 runs 2 stages of
// {A_hi, A_lo, B_hi, B_lo} and issues the three products from one stage
constexpr int RING_BYTES = 4 * (A_BYTES + B_BYTES);
constexpr int MAXSTAGES = 4;
constexpr int EPI_LD = 17;  // 16 columns + 1 pad
// per epilogue warp: a 32 x 16 transpose tile, then the 32 rows' output row
// and column base (int64 each)
constexpr int EPI_WARP_BYTES = 32 * EPI_LD * 4 + 32 * 16;
constexpr int EPI_WARPS = 8;  // two per TMEM lane quadrant, splitting the columns
constexpr int EPI_BYTES = EPI_WARPS * EPI_WARP_BYTES;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = 1024 + RING_BYTES + EPI_BYTES + BAR_BYTES;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr long long TIMEOUT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz
// K is accumulated in chunks of CHUNK_KB k-blocks (1024 products): each chunk
// goes to a fresh TMEM accumulator and the epilogue warps add it into the
// tile's main accumulator with round-to-nearest FP32 adds, so the error of the
// tensor cores' own accumulation does not grow with N.
constexpr int CHUNK_KB = 16;

struct Launch {
  const Job* jobs;
  const int4* tiles;  // (job, row tile, column tile, 0)
  int ntiles;
  int passes;         // 1: hi*hi;  3: hi*hi + hi*lo + lo*hi (one stage holds all four tiles)
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: on timeout (or when another role already gave up) raise the
// error flag and the CTA's abort flag and return false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err,
                                          volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > TIMEOUT_CYCLES) {
      *(volatile int*)err = 1;  // mapped host memory: read by the host without a sync
      *abort_flag = 1;
      return false;
    }
  }
}

// Operand tile load with an L2 evict-last policy: the operands are re-read by
// many tiles, while the output streams past them.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t evict_last_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128 B,
// 8-row core-matrix groups 1024 B apart (SBO), version 1 (tcgen05).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads and one wait (the wait covers both).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
      "%27, %28, %29, %30, %31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr), "r"(taddr + 16)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// First concatenated A row of unit p for the Hessian layer mapping:
// unit p owns rows (i, q) for i = p..Tout-1, q = 0..Tin-1.
__host__ __device__ __forceinline__ int64_t rows_before(int64_t p, int64_t Tin, int64_t Tout) {
  return Tin * (p * Tout - p * (p - 1) / 2);
}

// Output coordinates of tile row m: the entry (m, n) of the product lands at
// (orow, ocolb + n).  Mode 1: rows are the weight directions W_(p,q) of one
// layer, repeated for every output unit i >= p (the Hessian columns that can
// lie on or above the diagonal); the product column n is the input unit k of
// the Hessian column W_(i,k).  Mode 2: the tile's unit u = tile_y / ntn; rows
// are the directions W_(u,q) and the product column n is the n-th Hessian
// column from the layer's bias on.
// Unit u of concatenated W row r: rows_before(u) <= r < rows_before(u + 1)
// (the root of the quadratic rows_before as an FP32 estimate -- FP64 is slow
// on this GPU and the estimate only needs to be near -- then corrected by
// whole steps in integer arithmetic).
__device__ __forceinline__ int64_t wrow_unit(int64_t r, int64_t Tin, int64_t Tout) {
  const float b = 2.0f * (float)Tout + 1.0f;
  const float q = (float)(r / Tin);  // whole units of Tin rows
  int64_t u = (int64_t)floorf((b - sqrtf(fmaxf(b * b - 8.0f * q, 0.0f))) * 0.5f);
  if (u < 0) u = 0;
  if (u > Tout - 1) u = Tout - 1;
  while (u > 0 && rows_before(u, Tin, Tout) > r) --u;
  while (u + 1 < Tout && rows_before(u + 1, Tin, Tout) <= r) ++u;
  return u;
}

__device__ __forceinline__ void row_map(const Job& p, int64_t m, int tile_y, int64_t& orow,
                                        int64_t& ocolb) {
  if (p.mode == 0 || p.mode == 3) {
    orow = m;
    ocolb = 0;
    return;
  }
  const int64_t Tin = p.Tin, Tout = p.Tout;
  if (p.mode == 2) {
    // rows q < Tin: W_(u,q); row Tin: the bias b_u (the ones row of A)
    const int64_t u = p.p0 + tile_y / p.ntn;
    orow = m < Tin ? p.woff + u * Tin + m : p.boff + u;
    ocolb = p.boff;
    return;
  }
  const int64_t r = m + p.R0;
  const int64_t u = wrow_unit(r, Tin, Tout);
  const int64_t rr = r - rows_before(u, Tin, Tout);
  const int64_t i = u + rr / Tin, q = rr % Tin;
  orow = p.woff + u * Tin + q;
  ocolb = p.woff + i * Tin;
}

__global__ void __launch_bounds__(THREADS, 1)
    umma_gemm_kernel(const Launch L) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // the ring's 1024-byte alignment as an offset from the array, so that the
  // compiler still knows every pointer below addresses shared memory (an
  // integer round trip would make the epilogue's accesses generic ones)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* epi = reinterpret_cast<float*>(smem + RING_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES + EPI_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MAXSTAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const bool x3 = L.passes == 3;
  const int STAGES = x3 ? 2 : 4;
  const int STAGE_BYTES = x3 ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
  // offsets inside a stage (all multiples of 1024 bytes)
  const int OFF_ALO = A_BYTES, OFF_BHI = x3 ? 2 * A_BYTES : A_BYTES,
            OFF_BLO = 2 * A_BYTES + B_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + MAXSTAGES + s); };
  auto tfull = [&](int a) { return smem_u32(bars + 2 * MAXSTAGES + a); };
  auto tempty = [&](int a) { return smem_u32(bars + 2 * MAXSTAGES + 2 + a); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), 32 * EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      int last_job = -1;
      const uint64_t pol = evict_last_policy();
      for (int t = blockIdx.x; t < L.ntiles && ok; t += gridDim.x) {
        const int4 tile = L.tiles[t];
        const Job& jb = L.jobs[tile.x];
        if (tile.x != last_job) {
          // the maps live in global memory, written before the launch
          const CUtensorMap* maps[4] = {&jb.a_hi, &jb.a_lo, &jb.b_hi, &jb.b_lo};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                             reinterpret_cast<uint64_t>(maps[q]))
                         : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(maps[q])) : "memory");
          }
          last_job = tile.x;
        }
        // job fields in registers: the asm statements below clobber memory,
        // which would make every use of jb.* a fresh global load
        const int jbn = jb.BN, jnkb = jb.nkb;
        const uint32_t tx_bytes = (A_BYTES + jbn * BK * 2) * (x3 ? 2 : 1);
        const int brow0 = jb.mode == 2 ? (int)((tile.z / jb.ntn) * jb.brow + (tile.z % jb.ntn) * jbn)
                                       : tile.z * jbn;
        const CUtensorMap* m_ahi = &jb.a_hi;
        const CUtensorMap* m_alo = &jb.a_lo;
        const CUtensorMap* m_bhi = &jb.b_hi;
        const CUtensorMap* m_blo = &jb.b_lo;
        for (int j = 0; j < jnkb; ++j, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(empty(s), ph ^ 1, L.err, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(full(s), tx_bytes);
          tma_load_2d(smem_u32(st), m_ahi, j * BK, tile.y * BM, full(s), pol);
          tma_load_2d(smem_u32(st + OFF_BHI), m_bhi, j * BK, brow0, full(s), pol);
          if (x3) {
            tma_load_2d(smem_u32(st + OFF_ALO), m_alo, j * BK, tile.y * BM, full(s), pol);
            tma_load_2d(smem_u32(st + OFF_BLO), m_blo, j * BK, brow0, full(s), pol);
          }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA can exit
        const int first = it - STAGES > 0 ? it - STAGES : 0;
        for (int k = first; k < it; ++k) {
          const int s = k % STAGES;
          long long t0 = clock64();
          while (!mbar_try_wait(full(s), (k / STAGES) & 1) && clock64() - t0 < TIMEOUT_CYCLES) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tcount = 0;
      unsigned uses[2] = {0u, 0u};  // chunks written into each TMEM buffer so far
      bool ok = true;
      for (int t = blockIdx.x; t < L.ntiles && ok; t += gridDim.x, ++tcount) {
        const Job& jb = L.jobs[L.tiles[t].x];
        const int nvk = jb.nkb;
        const uint32_t idesc = jb.idesc;
        const int ckb = jb.chunk_kb > 0 ? jb.chunk_kb : CHUNK_KB;
        const int nchunk = (nvk + ckb - 1) / ckb;
        // the first chunk goes to the tile's main buffer, the others to the
        // second buffer, which the epilogue merges into the main one
        const int mainb = tcount & 1;
        for (int ch = 0; ch < nchunk && ok; ++ch) {
          const int buf = ch == 0 ? mainb : mainb ^ 1;
          if (!mbar_wait(tempty(buf), (uses[buf] & 1u) ^ 1u, L.err, abort_flag)) {
            ok = false;
            break;
          }
          ++uses[buf];
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + buf * MAXBN;
          const int j0 = ch * ckb, j1 = min(nvk, j0 + ckb);
          for (int j = j0; j < j1; ++j, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(full(s), ph, L.err, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint8_t* st = smem + s * STAGE_BYTES;
            const uint64_t ah = sdesc(smem_u32(st));
            const uint64_t bh = sdesc(smem_u32(st + OFF_BHI));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              umma_bf16(d_tmem, ah + 2 * kk, bh + 2 * kk, idesc, (j > j0 || kk > 0) ? 1u : 0u);
            if (x3) {
              const uint64_t al = sdesc(smem_u32(st + OFF_ALO));
              const uint64_t bl = sdesc(smem_u32(st + OFF_BLO));
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) umma_bf16(d_tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1u);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) umma_bf16(d_tmem, al + 2 * kk, bh + 2 * kk, idesc, 1u);
            }
            umma_commit(empty(s));
          }
          if (ok) umma_commit(tfull(buf));
        }
      }
    }
    __syncwarp();
  } else {
    const int q = warp & 3;               // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;     // which 32-column groups of the tile it handles
    float* e = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(epi) + (warp - 2) * EPI_WARP_BYTES);
    // per row of the warp's 32: where column n of the tile goes directly
    // (sptr[i] + n, null for rows past M) and the first column stored
    // directly (the diagonal for symmetric outputs)
    float** sptr = reinterpret_cast<float**>(e + 32 * EPI_LD);    // [32]
    int64_t* sdm = reinterpret_cast<int64_t*>(sptr + 32);         // [32]
    int tcount = 0;
    unsigned fulls[2] = {0u, 0u};  // chunk results consumed from each TMEM buffer
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    bool alive = true;
    for (int t = blockIdx.x; t < L.ntiles && alive; t += gridDim.x, ++tcount) {
      const int4 tile = L.tiles[t];
      const Job& p = L.jobs[tile.x];
      // job fields in registers (see the producer)
      const int BN = p.BN;
      const int64_t pM = p.M, Nn = p.Nn, ldo = p.ldo;
      const float scale = p.scale;
      float* const out = p.out;
      const bool sym = p.mode != 3;  // mode 3: a general product, every entry direct
      const int ckb = p.chunk_kb > 0 ? p.chunk_kb : CHUNK_KB;
      const int nchunk = (p.nkb + ckb - 1) / ckb;
      const int acc = tcount & 1;
      const bool got = mbar_wait(tfull(acc), fulls[acc] & 1u, L.err, abort_flag);
      if (__any_sync(0xffffffffu, !got)) break;
      ++fulls[acc];
      tc_fence_after();
      // merge the later K chunks into the main accumulator
      const int part = acc ^ 1;
      for (int ch = 1; ch < nchunk; ++ch) {
        const bool g2 = mbar_wait(tfull(part), fulls[part] & 1u, L.err, abort_flag);
        if (__any_sync(0xffffffffu, !g2)) {
          alive = false;
          break;
        }
        ++fulls[part];
        tc_fence_after();
        const uint32_t pm = tmem_base + acc * MAXBN + lane_off;
        const uint32_t pp = tmem_base + part * MAXBN + lane_off;
        for (int c = 0; c < BN / 16; ++c) {
          if (((c >> 1) & 1) != half) continue;
          float vm[16], vp[16];
          tmem_ld16(pp + c * 16, vp);
          tmem_ld16(pm + c * 16, vm);
#pragma unroll
          for (int i = 0; i < 16; ++i) vm[i] += vp[i];
          tmem_st16(pm + c * 16, vm);
        }
        tc_fence_before();
        mbar_arrive(tempty(part));
      }
      if (!alive) break;
      const int64_t m = (int64_t)tile.y * BM + q * 32 + lane;
      const bool rvalid = m < pM;
      int64_t orow = 0, ocolb = 0;
      if (rvalid) row_map(p, m, tile.z, orow, ocolb);
      const int64_t nbase = p.mode == 2 ? (int64_t)(tile.z % p.ntn) * BN : (int64_t)tile.z * BN;
      // column n of this lane's row: direct at out + orow ldo + ocolb + n when
      // n >= dmin (symmetric outputs: on or above the diagonal), mirrored at
      // out + (ocolb + n) ldo + orow when n > dmin
      const int64_t dmin = sym ? orow - ocolb : INT64_MIN / 2;
      const bool mir = sym && rvalid;
      sptr[lane] = rvalid ? out + orow * ldo + ocolb : nullptr;
      sdm[lane] = dmin;
      __syncwarp();
      // this lane's share of the direct stores: rows rg + 8 r (r < 4) of the
      // warp's 32, columns 4 cq .. 4 cq + 3 of each group of 16
      const int cq = lane & 3, rg = lane >> 2;
      float* rps[4];
      int64_t dms[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        rps[r] = sptr[rg + 8 * r];
        dms[r] = sdm[rg + 8 * r];
      }
      const uint32_t tbase = tmem_base + acc * MAXBN + (static_cast<uint32_t>(q * 32) << 16);
      // 16 columns of the tile: the mirror image (for a fixed column the
      // warp's 32 rows are adjacent), then the direct entries transposed
      // through shared memory: 8 rows x 4 column quads per warp store,
      // 16-byte stores where the address allows
      auto emit16 = [&](const float* v, int64_t n0) {
        float* mp = mir ? out + (ocolb + n0) * ldo + orow : nullptr;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int64_t n = n0 + jj;
          const float val = v[jj] * scale;
          e[lane * EPI_LD + jj] = val;
          if (mir) {
            if (n < Nn && n > dmin) __stcs(mp, val);
            mp += ldo;
          }
        }
        __syncwarp();
        const int64_t n = n0 + 4 * cq;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float* const rp = rps[r];
          if (rp != nullptr) {
            const int i = rg + 8 * r;
            const int64_t dm = dms[r];
            float a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = e[i * EPI_LD + 4 * cq + u];
            const uintptr_t ad = reinterpret_cast<uintptr_t>(rp + n);
            if (n >= dm && n + 3 < Nn && (ad & 15u) == 0u) {
              __stcs(reinterpret_cast<float4*>(rp + n), make_float4(a[0], a[1], a[2], a[3]));
            } else if (n >= dm && n + 3 < Nn && (ad & 7u) == 0u) {
              __stcs(reinterpret_cast<float2*>(rp + n), make_float2(a[0], a[1]));
              __stcs(reinterpret_cast<float2*>(rp + n + 2), make_float2(a[2], a[3]));
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (n + u < Nn && n + u >= dm) __stcs(rp + n + u, a[u]);
            }
          }
        }
        __syncwarp();
      };
      int c = 0;
      for (; c + 2 <= BN / 16; c += 2) {
        if (((c >> 1) & 1) != half) continue;
        float v[32];
        tmem_ld32(tbase + c * 16, v);
        emit16(v, nbase + c * 16);
        emit16(v + 16, nbase + c * 16 + 16);
      }
      if (c < BN / 16 && ((c >> 1) & 1) == half) {
        float v[16];
        tmem_ld16(tbase + c * 16, v);
        emit16(v, nbase + c * 16);
      }
      tc_fence_before();
      mbar_arrive(tempty(acc));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------ operand builders
__device__ __forceinline__ void split2(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// out[c][r] = in[r][c] split into bf16 hi/lo; r in [rows, ld) is zero padding.
__global__ void transpose_split_kernel(const float* in, int64_t rows, int64_t cols, int64_t ldin,
                                       __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ld) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? in[r * ldin + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < ld) {
      __nv_bfloat16 h, l;
      split2(t[threadIdx.x][y], h, l);
      hi[c * ld + r] = h;
      lo[c * ld + r] = l;
    }
  }
}

// out[c * ld + r] = in[r * ldin + c] for r < rows, 0 for rows <= r < ld: an
// example-major array turned example-fastest, so that the operand builders
// below read and write along the examples with whole-warp accesses.
__global__ void transpose_pad_kernel(const float* in, int64_t rows, int64_t cols, int64_t ldin, float* out,
                                     int64_t ld) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? in[r * ldin + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < ld) out[c * ld + r] = t[threadIdx.x][y];
  }
}


// Eight consecutive values split into bf16 hi/lo planes, 16-byte stores.
__device__ __forceinline__ void split8_store(const float (&v)[8], __nv_bfloat16* hi, __nv_bfloat16* lo,
                                             int64_t at) {
  uint4 h, l;
  uint32_t* hp = &h.x;
  uint32_t* lp = &l.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    hp[i] = *reinterpret_cast<const uint32_t*>(&hh);
    lp[i] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  *reinterpret_cast<uint4*>(hi + at) = h;
  *reinterpret_cast<uint4*>(lo + at) = l;
}

// Row Tin of the mode-2 A operand: ones over the examples (zero padding
// beyond N), so that the same job also yields the bias rows:
// H[b_u, c] = (1/N) sum_n F[n, u, c].
__global__ void ones_row_kernel(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t N, int64_t ld) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ld; n += (int64_t)gridDim.x * blockDim.x) {
    hi[n] = __float2bfloat16_rn(n < N ? 1.f : 0.f);
    lo[n] = __float2bfloat16_rn(0.f);
  }
}

// A operand of the Hessian rows of weight layer W (T_out x T_in): rows
// R0 .. R0 + nrows - 1 of the concatenation over units u of the rows
// (u, i, q), i = u..Tout-1, each holding, at example n,
//   R{delta}[n, b_u, i] * a[n, q]
// -- the R-operator of the weight direction W_(u,q) is a[n,q] times that of
// the bias direction b_u, because a unit direction only moves z_u.
// rdT: [u][i][ld] and aT: [q][ld], example-fastest and zero-padded.
__global__ void build_wrows_kernel(const float* rdT, const float* aT, int Tin, int Tout, int64_t R0,
                                   int64_t nrows, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ld) {
  // one warp per row, lanes along the examples (8 per lane per pass)
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < nrows; r += nw) {
    const int64_t g = r + R0;
    const int64_t u = wrow_unit(g, Tin, Tout);
    const int64_t rr = g - rows_before(u, Tin, Tout);
    const int64_t i = u + rr / Tin, q = rr % Tin;
    const float4* x = reinterpret_cast<const float4*>(rdT + (u * Tout + i) * ld);
    const float4* y = reinterpret_cast<const float4*>(aT + q * ld);
    const int64_t at = r * ld;
    for (int64_t j = lane; j < ld / 8; j += 32) {
      const float4 p0 = x[2 * j], p1 = x[2 * j + 1], w0 = y[2 * j], w1 = y[2 * j + 1];
      const float v[8] = {p0.x * w0.x, p0.y * w0.y, p0.z * w0.z, p0.w * w0.w,
                          p1.x * w1.x, p1.y * w1.y, p1.z * w1.z, p1.w * w1.w};
      split8_store(v, hi, lo, at + 8 * j);
    }
  }
}

// F[n, u, c] over the Hessian columns after W^(jm): the bias b^(jm+1) and all
// later layers, for the bias directions b_u of layer jm (the weight
// directions W_(u,q) then follow as a[n,q] F[n, u, c]):
//   column b_i of layer jl:     R{delta^(jl)}[n,u,i]
//   column W_(i,k) of layer jl: R{delta^(jl)}[n,u,i] a^(jl-1)[n,k]
//                               + delta^(jl)[n,i] R{a^(jl-1)}[n,u,k]
// Every input is example-fastest and zero-padded to ld.
struct FSeg {
  int64_t c0;  // first column of the segment (relative)
  int64_t nW;  // Tout*Tin of the layer (0 for the first segment)
  int Tin, Tout;
  const float* rd;    // [u][Tout][ld]
  const float* a;     // [Tin][ld]
  const float* dlt;   // [Tout][ld]
  const float* ra;    // [u][Tin][ld] or null
};
constexpr int MAXSEG = 8;
struct FArgs {
  int nseg;
  FSeg seg[MAXSEG];
  int64_t cols;
};
// The same F as split-BF16 planes, K-major for the tensor cores: row
// (u - p0) * cols + c holds F[., u, c] over the examples (zero-padded to ld).
__global__ void build_f_bf16_kernel(FArgs f, int p0, int np, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                    int64_t ld) {
  // one warp per row, lanes along the examples (8 per lane per pass)
  const int lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)np * f.cols;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < rows; row += nw) {
    const int u = p0 + (int)(row / f.cols);
    const int64_t c = row % f.cols;
    int s = 0;
    while (s + 1 < f.nseg && f.seg[s + 1].c0 <= c) ++s;
    const FSeg& g = f.seg[s];
    const int64_t cl = c - g.c0;
    const float4 *x1, *y1 = nullptr, *x2 = nullptr, *y2 = nullptr;
    if (cl < g.nW) {
      const int i = (int)(cl / g.Tin), k = (int)(cl % g.Tin);
      x1 = reinterpret_cast<const float4*>(g.rd + ((int64_t)u * g.Tout + i) * ld);
      y1 = reinterpret_cast<const float4*>(g.a + (int64_t)k * ld);
      if (g.ra) {
        x2 = reinterpret_cast<const float4*>(g.dlt + (int64_t)i * ld);
        y2 = reinterpret_cast<const float4*>(g.ra + ((int64_t)u * g.Tin + k) * ld);
      }
    } else {
      x1 = reinterpret_cast<const float4*>(g.rd + ((int64_t)u * g.Tout + (cl - g.nW)) * ld);
    }
    const int64_t at = row * ld;
    for (int64_t j = lane; j < ld / 8; j += 32) {
      float v[8];
      {
        const float4 a0 = x1[2 * j], a1 = x1[2 * j + 1];
        v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
        v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
      }
      if (y1) {
        const float4 b0 = y1[2 * j], b1 = y1[2 * j + 1];
        v[0] *= b0.x; v[1] *= b0.y; v[2] *= b0.z; v[3] *= b0.w;
        v[4] *= b1.x; v[5] *= b1.y; v[6] *= b1.z; v[7] *= b1.w;
      }
      if (x2) {
        const float4 d0 = x2[2 * j], d1 = x2[2 * j + 1], r0 = y2[2 * j], r1 = y2[2 * j + 1];
        v[0] = fmaf(d0.x, r0.x, v[0]); v[1] = fmaf(d0.y, r0.y, v[1]);
        v[2] = fmaf(d0.z, r0.z, v[2]); v[3] = fmaf(d0.w, r0.w, v[3]);
        v[4] = fmaf(d1.x, r1.x, v[4]); v[5] = fmaf(d1.y, r1.y, v[5]);
        v[6] = fmaf(d1.z, r1.z, v[6]); v[7] = fmaf(d1.w, r1.w, v[7]);
      }
      split8_store(v, hi, lo, at + 8 * j);
    }
  }
}

// --------------------------------------------------------------- host ----
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

hess_status get_encode() {
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return set_error(HESS_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
  return HESS_OK;
}

hess_status make_map(CUtensorMap* m, const void* ptr, int64_t ld, int64_t rows, int box_rows) {
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld % BK))
    return set_error(HESS_ERR_INVALID_ARG, "tensor map: misaligned operand");
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(HESS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return HESS_OK;
}

// Tile columns: multiple of 16 up to 256 minimising tiles * (BN + 64).
int pick_bn(int64_t Nn) {
  int best = 256;
  double bc = 1e300;
  for (int bn = 64; bn <= 256; bn += 16) {
    double cost = (double)cdiv(Nn, bn) * (bn + 64);
    if (cost < bc - 1e-9) {
      bc = cost;
      best = bn;
    }
  }
  return best;
}

uint32_t make_idesc(int BN) {
  return (1u << 4)                            // D: f32
         | (1u << 7)                          // A: bf16
         | (1u << 10)                         // B: bf16
         | ((uint32_t)(BN >> 3) << 17)        // N
         | ((uint32_t)(BM >> 4) << 24);       // M
}

}  // namespace tc

hess_status tc_available(hess_mlp* h) {
  int major = 0, minor = 0;
  HM_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device));
  HM_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device));
  if (major != 10 || minor != 3)
    return set_error(HESS_ERR_UNSUPPORTED, "tensor-core path is built for sm_103 (device is sm_%d%d)",
                     major, minor);
  return tc::get_encode();
}

namespace {

struct TcOperands {
  const void* Ahi;
  const void* Alo;
  int64_t arows;
  const void* Bhi;
  const void* Blo;
  int64_t brows;
  int64_t ld;
};

// Fill a job's operand maps, K and instruction descriptor; the caller sets
// the shape and output mapping.
hess_status make_job(const TcOperands& op, int BN, tc::Job* j) {
  using namespace tc;
  HM_TRY(make_map(&j->a_hi, op.Ahi, op.ld, op.arows, BM));
  HM_TRY(make_map(&j->a_lo, op.Alo, op.ld, op.arows, BM));
  HM_TRY(make_map(&j->b_hi, op.Bhi, op.ld, op.brows, BN));
  HM_TRY(make_map(&j->b_lo, op.Blo, op.ld, op.brows, BN));
  j->BN = BN;
  j->nkb = (int)(op.ld / BK);
  j->idesc = make_idesc(BN);
  return HESS_OK;
}

// Copy jobs and tiles to the device regions given and launch the
// persistent kernel over them.
hess_status launch_jobs(int sm_count, const tc::Job* jobs, int njobs, const int4* tiles, int ntiles,
                        tc::Job* jobs_d, int4* tiles_d, bool x3, int* err, PinnedStage& stage, cudaStream_t s) {
  using namespace tc;
  if (ntiles < 1) return HESS_OK;
  {
    // once per process (calls from several threads must not race on it)
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
      e = cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    HM_CUDA(e);
  }
  const void* src[2] = {jobs, tiles};
  const size_t bytes[2] = {njobs * sizeof(Job), ntiles * sizeof(int4)};
  void* dst[2] = {jobs_d, tiles_d};
  HM_TRY(stage_copy(stage, src, bytes, dst, 2, s));
  Launch L{jobs_d, tiles_d, ntiles, x3 ? 3 : 1, err};
  const int grid = ntiles < sm_count ? ntiles : sm_count;
  umma_gemm_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(L);
  HM_LAUNCHED();
  return HESS_OK;
}

template <typename T>
struct InF {
  const T* user;
  int on_dev;
};

hess_status classify_ptr(const hess_mlp* h, const void* p, int* on_dev) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *on_dev = 0;
    return HESS_OK;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    if (at.type == cudaMemoryTypeDevice && at.device != h->device)
      return set_error(HESS_ERR_INVALID_ARG, "buffer on device %d, handle on device %d", at.device,
                       h->device);
    *on_dev = 1;
  } else {
    *on_dev = 0;
  }
  return HESS_OK;
}

}  // namespace

double hcontract_flops(const Net& net, int64_t N, int jm, int jl, int64_t d0, int B);

// Upper tiles of a P x P symmetric update with BM x BN tiles (the column
// range reaches the diagonal), grouped by 8 tile rows so that concurrent tiles
// share operand panels in L2.
static int64_t syrk_tile_count(int64_t P, int BN) {
  using namespace tc;
  int64_t n = 0;
  const int64_t mt = cdiv(P, BM), nt = cdiv(P, BN);
  for (int64_t tn = 0; tn < nt; ++tn)
    for (int64_t tm = 0; tm < mt; ++tm)
      if (tn * BN + BN - 1 >= tm * BM) ++n;
  return n;
}

static void syrk_tiles(int64_t P, int BN, int job, std::vector<int4>& tiles) {
  using namespace tc;
  const int64_t mt = cdiv(P, BM), nt = cdiv(P, BN);
  for (int64_t g0 = 0; g0 < mt; g0 += 8)
    for (int64_t tn = 0; tn < nt; ++tn)
      for (int64_t tm = g0; tm < g0 + 8 && tm < mt; ++tm)
        if (tn * BN + BN - 1 >= tm * BM) tiles.push_back(make_int4(job, (int)tm, (int)tn, 0));
}



// Upper-triangle entries of the W x W block of a weight layer (rows (u, i, q)
// with i >= u, columns from the row's own entry on): 2N flops each.
static double wblock_entries(int64_t Tin, int64_t Tout, int64_t p0, int64_t p1) {
  double ent = 0.0;
  for (int64_t u = p0; u < p1; ++u)
    ent += (double)(Tout - u) * Tin * Tin - (double)Tin * (Tin - 1) / 2.0;
  return ent;
}

// Example-fastest copies (zero-padded to ld) of what the Hessian operand
// builders read: activations a^(j) and errors delta^(j) of the network, and
// R{delta^(j)}, R{a^(j)} of the current weight layer's bias directions.
struct TQ {
  float* a[kMaxLayers] = {};   // positions 0..L-2: [T_j][ld]
  float* d[kMaxLayers] = {};   // positions 2..L-1: [T_j][ld]
  float* rd[kMaxLayers] = {};  // positions 1..L-1: [u][T_j][ld] (reused for every weight layer)
  float* ra[kMaxLayers] = {};  // positions 1..L-2: [u][T_j][ld]
};

static void plan_tq(Arena& ar, const Net& net, int64_t ld, int Bmax, TQ& t) {
  const int L = net.L;
  for (int j = 0; j + 1 < L; ++j) t.a[j] = ar.take<float>((int64_t)net.T[j] * ld);
  for (int j = 2; j < L; ++j) t.d[j] = ar.take<float>((int64_t)net.T[j] * ld);
  for (int j = 1; j < L; ++j) t.rd[j] = ar.take<float>((int64_t)Bmax * net.T[j] * ld);
  for (int j = 1; j + 1 < L; ++j) t.ra[j] = ar.take<float>((int64_t)Bmax * net.T[j] * ld);
}

static hess_status transpose_pad(const float* in, int64_t rows, int64_t cols, float* out, int64_t ld,
                                 cudaStream_t s) {
  tc::transpose_pad_kernel<<<dim3((unsigned)cdiv(ld, 32), (unsigned)cdiv(cols, 32)), dim3(32, 8), 0, s>>>(
      in, rows, cols, cols, out, ld);
  HM_LAUNCHED();
  return HESS_OK;
}

static hess_status transpose_caches(const Net& net, const Caches<float>& c, int64_t N, int64_t ld, TQ& t,
                                    cudaStream_t s) {
  const int L = net.L;
  for (int j = 0; j + 1 < L; ++j) HM_TRY(transpose_pad(c.a[j], N, net.T[j], t.a[j], ld, s));
  for (int j = 2; j < L; ++j) HM_TRY(transpose_pad(c.d[j], N, net.T[j], t.d[j], ld, s));
  return HESS_OK;
}

// R-quantities of weight layer jm's B = T_jm bias directions, [n][u][t] ->
// [u][t][n].
static hess_status transpose_rop(const Net& net, const RopBufs<float>& rb, int jm, int64_t N, int64_t ld,
                                 TQ& t, cudaStream_t s) {
  const int L = net.L, B = net.T[jm];
  for (int j = jm; j < L; ++j) HM_TRY(transpose_pad(rb.rd[j], N, (int64_t)B * net.T[j], t.rd[j], ld, s));
  for (int j = jm; j + 1 < L; ++j) HM_TRY(transpose_pad(rb.ra[j], N, (int64_t)B * net.T[j], t.ra[j], ld, s));
  return HESS_OK;
}

// F segments of weight layer jm: the bias b^(jm+1) and every later layer.
static hess_status f_args(const Net& net, const TQ& t, int jm, tc::FArgs& fa) {
  using namespace tc;
  const int L = net.L;
  const int64_t boff = net.boff[jm - 1];
  fa = FArgs{};
  fa.cols = net.P - boff;
  FSeg g{};
  g.Tin = net.T[jm - 1];
  g.Tout = net.T[jm];
  g.rd = t.rd[jm];
  fa.seg[fa.nseg++] = g;
  for (int jl = jm + 1; jl < L; ++jl) {
    if (fa.nseg >= MAXSEG) return set_error(HESS_ERR_UNSUPPORTED, "too many layers for the tensor-core Hessian");
    FSeg q{};
    q.c0 = net.woff[jl - 1] - boff;
    q.nW = (int64_t)net.T[jl - 1] * net.T[jl];
    q.Tin = net.T[jl - 1];
    q.Tout = net.T[jl];
    q.rd = t.rd[jl];
    q.a = t.a[jl - 1];
    q.dlt = t.d[jl];
    q.ra = t.ra[jl - 1];
    fa.seg[fa.nseg++] = q;
  }
  return HESS_OK;
}

// Blocks of 256 threads (a warp per row) for an operand builder over `rows`
// rows: enough to fill every SM several times, each warp looping over rows.
static unsigned builder_blocks(int64_t rows, int sms) {
  const int64_t want = cdiv(rows, 8), cap = (int64_t)sms * 16;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Operands of weight layer jm shared by its W-row and F contractions: the
// layer input a^(jm-1) as split planes, rows 0..Tin-1, and the ones row Tin.
static hess_status build_layer_b(const Net& net, const Caches<float>& c, int jm, int64_t N, int64_t ld,
                                 __nv_bfloat16* bhi, __nv_bfloat16* blo, cudaStream_t s) {
  const int Tin = net.T[jm - 1];
  tc::transpose_split_kernel<<<dim3((unsigned)cdiv(ld, 32), (unsigned)cdiv(Tin, 32)), dim3(32, 8), 0, s>>>(
      c.a[jm - 1], N, Tin, Tin, bhi, blo, ld);
  HM_LAUNCHED();
  tc::ones_row_kernel<<<(unsigned)cdiv(ld, 256), 256, 0, s>>>(bhi + (int64_t)Tin * ld, blo + (int64_t)Tin * ld,
                                                               N, ld);
  HM_LAUNCHED();
  return HESS_OK;
}

// W rows of units [p0, p1), where R0 = rows_before(p0).
static hess_status build_wrows(const Net& net, const TQ& t, int jm, int p1, int64_t R0, int64_t ld, int sms,
                               __nv_bfloat16* ahi, __nv_bfloat16* alo, cudaStream_t s) {
  const int Tin = net.T[jm - 1], Tout = net.T[jm];
  const int64_t nrows = tc::rows_before(p1, Tin, Tout) - R0;
  tc::build_wrows_kernel<<<builder_blocks(nrows, sms), 256, 0, s>>>(t.rd[jm], t.a[jm - 1], Tin, Tout, R0, nrows,
                                                                      ahi, alo, ld);
  HM_LAUNCHED();
  return HESS_OK;
}

static hess_status build_f(const tc::FArgs& fa, int p0, int np, int64_t ld, int sms, __nv_bfloat16* fhi,
                           __nv_bfloat16* flo, cudaStream_t s) {
  tc::build_f_bf16_kernel<<<builder_blocks((int64_t)np * fa.cols, sms), 256, 0, s>>>(fa, p0, np, fhi, flo, ld);
  HM_LAUNCHED();
  return HESS_OK;
}

// Jobs of weight layer jm: W rows (u, i, q) for units [p0, p1) against the
// W columns (mode 1); W and bias rows of units [q0, q0 + np) against the
// columns after W (mode 2).
static void wrow_job(const Net& net, int jm, int p0, int p1, int64_t R0, float* out, int64_t N, int BN,
                     tc::Job& job, std::vector<int4>& tiles, int jid) {
  using namespace tc;
  const int Tin = net.T[jm - 1], Tout = net.T[jm];
  const int64_t rows = rows_before(p1, Tin, Tout) - R0;
  job.BN = BN;
  job.M = rows;
  job.Nn = Tin;
  job.scale = 1.0f / (float)N;
  job.out = out;
  job.ldo = net.P;
  job.mode = 1;
  job.woff = net.woff[jm - 1];
  job.Tin = Tin;
  job.Tout = Tout;
  job.p0 = p0;
  job.R0 = R0;
  for (int64_t tm = 0; tm < cdiv(rows, BM); ++tm)
    for (int64_t tn = 0; tn < cdiv(Tin, BN); ++tn) tiles.push_back(make_int4(jid, (int)tm, (int)tn, 0));
}

static void f_job(const Net& net, int jm, int q0, int np, float* out, int64_t N, int BN, tc::Job& job,
                  std::vector<int4>& tiles, int jid) {
  using namespace tc;
  const int Tin = net.T[jm - 1], Tout = net.T[jm];
  const int64_t boff = net.boff[jm - 1], rest = net.P - boff;
  const int ntn = (int)cdiv(rest, BN);
  job.BN = BN;
  job.M = Tin + 1;
  job.Nn = rest;
  job.scale = 1.0f / (float)N;
  job.out = out;
  job.ldo = net.P;
  job.mode = 2;
  job.woff = net.woff[jm - 1];
  job.boff = boff;
  job.Tin = Tin;
  job.Tout = Tout;
  job.p0 = q0;
  job.ntn = ntn;
  job.brow = rest;
  for (int64_t tm = 0; tm < cdiv(Tin + 1, BM); ++tm)
    for (int u = 0; u < np; ++u)
      for (int tn = 0; tn < ntn; ++tn) tiles.push_back(make_int4(jid, (int)tm, u * ntn + tn, 0));
}

// Algorithmic flops of weight layer jm's contractions: the upper triangle of
// the W x W block for units [p0, p1), and the W and bias rows of np units
// against the columns after W, 2N each.
static double wrow_flops(int64_t Tin, int64_t Tout, int64_t p0, int64_t p1, int64_t N) {
  return 2.0 * N * wblock_entries(Tin, Tout, p0, p1);
}
static double f_flops(int64_t Tin, int64_t rest, int64_t np, int64_t N) {
  return 2.0 * N * (double)np * (Tin + 1) * rest;
}

// ------------------------------------------------------------ autotuner --
// Tile width of a contraction.  By default a cost model (pick_bn); with
// tuning on, the first contraction of each shape (mode, columns, K blocks,
// products) is timed alone at every candidate width on its real operands --
// the output is written each time, with the same values -- and the fastest
// width is kept for the process (and can be saved and loaded as a table).
namespace {
struct TuneKey {
  int mode;
  int64_t nn;
  int nkb;
  int x3;
  bool operator<(const TuneKey& o) const {
    if (mode != o.mode) return mode < o.mode;
    if (nn != o.nn) return nn < o.nn;
    if (nkb != o.nkb) return nkb < o.nkb;
    return x3 < o.x3;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
std::atomic<int> g_tune_on{0};
constexpr int kTuneCand[] = {64, 96, 128, 160, 192, 224, 256};
struct TuneBuf {
  tc::Job* jobs = nullptr;
  int4* tiles = nullptr;
  size_t cap = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
TuneBuf g_tune_buf;  // one per process (tuning is serialised by g_tune_mu)
}  // namespace

// The width for a contraction: tuned if known, else the cost model.
// `*untuned` tells the caller that tuning is on and this shape has no entry.
static int choose_bn(int mode, int64_t nn, int nkb, bool x3, bool* untuned) {
  const TuneKey key{mode, nn, nkb, x3 ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      *untuned = false;
      return it->second;
    }
  }
  *untuned = g_tune_on.load() != 0;
  return mode == 0 ? 256 : tc::pick_bn(nn);
}

// Builds the job and its tiles for a width (maps, fields, tile list).
using JobBuilder = std::function<hess_status(int BN, tc::Job& job, std::vector<int4>& tiles)>;

// Times the job alone at each candidate width and records the fastest.
static hess_status tune_job(int sm_count, int mode, int64_t nn, int nkb, bool x3, const JobBuilder& build,
                            PinnedStage& stage, int* err, cudaStream_t s, int* best_bn) {
  const TuneKey key{mode, nn, nkb, x3 ? 1 : 0};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto found = g_tuned.find(key);
  if (found != g_tuned.end()) {
    *best_bn = found->second;
    return HESS_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HM_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // no timing inside a graph capture
    *best_bn = mode == 0 ? 256 : tc::pick_bn(nn);
    return HESS_OK;
  }
  TuneBuf& b = g_tune_buf;
  if (!b.e0) {
    HM_CUDA(cudaEventCreate(&b.e0));
    HM_CUDA(cudaEventCreate(&b.e1));
  }
  float best_ms = 1e30f;
  int best = mode == 0 ? 256 : tc::pick_bn(nn);
  for (int bn : kTuneCand) {
    // a narrower candidate already covers every column in one tile
    if (bn > kTuneCand[0] && bn - 32 >= (int64_t)align_up((size_t)nn, 16)) continue;
    tc::Job job{};
    std::vector<int4> tiles;
    HM_TRY(build(bn, job, tiles));
    for (int4& t : tiles) t.x = 0;  // the job runs alone: its table has one entry
    const size_t need = tiles.size() + 1;
    if (need > b.cap) {
      HM_CUDA(cudaStreamSynchronize(s));
      cudaFree(b.jobs);
      cudaFree(b.tiles);
      b.jobs = nullptr;
      b.tiles = nullptr;
      b.cap = 0;
      HM_CUDA(cudaMalloc(&b.jobs, sizeof(tc::Job)));
      HM_CUDA(cudaMalloc(&b.tiles, need * sizeof(int4)));
      b.cap = need;
    }
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms caches and tables
      HM_CUDA(cudaEventRecord(b.e0, s));
      HM_TRY(launch_jobs(sm_count, &job, 1, tiles.data(), (int)tiles.size(), b.jobs, b.tiles, x3, err, stage, s));
      HM_CUDA(cudaEventRecord(b.e1, s));
    }
    HM_CUDA(cudaEventSynchronize(b.e1));
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, b.e0, b.e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
  }
  g_tuned[key] = best;
  *best_bn = best;
  return HESS_OK;
}

namespace {
// the handle's stream set to s for a scope (h may be null: nothing)
struct StreamScope {
  StreamScope(hess_mlp* h, cudaStream_t s) : h_(h), keep_(h ? h->stream : nullptr) {
    if (h_) h_->stream = s;
  }
  ~StreamScope() {
    if (h_) h_->stream = keep_;
  }
  hess_mlp* h_;
  cudaStream_t keep_;
};
}  // namespace

hess_status tc_prep(hess_mlp* h, const TcItem& it, Arena& ar, bool live, TcPlan& plan, cudaStream_t s,
                    const TcFork* fork) {
  using namespace tc;
  using bf = __nv_bfloat16;
  const Net& net = h->net;
  const int L = net.L;
  const int64_t P = net.P, N = it.N;
  const int64_t ld = align_up((size_t)N, BK);
  const float* omega = h->omega32;
  hess_mlp* th = s == h->stream ? h : nullptr;  // per-class timing on the handle's own stream
  Caches<float> c;
  plan_caches(ar, net, N, c);
  if (live) HM_TRY(forward_backward(net, omega, it.X, it.Y, c, s));
  const bool forked = live && fork && it.want_hess;
  if (forked) {
    HM_CUDA(cudaEventRecord(fork->after_fb, s));
    HM_CUDA(cudaStreamWaitEvent(fork->s, fork->after_fb, 0));
  }
  if (it.want_opg) {
    // OPG = G^T G / N (Sec. 3, the outer-product approximation): G is written
    // once in FP32, then split into K-major bf16 planes
    float* G = ar.take<float>(N * P);
    bf* hi = ar.take<bf>(P * ld);
    bf* lo = ar.take<bf>(P * ld);
    const double fl = (double)N * P * (P + 1);
    plan.syrk_flops += fl;
    if (live) {
      {
        Tick t(th, HESS_K_GRADS, 0.0, (double)N * P * 4.0);
        HM_TRY(write_grads(net, c, G, P, s));
      }
      transpose_split_kernel<<<dim3((unsigned)cdiv(ld, 32), (unsigned)cdiv(P, 32)), dim3(32, 8), 0, s>>>(
          G, N, P, P, hi, lo, ld);
      HM_LAUNCHED();
    }
    const int jid = (int)plan.jobs.size();
    JobBuilder build = [&](int BN, Job& job, std::vector<int4>& tl) -> hess_status {
      if (live) HM_TRY(make_job(TcOperands{hi, lo, P, hi, lo, P, ld}, BN, &job));
      job.BN = BN;
      job.M = P;
      job.Nn = P;
      job.scale = 1.0f / (float)N;
      job.out = it.opg;
      job.ldo = P;
      job.mode = 0;
      syrk_tiles(P, BN, jid, tl);
      return HESS_OK;
    };
    bool untuned = false;
    int BN = choose_bn(0, P, (int)(ld / BK), it.x3, &untuned);
    if (live && untuned) HM_TRY(tune_job(h->sm_count, 0, P, (int)(ld / BK), it.x3, build, h->stage, h->err_dev, s, &BN));
    Job job{};
    HM_TRY(build(BN, job, plan.tiles));
    plan.jobs.push_back(job);
    plan.caps.push_back(syrk_tile_count(P, kTuneCand[0]));
    plan.tiles_cap += plan.caps.back();
  }
  if (it.want_hess) {
    // exact Hessian (Sec. 3, Eq. for H_ij) from the R-operator over the bias
    // directions of each weight layer: the W x W block (mode 1) and the W and
    // bias rows against the columns after W (mode 2), all on the tensor cores
    // (on the fork's stream, with the per-class timing there too)
    const cudaStream_t sh = forked ? fork->s : s;
    StreamScope scope(th && forked ? h : nullptr, sh);
    int Tmax = 0;
    for (int jm = 1; jm < L; ++jm) Tmax = net.T[jm] > Tmax ? net.T[jm] : Tmax;
    RopBufs<float> r;
    plan_rop(ar, net, N, 1, Tmax, r);
    TQ tq;
    plan_tq(ar, net, ld, Tmax, tq);
    if (live) HM_TRY(transpose_caches(net, c, N, ld, tq, sh));
    for (int jm = 1; jm < L; ++jm) {
      const int Tin = net.T[jm - 1], Tout = net.T[jm];
      const int64_t boff = net.boff[jm - 1];
      const int64_t rows = rows_before(Tout, Tin, Tout);
      const int64_t rest = P - boff;
      bf* bhi = ar.take<bf>((int64_t)(Tin + 1) * ld);
      bf* blo = ar.take<bf>((int64_t)(Tin + 1) * ld);
      bf* ahi = ar.take<bf>(rows * ld);
      bf* alo = ar.take<bf>(rows * ld);
      bf* fhi = ar.take<bf>((int64_t)Tout * rest * ld);
      bf* flo = ar.take<bf>((int64_t)Tout * rest * ld);
      plan.hess_flops += wrow_flops(Tin, Tout, 0, Tout, N) + f_flops(Tin, rest, Tout, N);
      FArgs fa;
      HM_TRY(f_args(net, tq, jm, fa));
      if (live) {
        RopBufs<float> rb = r;
        rb.B = Tout;
        {
          Tick t(th, HESS_K_ROP, 0.0, 0.0);
          HM_TRY(rop_block(net, omega, c, jm, boff, Tout, rb, sh));
        }
        HM_TRY(transpose_rop(net, rb, jm, N, ld, tq, sh));
        HM_TRY(build_layer_b(net, c, jm, N, ld, bhi, blo, sh));
        HM_TRY(build_wrows(net, tq, jm, Tout, 0, ld, h->sm_count, ahi, alo, sh));
        HM_TRY(build_f(fa, 0, Tout, ld, h->sm_count, fhi, flo, sh));
      }
      const int nkb = (int)(ld / BK);
      {
        const int jid = (int)plan.jobs.size();
        JobBuilder build = [&](int BN, Job& job, std::vector<int4>& tl) -> hess_status {
          if (live) HM_TRY(make_job(TcOperands{ahi, alo, rows, bhi, blo, Tin, ld}, BN, &job));
          wrow_job(net, jm, 0, Tout, 0, it.hess, N, BN, job, tl, jid);
          return HESS_OK;
        };
        bool untuned = false;
        int BN = choose_bn(1, Tin, nkb, it.x3, &untuned);
        if (live && untuned) HM_TRY(tune_job(h->sm_count, 1, Tin, nkb, it.x3, build, h->stage, h->err_dev, sh, &BN));
        Job jw{};
        HM_TRY(build(BN, jw, plan.tiles));
        plan.jobs.push_back(jw);
        plan.caps.push_back(cdiv(rows, BM) * cdiv(Tin, kTuneCand[0]));
        plan.tiles_cap += plan.caps.back();
      }
      {
        const int jid = (int)plan.jobs.size();
        JobBuilder build = [&](int BN, Job& job, std::vector<int4>& tl) -> hess_status {
          if (live) HM_TRY(make_job(TcOperands{bhi, blo, Tin + 1, fhi, flo, (int64_t)Tout * rest, ld}, BN, &job));
          f_job(net, jm, 0, Tout, it.hess, N, BN, job, tl, jid);
          return HESS_OK;
        };
        bool untuned = false;
        int BN = choose_bn(2, rest, nkb, it.x3, &untuned);
        if (live && untuned) HM_TRY(tune_job(h->sm_count, 2, rest, nkb, it.x3, build, h->stage, h->err_dev, sh, &BN));
        Job jf{};
        HM_TRY(build(BN, jf, plan.tiles));
        plan.jobs.push_back(jf);
        plan.caps.push_back(cdiv(Tin + 1, BM) * (int64_t)Tout * cdiv(rest, kTuneCand[0]));
        plan.tiles_cap += plan.caps.back();
      }
    }
    if (forked) HM_CUDA(cudaEventRecord(fork->done, sh));
  }
  return HESS_OK;
}

void tc_split_plan(const TcPlan& both, int nfirst, TcPlan& first, TcPlan& rest) {
  first = TcPlan{};
  rest = TcPlan{};
  for (int j = 0; j < (int)both.jobs.size(); ++j) {
    TcPlan& dst = j < nfirst ? first : rest;
    dst.jobs.push_back(both.jobs[j]);
    const int64_t cap = j < (int)both.caps.size() ? both.caps[j] : 0;
    dst.caps.push_back(cap);
    dst.tiles_cap += cap;
  }
  for (const int4& t : both.tiles) {
    if (t.x < nfirst)
      first.tiles.push_back(t);
    else
      rest.tiles.push_back(make_int4(t.x - nfirst, t.y, t.z, t.w));
  }
  first.syrk_flops = both.syrk_flops;
  rest.hess_flops = both.hess_flops;
}

hess_status tc_launch_plan(int sm_count, const TcPlan& plan, Arena& ar, bool live, bool x3, int* err,
                           PinnedStage& stage, cudaStream_t s) {
  using namespace tc;
  // room for the tile list at any candidate width, so that a planning pass
  // (before tuning) lays out enough
  const size_t nt = plan.tiles.size() > (size_t)plan.tiles_cap ? plan.tiles.size() : (size_t)plan.tiles_cap;
  tc::Job* jd = ar.take<tc::Job>(plan.jobs.size() ? plan.jobs.size() : 1);
  int4* td = ar.take<int4>(nt ? nt : 1);
  if (!live || plan.tiles.empty()) return HESS_OK;
  // longest tiles first (K and tile width), so that a static round-robin over
  // the CTAs ends with short tiles; the stable order keeps each job's L2
  // grouping
  std::vector<int4> order(plan.tiles);
  std::stable_sort(order.begin(), order.end(), [&](const int4& a, const int4& b) {
    const Job& ja = plan.jobs[a.x];
    const Job& jb = plan.jobs[b.x];
    return (int64_t)ja.nkb * ja.BN > (int64_t)jb.nkb * jb.BN;
  });
  return launch_jobs(sm_count, plan.jobs.data(), (int)plan.jobs.size(), order.data(), (int)order.size(), jd,
                     td, x3, err, stage, s);
}

// Stages host inputs and outputs for the single-network calls.
struct Staged {
  const float* X;
  const float* Y;
  float* out;
  int x_dev, y_dev, o_dev;  // 1: device-accessible as given (device memory or mapped pinned host memory)
  int o_host;               // the output is host memory written in place (no copy back)
};

// The device alias of pinned (page-locked, mapped) host memory, or null: the
// kernels then read and write it in place over the host link.
static void* host_alias(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

static hess_status stage(hess_mlp* h, Arena& ar, bool live, const void* X, const void* Y, void* out, int64_t N,
                         const Staged& st, Staged& d) {
  const Net& net = h->net;
  const int64_t P = net.P, T1 = net.T[0], TL = net.T[net.L - 1];
  d = st;
  float* xs = st.x_dev ? nullptr : ar.take<float>(N * T1);
  float* ys = st.y_dev ? nullptr : ar.take<float>(N * TL);
  float* os = st.o_dev ? nullptr : ar.take<float>(P * P);
  if (!st.x_dev) d.X = xs;
  if (!st.y_dev) d.Y = ys;
  if (!st.o_dev) d.out = os;
  if (live && !st.x_dev) HM_CUDA(cudaMemcpyAsync(xs, X, N * T1 * 4, cudaMemcpyHostToDevice, h->stream));
  if (live && !st.y_dev) HM_CUDA(cudaMemcpyAsync(ys, Y, N * TL * 4, cudaMemcpyHostToDevice, h->stream));
  return HESS_OK;
}

// One network through tc_prep + one persistent launch (kind 0: OPG, 1: H).
static hess_status run_single(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3, void* out,
                              int kind) {
  Staged st{(const float*)X, (const float*)Y, (float*)out, 0, 0, 0, 0};
  HM_TRY(classify_ptr(h, X, &st.x_dev));
  HM_TRY(classify_ptr(h, Y, &st.y_dev));
  HM_TRY(classify_ptr(h, out, &st.o_dev));
  if (!st.o_dev) {
    // pinned host output: written in place by the kernels (the transfer
    // overlaps the contraction instead of following it)
    if (void* a = host_alias(out)) {
      st.out = static_cast<float*>(a);
      st.o_dev = 1;
      st.o_host = 1;
    }
  }
  cudaStream_t s = h->stream;
  char* split = nullptr;
  TcPlan plan;
  auto build = [&](Arena& ar, bool live) -> hess_status {
    Staged d;
    HM_TRY(stage(h, ar, live, X, Y, out, N, st, d));
    split = ar.take<char>(kSplitBytes);
    TcItem it{d.X, d.Y, N, kind == 0, kind == 1, kind == 0 ? d.out : nullptr, kind == 1 ? d.out : nullptr, x3};
    SplitGuard sg(split, kSplitBytes, h->sm_count);
    HM_TRY(tc_prep(h, it, ar, live, plan, s));
    Tick t(live ? h : nullptr, kind == 0 ? HESS_K_SYRK : HESS_K_HCONTRACT,
           kind == 0 ? plan.syrk_flops : plan.hess_flops, 0.0);
    return tc_launch_plan(h->sm_count, plan, ar, live, x3, h->err_dev, h->stage, s);
  };
  Arena ar;
  HM_TRY(build(ar, false));
  HM_TRY(ensure_ws(h, ar.off));
  plan = TcPlan{};
  ar = Arena{h->ws, 0};
  HM_TRY(build(ar, true));
  if (!st.o_dev) {
    const int64_t P = h->net.P;
    Staged d;
    Arena a2{h->ws, 0};
    HM_TRY(stage(h, a2, false, X, Y, out, N, st, d));
    HM_CUDA(cudaMemcpyAsync(out, d.out, P * P * 4, cudaMemcpyDeviceToHost, s));
  }
  if (!st.o_dev || st.o_host || !st.x_dev || !st.y_dev) {
    // host buffers involved: the call waits for its work
    HM_CUDA(cudaStreamSynchronize(s));
    return take_sticky_error(h);
  }
  return HESS_OK;
}

// Bytes of the whole-operand Hessian plan (caches, R-op buffers, operands).
static size_t hessian_plan_bytes(hess_mlp* h, int64_t N) {
  TcPlan plan;
  Arena ar;
  TcItem it{nullptr, nullptr, N, false, true, nullptr, nullptr};
  tc_prep(h, it, ar, false, plan, h->stream);
  return ar.off;
}

// Chunked Hessian for problems whose whole operand set exceeds the handle's
// operand limit: W-row blocks and F units are built and contracted a chunk at
// a time in reused buffers (one launch per chunk).  Same operands and tiles
// per entry as the one-launch schedule, so the same bits.
hess_status run_hessian_chunked(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3,
                                void* Hout) {
  using namespace tc;
  using bf = __nv_bfloat16;
  const Net& net = h->net;
  const int L = net.L;
  const int64_t P = net.P;
  Staged st{(const float*)X, (const float*)Y, (float*)Hout, 0, 0, 0};
  HM_TRY(classify_ptr(h, X, &st.x_dev));
  HM_TRY(classify_ptr(h, Y, &st.y_dev));
  HM_TRY(classify_ptr(h, Hout, &st.o_dev));
  const int64_t ld = align_up((size_t)N, BK);
  int Tmax = 0, Tinmax = 0;
  int64_t maxRest = 0;
  for (int jm = 1; jm < L; ++jm) {
    Tmax = net.T[jm] > Tmax ? net.T[jm] : Tmax;
    Tinmax = net.T[jm - 1] > Tinmax ? net.T[jm - 1] : Tinmax;
    const int64_t rest = P - net.boff[jm - 1];
    maxRest = rest > maxRest ? rest : maxRest;
  }
  // operand budget: A rows per chunk and units per F chunk
  const double budget = (double)h->op_limit;
  int64_t arows_cap = (int64_t)(budget / (double)(ld * 4));
  int64_t arows_max = 0;
  for (int jm = 1; jm < L; ++jm) {
    const int64_t Tin = net.T[jm - 1], Tout = net.T[jm];
    const int64_t tot = rows_before(Tout, Tin, Tout);
    // at least one unit (the first is the largest: Tout * Tin rows)
    const int64_t need = tot < arows_cap ? tot : (Tout * Tin > arows_cap ? Tout * Tin : arows_cap);
    arows_max = need > arows_max ? need : arows_max;
  }
  int pchunk = (int)(budget / (double)(ld * maxRest * 4));
  pchunk = pchunk > Tmax ? Tmax : (pchunk < 1 ? 1 : pchunk);
  int64_t max_tiles = cdiv(arows_max, BM) * cdiv(Tinmax, 64);
  for (int jm = 1; jm < L; ++jm) {
    const int64_t rest = P - net.boff[jm - 1];
    const int64_t t2 = cdiv(net.T[jm - 1] + 1, BM) * pchunk * cdiv(rest, pick_bn(rest));
    max_tiles = t2 > max_tiles ? t2 : max_tiles;
  }
  cudaStream_t s = h->stream;
  Staged d;
  Caches<float> c;
  RopBufs<float> r;
  TQ tq;
  bf *bhi, *blo, *ahi, *alo, *fhi, *flo;
  int4* tl;
  Job* jd;
  char* split;
  auto plan = [&](Arena& ar, bool live) -> hess_status {
    HM_TRY(stage(h, ar, live, X, Y, Hout, N, st, d));
    plan_caches(ar, net, N, c);
    plan_rop(ar, net, N, 1, Tmax, r);
    plan_tq(ar, net, ld, Tmax, tq);
    bhi = ar.take<bf>((int64_t)(Tinmax + 1) * ld);
    blo = ar.take<bf>((int64_t)(Tinmax + 1) * ld);
    ahi = ar.take<bf>(arows_max * ld);
    alo = ar.take<bf>(arows_max * ld);
    fhi = ar.take<bf>((int64_t)pchunk * maxRest * ld);
    flo = ar.take<bf>((int64_t)pchunk * maxRest * ld);
    tl = ar.take<int4>(max_tiles);
    jd = ar.take<Job>(1);
    split = ar.take<char>(kSplitBytes);
    return HESS_OK;
  };
  Arena ar;
  HM_TRY(plan(ar, false));
  HM_TRY(ensure_ws(h, ar.off));
  ar = Arena{h->ws, 0};
  HM_TRY(plan(ar, true));
  SplitGuard sg(split, kSplitBytes, h->sm_count);
  float* O = d.out;
  const float* omega = h->omega32;
  HM_TRY(forward_backward(net, omega, d.X, d.Y, c, s));
  HM_TRY(transpose_caches(net, c, N, ld, tq, s));
  std::vector<int4> tiles;
  for (int jm = 1; jm < L; ++jm) {
    const int Tin = net.T[jm - 1], Tout = net.T[jm];
    const int64_t boff = net.boff[jm - 1], rest = P - boff;
    RopBufs<float> rb = r;
    rb.B = Tout;
    {
      Tick t(h, HESS_K_ROP, 0.0, 0.0);
      HM_TRY(rop_block(net, omega, c, jm, boff, Tout, rb, s));
    }
    HM_TRY(transpose_rop(net, rb, jm, N, ld, tq, s));
    HM_TRY(build_layer_b(net, c, jm, N, ld, bhi, blo, s));
    // W x W block, a run of whole units at a time
    for (int p0 = 0; p0 < Tout;) {
      int p1 = p0 + 1;
      while (p1 < Tout && rows_before(p1 + 1, Tin, Tout) - rows_before(p0, Tin, Tout) <= arows_max) ++p1;
      const int64_t R0 = rows_before(p0, Tin, Tout);
      HM_TRY(build_wrows(net, tq, jm, p1, R0, ld, h->sm_count, ahi, alo, s));
      Job job{};
      bool untuned = false;
      const int BN = choose_bn(1, Tin, (int)(ld / BK), x3, &untuned);
      HM_TRY(make_job(TcOperands{ahi, alo, rows_before(p1, Tin, Tout) - R0, bhi, blo, Tin, ld}, BN, &job));
      tiles.clear();
      wrow_job(net, jm, p0, p1, R0, O, N, BN, job, tiles, 0);
      {
        Tick t(h, HESS_K_HCONTRACT, wrow_flops(Tin, Tout, p0, p1, N), 0.0);
        HM_TRY(launch_jobs(h->sm_count, &job, 1, tiles.data(), (int)tiles.size(), jd, tl, x3, h->err_dev, h->stage, s));
      }
      p0 = p1;
    }
    // columns after W: the bias of this layer and every later layer
    FArgs fa;
    HM_TRY(f_args(net, tq, jm, fa));
    for (int q0 = 0; q0 < Tout; q0 += pchunk) {
      const int pc = Tout - q0 < pchunk ? Tout - q0 : pchunk;
      HM_TRY(build_f(fa, q0, pc, ld, h->sm_count, fhi, flo, s));
      Job job{};
      bool untuned = false;
      const int BN = choose_bn(2, rest, (int)(ld / BK), x3, &untuned);
      HM_TRY(make_job(TcOperands{bhi, blo, Tin + 1, fhi, flo, (int64_t)pc * rest, ld}, BN, &job));
      tiles.clear();
      f_job(net, jm, q0, pc, O, N, BN, job, tiles, 0);
      {
        Tick t(h, HESS_K_HCONTRACT, f_flops(Tin, rest, pc, N), 0.0);
        HM_TRY(launch_jobs(h->sm_count, &job, 1, tiles.data(), (int)tiles.size(), jd, tl, x3, h->err_dev, h->stage, s));
      }
    }
  }
  if (!st.o_dev) HM_CUDA(cudaMemcpyAsync(Hout, O, P * P * 4, cudaMemcpyDeviceToHost, s));
  if (!st.o_dev || !st.x_dev || !st.y_dev) {
    // host buffers involved: the call waits for its work
    HM_CUDA(cudaStreamSynchronize(s));
    return take_sticky_error(h);
  }
  return HESS_OK;
}

// OPG = G^T G / N with split-BF16 (or BF16) operands on the tensor cores.
hess_status run_opg_tc(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3, void* Oout) {
  HM_TRY(tc_available(h));
  return run_single(h, X, Y, N, x3, Oout, 0);
}

// Exact Hessian on the tensor cores: one persistent launch over every weight
// layer's blocks when the whole operand set fits the handle's operand limit,
// else the chunked schedule.
hess_status run_hessian_tc(hess_mlp* h, const void* X, const void* Y, int64_t N, bool x3, void* Hout) {
  HM_TRY(tc_available(h));
  if (hessian_plan_bytes(h, N) <= h->op_limit) return run_single(h, X, Y, N, x3, Hout, 1);
  return run_hessian_chunked(h, X, Y, N, x3, Hout);
}

// ============================================ exact-digit FP64 products
// A FP64 product A A^T on the BF16 tensor cores (the splitting scheme of
// Ozaki et al.): each row r of A is scaled by 2^-e_r (its largest magnitude
// below 1) and written as eight signed integer digits,
//   a = 2^e_r sum_d q_d 2^(-6 - 7d),   |q_d| <= 64,
// exact to 2^-56 of the row's largest entry.  The digit products of equal
// weight, sum over d + d' = w of Q_d Q_d'^T, are one contraction over the
// digits laid side by side along K (Q_0 | Q_1 | ... against the reversed
// order Q_7 | ... | Q_0); a contraction spans at most 4096 products per
// entry, so with |q q'| <= 2^12 its FP32 sums stay below 2^24 and are exact.
// The few integer matrices are combined in FP64 with their weights
// 2^(e_r + e_c - 12 - 7w), smallest first.  Groups of contractions whose
// FP32 results fit a bounded buffer run one persistent launch each.
namespace {

constexpr int kDigits = 8;
constexpr size_t kPairBudget = (size_t)1 << 30;
constexpr int64_t kExactK = 4096;  // products per entry with exact FP32 sums

// round(x 2^(62 - E)) for |x| < 2^E, from the bits of x with integer
// operations only (an FP64 operation costs many cycles per warp on this GPU):
// x = mant 2^e, so the result is mant shifted by e + 62 - E (left by at most
// 9, since mant >= 2^52; right shifts round half up, and values below 2^-63
// of the scale vanish).
__device__ __forceinline__ long long fixed62(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long mant = bits & 0xfffffffffffffull;
  if (ex == 0 && mant == 0ull) return 0ll;
  int e;
  if (ex == 0) {
    e = -1074;  // subnormal
  } else {
    mant |= 1ull << 52;
    e = ex - 1075;
  }
  const int sh = e + 62 - E;
  long long v;
  if (sh >= 0) {
    v = (long long)(mant << sh);
  } else if (sh > -64) {
    const int r = -sh;
    v = (long long)((mant + (1ull << (r - 1))) >> r);
  } else {
    v = 0ll;
  }
  return (bits >> 63) ? -v : v;
}

struct JobWeightsFwd {
  double w[2 * kDigits * kDigits];  // 2^(-12 - 7w) of each contraction of the group
  int count;
};

// Row digits: fwd[r][d ldk + k] = q_d and rev[r][(7 - d) ldk + k] = q_d.  The
// row's value scaled into (-1, 1) becomes the integer m = v 2^62 (dropping
// below 2^-62), whose digits come off by rounding shifts.
// pm: plane-major digits of groups of gn rows: row r of group g = r / gn
// (ng = min(gn, n - g gn) rows) has digit d at pm + (g 8 gn + d ng + r - g gn) ldk.
// A block of 256 threads splits two rows, 128 threads per row, each thread
// two adjacent k at a time (4-byte stores of BF16 pairs).
constexpr int kDrRow = 128;
__global__ void __launch_bounds__(256) digits_rows_kernel(const double* A, int64_t rs, int64_t ks, int64_t n,
                                                          int64_t K, int64_t ldk, __nv_bfloat16* fwd,
                                                          __nv_bfloat16* rev, __nv_bfloat16* pm, int* ex,
                                                          int64_t gn) {
  __shared__ double smx[2][kDrRow / 32];
  const int rl = threadIdx.x / kDrRow, t = threadIdx.x % kDrRow, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 2 + rl;
  const bool live = r < n;
  const double* a = A + (live ? r : 0) * rs;  // element (r, k) = a[k * ks]
  double mx = 0.0;
  if (live) {
#pragma unroll 4
    for (int64_t k = t; k < K; k += kDrRow) mx = fmax(mx, fabs(a[k * ks]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smx[rl][t >> 5] = mx;
  __syncthreads();
  if (!live) return;
  mx = fmax(fmax(smx[rl][0], smx[rl][1]), fmax(smx[rl][2], smx[rl][3]));
  int E = 0;
  if (mx > 0.0 && mx <= DBL_MAX) frexp(mx, &E);  // mx = f 2^E, f in [0.5, 1)
  if (t == 0) ex[r] = E;
  const int64_t L = (int64_t)kDigits * ldk;
  __nv_bfloat16* fr = fwd ? fwd + r * L : nullptr;
  __nv_bfloat16* rr = rev ? rev + r * L : nullptr;
  const int64_t grp = r / gn, rg = r - grp * gn, ng = n - grp * gn < gn ? n - grp * gn : gn;
  __nv_bfloat16* pr = pm ? pm + (grp * kDigits * gn + rg) * ldk : nullptr;
#pragma unroll 2
  for (int64_t k = 2 * t; k < ldk; k += 2 * kDrRow) {  // ldk is even: k + 1 < ldk
    long long m0 = k < K ? fixed62(a[k * ks], E) : 0ll;  // |m| <= 2^62
    long long m1 = k + 1 < K ? fixed62(a[(k + 1) * ks], E) : 0ll;
#pragma unroll
    for (int d = 0; d < kDigits; ++d) {
      const int sh = 56 - 7 * d;
      const long long q0 = (m0 + (1ll << (sh - 1))) >> sh;  // round to nearest
      const long long q1 = (m1 + (1ll << (sh - 1))) >> sh;
      m0 -= q0 << sh;
      m1 -= q1 << sh;
      __nv_bfloat162 v;
      v.x = __int2bfloat16_rn((int)q0);  // |q| <= 64: exact
      v.y = __int2bfloat16_rn((int)q1);
      if (fr) *reinterpret_cast<__nv_bfloat162*>(fr + (int64_t)d * ldk + k) = v;
      if (rr) *reinterpret_cast<__nv_bfloat162*>(rr + (int64_t)(kDigits - 1 - d) * ldk + k) = v;
      if (pr) *reinterpret_cast<__nv_bfloat162*>(pr + (int64_t)d * ng * ldk + k) = v;  // rows (d, r) of the group
    }
  }
}

// max(m, |x|) on the bit patterns of doubles (integer order is the order of
// non-negative doubles); NaN is skipped, as fmax skips it
__device__ __forceinline__ unsigned long long max_abs_bits(unsigned long long m, double x) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return (a <= 0x7ff0000000000000ull && a > m) ? a : m;
}

// mx[c] = max_r |G[r][c]| as FP64 bits (non-negative doubles order as their
// bit patterns) for the columns of a row-major n x mg FP64 array G (the rows
// of G^T); mx is zeroed beforehand.  Block (32 x 8): 32 adjacent columns, 8
// slices of its share of the rows (gridDim.y shares), maxima on the integer
// pipe, one atomic per column and block.
__global__ void colmax_bits_kernel(const double* G, int64_t ldg, int64_t n, int64_t mg, unsigned long long* mx) {
  __shared__ unsigned long long red[8][33];
  const int64_t c = blockIdx.x * (int64_t)32 + threadIdx.x;
  unsigned long long v = 0ull;
  if (c < mg) {
    const int64_t step = (int64_t)gridDim.y * 8;
    int64_t r = (int64_t)blockIdx.y * 8 + threadIdx.y;
    for (; r + 3 * step < n; r += 4 * step) {
      double x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = G[(r + u * step) * ldg + c];
#pragma unroll
      for (int u = 0; u < 4; ++u) v = max_abs_bits(v, x[u]);
    }
    for (; r < n; r += step) v = max_abs_bits(v, G[r * ldg + c]);
  }
  red[threadIdx.y][threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.y == 0 && c < mg) {
    for (int y = 1; y < 8; ++y) v = red[y][threadIdx.x] > v ? red[y][threadIdx.x] : v;
    if (v) atomicMax(mx + c, v);
  }
}

// The exponent E with max_r |G[r][c]| = f 2^E, f in [0.5, 1) (0 for a zero or
// non-finite maximum); the all-ones columns c >= mg have E = 1.
__device__ __forceinline__ int col_exp(const unsigned long long* mx, int64_t c, int64_t mg) {
  if (c >= mg) return 1;
  const double v = __longlong_as_double((long long)mx[c]);
  int E = 0;
  if (v > 0.0 && v <= DBL_MAX) frexp(v, &E);
  return E;
}

// Digits of the rows of G^T (G row-major n x mg, then m - mg all-ones
// columns): fwd[c][d ldk + r] = q_d of G[r][c] scaled by 2^-ex[c], with ex[c]
// from the column maxima mx (written to ex by the blocks of the first row
// tile); rows r in [n, ldk) are zero.  A 128 x 32 tile (128 rows r, 32
// columns c) is read along c and written along r through shared memory, four
// consecutive r per thread (8-byte stores).
__global__ void digits_cols_kernel(const double* G, int64_t ldg, int64_t n, int64_t mg, int64_t m,
                                   const unsigned long long* mx, int* ex, int64_t ldk, __nv_bfloat16* fwd) {
  __shared__ double t[128][33];
  const int64_t r0 = (int64_t)blockIdx.x * 128, c0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 128; y += 8) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < n && c < m) ? (c < mg ? G[r * ldg + c] : 1.0) : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.y == 0 && c0 + threadIdx.x < m)
    ex[c0 + threadIdx.x] = col_exp(mx, c0 + threadIdx.x, mg);
  __syncthreads();
  const int64_t L = (int64_t)kDigits * ldk;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t c = c0 + y, r = r0 + 4 * threadIdx.x;
    if (c >= m || r >= ldk) continue;  // ldk is a multiple of 64: r..r+3 all in range
    const int e = col_exp(mx, c, mg);
    long long mm[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) mm[u] = fixed62(t[4 * threadIdx.x + u][y], e);
    __nv_bfloat16* fr = fwd + c * L + r;
#pragma unroll
    for (int d = 0; d < kDigits; ++d) {
      const int sh = 56 - 7 * d;
      __align__(8) __nv_bfloat16 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long q = (mm[u] + (1ll << (sh - 1))) >> sh;
        mm[u] -= q << sh;
        v[u] = __int2bfloat16_rn((int)q);
      }
      *reinterpret_cast<uint2*>(fr + (int64_t)d * ldk) = *reinterpret_cast<const uint2*>(v);
    }
  }
}

// Terms of a general digit product: the pairs (d, e), d + e <= 7, of a digit
// of A and one of B, numbered d-major with e ascending, kTerms per K segment.
constexpr int kTerms = kDigits * (kDigits + 1) / 2;
__host__ __device__ constexpr int term_of(int d, int e) { return kDigits * d - d * (d - 1) / 2 + e; }
__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// C = the combined terms of a general digit product whose Nt columns come in
// groups of Nn: group g (columns g Nn + c', c' < ng = min(Nn, Nt - g Nn)) keeps
// row r's terms side by side at T + g M nt Nn + r nt ng + (s kTerms + t) ng + c'
// (nt = nseg kTerms; s the K segment, t = term_of(d, e)).  The terms are
// integers below 2^24 in magnitude (at most 4096 products of digits in
// [-64, 64]), so those of one weight w = d + e are summed exactly as
// integers, and only the eight weighted sums, smallest weight first, are FP64
// operations: C(r, c) = 2^(exA_r + exB_c) sum_w 2^(-12 - 7 w) a_w, written to
// C[r scm + c scn].
__global__ void combine_terms_kernel(const float* T, int64_t M, int64_t Nn, int64_t Nt, int nseg, const int* exA,
                                     const int* exB, double* C, int64_t scm, int64_t scn) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * Nt) return;
  const int64_t r = idx / Nt, c = idx - r * Nt;
  const int64_t g = c / Nn, cc = c - g * Nn;
  const int64_t ng = Nt - g * Nn < Nn ? Nt - g * Nn : Nn;
  const int64_t nt = (int64_t)nseg * kTerms;
  const float* p = T + g * M * nt * Nn + r * nt * ng + cc;
  long long a[kDigits] = {};
  for (int sg = 0; sg < nseg; ++sg) {
    float v[kTerms];
#pragma unroll
    for (int t = 0; t < kTerms; ++t) v[t] = p[(int64_t)(sg * kTerms + t) * ng];
#pragma unroll
    for (int d = 0; d < kDigits; ++d)
#pragma unroll
      for (int e = 0; e < kDigits - d; ++e) a[d + e] += __float2int_rn(v[term_of(d, e)]);
  }
  double sum = 0.0;
#pragma unroll
  for (int w = kDigits - 1; w >= 0; --w) sum = fma((double)a[w], pow2i(-12 - 7 * w), sum);
  C[r * scm + c * scn] = ldexp(sum, exA[r] + exB[c]);
}

using JobWeights = JobWeightsFwd;

// Upper triangle (c >= r) of C = 2^(e_r + e_c) sum_j w_j T_j, added to C when
// accumulate is set; contractions in the order given (smallest weights
// first).
__global__ void combine_upper_kernel(const float* T, int64_t n, JobWeights jw, const int* ex, double* C, int64_t ldc,
                                     int accumulate) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = blockIdx.y;
  if (c >= n || c < r) return;
  const size_t plane = (size_t)n * n;
  double s = 0.0;
  for (int j = 0; j < jw.count; ++j) s = fma((double)T[(size_t)j * plane + (size_t)r * n + c], jw.w[j], s);
  s = ldexp(s, ex[r] + ex[c]);
  double* o = C + r * ldc + c;
  *o = accumulate ? *o + s : s;
}

// A BF16 tensor map over a column block of a wider row-major array: inner
// extent `inner` elements, rows `rows`, row stride `stride` elements.
hess_status make_block_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t stride, int64_t rows,
                           int box_rows) {
  using namespace tc;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (inner % BK) || (stride % 8))
    return set_error(HESS_ERR_INVALID_ARG, "tensor map: misaligned operand block");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)stride * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult res = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (res != CUDA_SUCCESS) return set_error(HESS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)res);
  return HESS_OK;
}

// The contractions: for each weight w = d + d' (0 .. 7), digits d in
// segments of at most kExactK / ldk.
struct Contraction {
  int w, d0, d1;
};
std::vector<Contraction> contractions(int64_t ldk) {
  const int seg = (int)std::max<int64_t>(1, kExactK / ldk);
  std::vector<Contraction> out;
  for (int w = kDigits - 1; w >= 0; --w)  // smallest weights first
    for (int d0 = 0; d0 <= w; d0 += seg) out.push_back({w, d0, std::min(w + 1, d0 + seg)});
  return out;
}

}  // namespace

bool f64_syrk_tc_eligible(hess_mlp* h, int64_t n, int64_t K) {
  if (K < 128 || K > kExactK || n < 128 || n > 16384) return false;
  if (tc_available(h) != HESS_OK) {
    clear_error();
    return false;
  }
  return true;
}

void plan_f64_syrk(Arena& ar, int64_t n, int64_t K, F64SyrkScratch& fs) {
  using namespace tc;
  fs.n = n;
  fs.ldk = (int64_t)align_up((size_t)K, BK);
  fs.D = ar.take<__nv_bfloat16>((int64_t)kDigits * n * fs.ldk);
  fs.R = ar.take<__nv_bfloat16>((int64_t)kDigits * n * fs.ldk);
  fs.ex = ar.take<int>(n);
  const int64_t njobs = (int64_t)contractions(fs.ldk).size();
  int64_t g = (int64_t)(kPairBudget / ((size_t)n * n * sizeof(float)));
  if (g < 1) g = 1;
  if (g > njobs) g = njobs;
  fs.group = (int)g;
  fs.T = ar.take<float>(g * n * n);
  fs.jobs = ar.take<tc::Job>(g);
  fs.tiles = ar.take<int4>(g * syrk_tile_count(n, 256));
}

hess_status f64_syrk_tc(hess_mlp* h, const double* A, int64_t lda, int64_t K, double* C, int64_t ldc,
                        const F64SyrkScratch& fs, cudaStream_t s, F64SyrkPlanes* defer) {
  using namespace tc;
  const int64_t n = fs.n, ldk = fs.ldk, L = (int64_t)kDigits * ldk;
  if (K > ldk) return set_error(HESS_ERR_INVALID_ARG, "exact-digit product: K %lld beyond its plan", (long long)K);
  {
    // (the only caller is the Gram matrix of the OPG eigen step)
    Tick t(h, HESS_K_GRAM, 0.0, 0.0);
    digits_rows_kernel<<<(unsigned)cdiv(n, 2), 256, 0, s>>>(A, lda, 1, n, K, ldk, fs.D, fs.R, nullptr, fs.ex, n);
    HM_LAUNCHED();
  }
  const std::vector<Contraction> cs = contractions(ldk);
  const int BN = 256;
  bool first = true;
  for (size_t j0 = 0; j0 < cs.size(); j0 += fs.group) {
    const size_t j1 = std::min(cs.size(), j0 + (size_t)fs.group);
    std::vector<Job> jobs;
    std::vector<int4> tiles;
    JobWeights jw{};
    jw.count = (int)(j1 - j0);
    for (size_t j = j0; j < j1; ++j) {
      const Contraction& c = cs[j];
      const int64_t inner = (int64_t)(c.d1 - c.d0) * ldk;
      const __nv_bfloat16* Ablk = fs.D + (int64_t)c.d0 * ldk;                       // Q_d0 | ... | Q_{d1-1}
      const __nv_bfloat16* Bblk = fs.R + (int64_t)(kDigits - 1 - c.w + c.d0) * ldk;  // Q_{w-d0} | ... | Q_{w-d1+1}
      Job job{};
      HM_TRY(make_block_map(&job.a_hi, Ablk, inner, L, n, BM));
      job.a_lo = job.a_hi;
      HM_TRY(make_block_map(&job.b_hi, Bblk, inner, L, n, BN));
      job.b_lo = job.b_hi;
      job.BN = BN;
      job.nkb = (int)(inner / BK);
      job.idesc = make_idesc(BN);
      job.M = n;
      job.Nn = n;
      job.mode = 0;  // upper tiles; the mirrored writes land below the diagonal, unread
      job.scale = 1.0f;
      job.chunk_kb = job.nkb;  // exact integer sums: no chunked accumulation
      job.out = fs.T + (j - j0) * (size_t)n * n;
      job.ldo = n;
      syrk_tiles(n, BN, (int)jobs.size(), tiles);
      jobs.push_back(job);
      jw.w[j - j0] = ldexp(1.0, -12 - 7 * c.w);
    }
    {
      double fl = 0.0;
      for (size_t j = j0; j < j1; ++j) fl += (double)n * (n + 1) * (double)(cs[j].d1 - cs[j].d0) * ldk;
      Tick t(h, HESS_K_DIGITS, fl, 0.0);
      HM_TRY(launch_jobs(h->sm_count, jobs.data(), (int)jobs.size(), tiles.data(), (int)tiles.size(), fs.jobs,
                         fs.tiles, false, h->err_dev, h->stage, s));
    }
    if (defer && j1 == cs.size() && jw.count <= kMaxSyrkPlanes) {
      defer->T = fs.T;
      defer->count = jw.count;
      for (int j = 0; j < jw.count; ++j) {
        defer->w[j] = jw.w[j];
        defer->wexp[j] = cs[j0 + j].w;
      }
      defer->ex = fs.ex;
      defer->part = first ? nullptr : C;
      defer->ldp = ldc;
      break;
    }
    {
      Tick t(h, HESS_K_GRAM, 0.0, 0.0);
      combine_upper_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)n), 256, 0, s>>>(fs.T, n, jw, fs.ex, C, ldc,
                                                                                     first ? 0 : 1);
      HM_LAUNCHED();
    }
    first = false;
  }
  return HESS_OK;
}

namespace {
int64_t k_segments(int64_t ldk) { return cdiv(ldk, kExactK); }
// Digit-major jobs of a general product with a group of ng columns: for each
// digit d of A, the digits e < kDigits - d of B in runs of at most 256 / ng
// (one tile column each); a run's terms are adjacent (term_of).
struct DigitJob {
  int d, e0, e1;
};
std::vector<DigitJob> digit_jobs(int64_t ng) {
  const int per = (int)std::max<int64_t>(1, 256 / ng);
  std::vector<DigitJob> out;
  for (int d = 0; d < kDigits; ++d)
    for (int e0 = 0; e0 < kDigits - d; e0 += per) out.push_back({d, e0, std::min(kDigits - d, e0 + per)});
  return out;
}
int64_t gemm_groups(int64_t Nn, int64_t Nt) { return cdiv(Nt, Nn); }
// jobs of all groups (each group's job count depends on its width)
int64_t gemm_job_count(int64_t Nn, int64_t Nt, int64_t nseg) {
  int64_t n = 0;
  for (int64_t c0 = 0; c0 < Nt; c0 += Nn) n += (int64_t)digit_jobs(std::min(Nn, Nt - c0)).size() * nseg;
  return n;
}
}  // namespace

bool f64_gemm_nt_tc_eligible(hess_mlp* h, int64_t M, int64_t Nn, int64_t K, int64_t Nt) {
  if (Nt < 0) Nt = Nn;
  if (K < 128 || M < 128 || Nn < 1 || Nn > 256 || Nt < 1) return false;
  // K in segments of at most kExactK products (exact FP32 sums each); every
  // term of every segment has its own FP32 result
  const int64_t ldk = (int64_t)align_up((size_t)K, tc::BK);
  const int64_t nt = k_segments(ldk) * kTerms;
  if ((double)M * nt * Nt * 4.0 > 8.0 * (1 << 30)) return false;  // FP32 results within 8 GB
  if (tc_available(h) != HESS_OK) {
    clear_error();
    return false;
  }
  return true;
}

void f64_gemm_nt_need(int64_t M, int64_t Nn, int64_t K, int64_t Nt, F64GemmNeed& nd) {
  using namespace tc;
  if (Nt < 0) Nt = Nn;
  const int64_t ldk = (int64_t)align_up((size_t)K, BK), nseg = k_segments(ldk);
  const int64_t nj = gemm_job_count(Nn, Nt, nseg);
  nd.M = std::max(nd.M, M);
  nd.Nt = std::max(nd.Nt, Nt);
  nd.ldk = std::max(nd.ldk, ldk);
  nd.t = std::max(nd.t, M * nseg * kTerms * Nt);
  nd.jobs = std::max(nd.jobs, nj);
  nd.tiles = std::max(nd.tiles, nj * cdiv(M, BM));
}

void plan_f64_gemm_nt(Arena& ar, const F64GemmNeed& nd, F64GemmScratch& fs) {
  fs.M = nd.M;
  fs.Mcap = nd.M;
  fs.Nt = nd.Nt;
  fs.ldk = nd.ldk;
  fs.DA = ar.take<__nv_bfloat16>((int64_t)kDigits * nd.M * nd.ldk);
  fs.RB = ar.take<__nv_bfloat16>((int64_t)kDigits * nd.Nt * nd.ldk);
  fs.exA = ar.take<int>(nd.M);
  fs.mxA = ar.take<unsigned long long>(nd.M);
  fs.exB = ar.take<int>(nd.Nt);
  fs.T = ar.take<float>(nd.t);
  fs.tsize = nd.t;
  fs.group = (int)nd.jobs;
  fs.ntiles = nd.tiles;
  fs.jobs = ar.take<tc::Job>(nd.jobs);
  fs.tiles = ar.take<int4>(nd.tiles);
}

hess_status f64_gemm_nt_split_a(const double* G, int64_t ldg, int64_t K, const F64GemmScratch& fs, cudaStream_t s,
                                int64_t Mg) {
  using namespace tc;
  const int64_t M = fs.M;
  const int64_t mg = Mg < 0 ? M : Mg;
  const int64_t ldk = (int64_t)align_up((size_t)K, BK);
  if (mg < 1 || mg > M || M > fs.Mcap || ldk > fs.ldk)
    return set_error(HESS_ERR_INVALID_ARG, "exact-digit product: bad operand of %lld x %lld", (long long)M,
                     (long long)K);
  // A = G^T: rows are the columns of G (rows [mg, M) all ones), split once
  HM_CUDA(cudaMemsetAsync(fs.mxA, 0, (size_t)M * sizeof(unsigned long long), s));
  const unsigned ry = (unsigned)std::max<int64_t>(1, std::min<int64_t>(16, cdiv(K, 64)));
  colmax_bits_kernel<<<dim3((unsigned)cdiv(mg, 32), ry), dim3(32, 8), 0, s>>>(G, ldg, K, mg, fs.mxA);
  HM_LAUNCHED();
  digits_cols_kernel<<<dim3((unsigned)cdiv(ldk, 128), (unsigned)cdiv(M, 32)), dim3(32, 8), 0, s>>>(
      G, ldg, K, mg, M, fs.mxA, fs.exA, ldk, fs.DA);
  HM_LAUNCHED();
  return HESS_OK;
}

hess_status f64_gemm_nt_tc(hess_mlp* h, const double* G, int64_t ldg, const double* B, int64_t b_rs, int64_t b_ks,
                           int64_t K, double* C, int64_t scm, int64_t scn, const F64GemmScratch& fs, cudaStream_t s,
                           int64_t Nn_total, int64_t Mg, bool a_split) {
  using namespace tc;
  const int64_t M = fs.M, Nn = fs.Nn;
  const int64_t Nt = Nn_total < 0 ? Nn : Nn_total;
  const int64_t mg = Mg < 0 ? M : Mg;  // columns of G; rows [mg, M) of A are ones
  if (mg < 1 || mg > M) return set_error(HESS_ERR_INVALID_ARG, "exact-digit product: bad column count of G");
  // this product's digit rows have its own length (the plan's is the longest)
  const int64_t ldk = (int64_t)align_up((size_t)K, BK), L = (int64_t)kDigits * ldk;
  const int64_t nseg = k_segments(ldk), nt = nseg * kTerms;
  const int64_t nj = gemm_job_count(Nn, Nt, nseg);
  if (M > fs.Mcap || ldk > fs.ldk || Nt > fs.Nt || M * nt * Nt > fs.tsize || nj > fs.group || nj * cdiv(M, BM) > fs.ntiles)
    return set_error(HESS_ERR_INVALID_ARG, "exact-digit product: %lld x %lld x %lld beyond its plan", (long long)M,
                     (long long)Nt, (long long)K);
  {
    // (the only caller is the back-projection of the OPG eigen step)
    Tick tp(h, HESS_K_BACKPROJ, 0.0, 0.0);
    // A = G^T (unless split beforehand) and B: rows (e, c') of each group of
    // Nn columns, plane-major; both split once
    if (!a_split) HM_TRY(f64_gemm_nt_split_a(G, ldg, K, fs, s, mg));
    digits_rows_kernel<<<(unsigned)cdiv(Nt, 2), 256, 0, s>>>(B, b_rs, b_ks, Nt, K, ldk, nullptr, nullptr, fs.RB,
                                                             fs.exB, Nn);
    HM_LAUNCHED();
  }
  std::vector<Job> jobs;
  std::vector<int4> tiles;
  for (int64_t c0 = 0, g = 0; c0 < Nt; c0 += Nn, ++g) {
    const int64_t ng = std::min(Nn, Nt - c0);
    float* Tg = fs.T + g * M * nt * Nn;
    const __nv_bfloat16* RBg = fs.RB + g * kDigits * Nn * ldk;
    const std::vector<DigitJob> js = digit_jobs(ng);
    for (int64_t sg = 0; sg < nseg; ++sg) {
      const int64_t k0 = sg * kExactK;
      const int64_t inner = std::min<int64_t>(kExactK, ldk - k0);  // a multiple of 64
      for (const DigitJob& dj : js) {
        const int j = (int)jobs.size();
        const int64_t cols = (int64_t)(dj.e1 - dj.e0) * ng;
        const int BN = (int)align_up((size_t)cols, 16);
        Job job{};
        HM_TRY(make_block_map(&job.a_hi, fs.DA + (int64_t)dj.d * ldk + k0, inner, L, M, BM));
        job.a_lo = job.a_hi;
        HM_TRY(make_block_map(&job.b_hi, RBg + (int64_t)dj.e0 * ng * ldk + k0, inner, ldk, cols, BN));
        job.b_lo = job.b_hi;
        job.BN = BN;
        job.nkb = (int)(inner / BK);
        job.idesc = make_idesc(BN);
        job.M = M;
        job.Nn = cols;
        job.mode = 3;
        job.scale = 1.0f;
        job.chunk_kb = job.nkb;  // exact integer sums: no chunked accumulation
        job.out = Tg + (sg * kTerms + term_of(dj.d, dj.e0)) * ng;
        job.ldo = nt * ng;
        for (int64_t tm = 0; tm < cdiv(M, BM); ++tm) tiles.push_back(make_int4(j, (int)tm, 0, 0));
        jobs.push_back(job);
      }
    }
  }
  {
    double fl = 0.0;
    for (const Job& jb : jobs) fl += 2.0 * (double)jb.M * jb.Nn * (double)jb.nkb * BK;
    Tick t(h, HESS_K_DIGITS, fl, 0.0);
    HM_TRY(launch_jobs(h->sm_count, jobs.data(), (int)jobs.size(), tiles.data(), (int)tiles.size(), fs.jobs,
                       fs.tiles, false, h->err_dev, h->stage, s));
  }
  Tick tc(h, HESS_K_BACKPROJ, 0.0, 0.0);
  combine_terms_kernel<<<(unsigned)cdiv(M * Nt, 256), 256, 0, s>>>(fs.T, M, Nn, Nt, (int)nseg, fs.exA, fs.exB, C,
                                                                   scm, scn);
  HM_LAUNCHED();
  return HESS_OK;
}

}  // namespace hm

extern "C" {

hess_status hess_autotune(int enable) {
  hm::clear_error();
  hm::g_tune_on.store(enable ? 1 : 0);
  return HESS_OK;
}

int hess_autotune_entries(void) {
  std::lock_guard<std::mutex> lk(hm::g_tune_mu);
  return (int)hm::g_tuned.size();
}

hess_status hess_autotune_save(const char* path) {
  hm::clear_error();
  if (!path) return hm::set_error(HESS_ERR_INVALID_ARG, "path is NULL");
  std::lock_guard<std::mutex> lk(hm::g_tune_mu);
  FILE* f = fopen(path, "w");
  if (!f) return hm::set_error(HESS_ERR_INVALID_ARG, "cannot write %s", path);
  fprintf(f, "# mode columns kblocks products3 width\n");
  for (const auto& kv : hm::g_tuned)
    fprintf(f, "%d %lld %d %d %d\n", kv.first.mode, (long long)kv.first.nn, kv.first.nkb, kv.first.x3, kv.second);
  fclose(f);
  return HESS_OK;
}

hess_status hess_autotune_load(const char* path) {
  hm::clear_error();
  if (!path) return hm::set_error(HESS_ERR_INVALID_ARG, "path is NULL");
  FILE* f = fopen(path, "r");
  if (!f) return hm::set_error(HESS_ERR_INVALID_ARG, "cannot read %s", path);
  std::lock_guard<std::mutex> lk(hm::g_tune_mu);
  char line[256];
  int bad = 0;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int mode, nkb, x3, bn;
    long long nn;
    if (sscanf(line, "%d %lld %d %d %d", &mode, &nn, &nkb, &x3, &bn) != 5 || mode < 0 || mode > 2 || bn < 16 ||
        bn > 256 || bn % 16 || nn < 1 || nkb < 1) {
      ++bad;
      continue;
    }
    hm::g_tuned[hm::TuneKey{mode, (int64_t)nn, nkb, x3 ? 1 : 0}] = bn;
  }
  fclose(f);
  if (bad) return hm::set_error(HESS_ERR_INVALID_ARG, "%d malformed lines in %s", bad, path);
  return HESS_OK;
}

}  // extern "C"
