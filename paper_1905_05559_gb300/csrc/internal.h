// Internal declarations shared by the translation units of libhessmlp.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <functional>
#include <vector>

#include "../../include/hessmlp.h"

namespace hm {

// ---------------------------------------------------------------- errors ----
hess_status set_error(hess_status s, const char* fmt, ...);
void clear_error();

#define HM_CUDA(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::hm::set_error(e_ == cudaErrorMemoryAllocation ? HESS_ERR_OOM : HESS_ERR_CUDA, \
                             "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                             __FILE__, __LINE__);                                       \
  } while (0)

#define HM_TRY(expr)                 \
  do {                               \
    hess_status s_ = (expr);         \
    if (s_ != HESS_OK) return s_;    \
  } while (0)

extern std::atomic<int64_t> g_launches;
#define HM_LAUNCHED()                                         \
  do {                                                        \
    ::hm::g_launches.fetch_add(1, std::memory_order_relaxed); \
    HM_CUDA(cudaGetLastError());                              \
  } while (0)

// Makes a device current for a scope.
struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------ workspace ----
// Two-pass bump allocator: a plan is run once with base == nullptr to size it,
// then again on the real buffer.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// --------------------------------------------------------------- network ----
constexpr int kMaxLayers = 32;

// Fixed-capacity description (no heap use, so it can be built by every entry
// point, including the allocation-free one).
struct Net {
  int L = 0;
  int T[kMaxLayers] = {};        // widths T_1..T_L stored at T[0..L-1]
  int act[kMaxLayers] = {};      // hidden activations for layers 2..L-1 at act[0..L-3]
  int64_t woff[kMaxLayers] = {}; // offset of W^(j) (j = 1..L-1) at woff[j-1]
  int64_t boff[kMaxLayers] = {}; // offset of b^(j+1) at boff[j-1]
  int64_t P = 0;
};

// Validate a description and fill a Net (HESS_ERR_INVALID_ARG on failure).
hess_status make_net(const hess_mlp_desc* desc, Net* net);

}  // namespace hm

namespace hm {
struct TimingRec {
  cudaEvent_t a, b;
  int cls;
  double flops, bytes;
  int sms;  // SMs the bracketed launches were given (0: all)
};
}  // namespace hm

namespace hm {
// Pinned host staging for the small tables a launch reads (jobs, tiles), so
// that their copies are asynchronous.  A slot's buffer is reused once its
// previous copy has completed (event).
struct PinnedSlot {
  char* p = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
};
// A ring of slots, so that a copy waits only for the one kStageSlots copies
// before it (not for the last): launches queued behind other work do not
// hold up the host.
constexpr int kStageSlots = 4;
struct PinnedStage {
  PinnedSlot slot[kStageSlots];
  int next = 0;
};
}  // namespace hm

namespace hm {
// The planning pass of a fused call (workspace size and region offsets), kept
// for the next call of the same shape so that the host queues work at once.
struct FusedPlanCache {
  bool valid = false;
  int64_t key[16] = {};
  size_t ws = 0, off_prep = 0, off_eig = 0;
};
}  // namespace hm

struct hess_mlp {
  hm::Net net;
  bool owns_params = true;  // false: omega64/omega32 borrowed from another handle
  bool timing = false;
  std::vector<hm::TimingRec> pending;
  std::vector<cudaEvent_t> event_pool;
  hess_kernel_stats acc[HESS_K_COUNT] = {};
  int device = 0;
  cudaStream_t stream = nullptr;
  double* omega64 = nullptr;  // device, P
  float* omega32 = nullptr;   // device, P
  char* ws = nullptr;         // device workspace
  size_t ws_bytes = 0;
  double* host_pinned = nullptr;  // small pinned scratch for scalars
  // sticky error flag in mapped pinned memory: kernels set it when a bounded
  // pipeline wait gives up; calls report it without synchronising
  int* err_host = nullptr;
  int* err_dev = nullptr;
  hm::PinnedStage stage;
  // second stream (the eigen step) and two copy streams (the matrices'
  // transfer to the host, each matrix in two halves, one per copy stream, so
  // that two copy engines share it) of the fused call, created on first use
  cudaStream_t stream2 = nullptr;
  cudaStream_t stream3 = nullptr;
  cudaStream_t stream4 = nullptr;
  // the fused call's stream for the Hessian's operand preparation
  cudaStream_t stream5 = nullptr;
  // the fused call's ordering events (created on first use, re-recorded by
  // every call)
  static constexpr int kFusedEvents = 13;
  cudaEvent_t fused_ev[kFusedEvents] = {};
  // batch object of hessian_minibatches (created on first use)
  hess_batch* mb_batch = nullptr;
  // second growable device buffer, for results that the single-call entry
  // points (which plan from the start of ws) must not overwrite
  char* ws2 = nullptr;
  size_t ws2_bytes = 0;
  int sm_count = 0;
  // operand bytes above which the tensor-core Hessian is built and contracted
  // in chunks (one launch per chunk) instead of in one launch
  size_t op_limit = (size_t)4 << 30;
  // blocks of the OPG eigen step's Lanczos kernel (0: one per SM)
  int lz_blocks = 0;
  hm::FusedPlanCache fplan;
};

namespace hm {

hess_status ensure_ws(hess_mlp* h, size_t bytes);
hess_status ensure_ws2(hess_mlp* h, size_t bytes);

// Host-side resources of a handle (pinned scratch, mapped error flag).
hess_status host_side_init(hess_mlp* h);
void host_side_free(hess_mlp* h);
// HESS_ERR_TIMEOUT (and clears the flag) if a kernel of an earlier call on
// the handle gave up a pipeline wait.
hess_status take_sticky_error(hess_mlp* h);
// *on_dev = 1 for device (or managed) memory of the handle's device, 0 for
// host memory; INVALID_ARG for another device's memory.
hess_status locate(const hess_mlp* h, const void* p, const char* name, int* on_dev);
// Copies n host tables through the pinned stage to device memory on s.
hess_status stage_copy(PinnedStage& st, const void* const* src, const size_t* bytes, void* const* dst, int n,
                       cudaStream_t s);
void stage_free(PinnedStage& st);

// Planning without work: while a dry run is active on this thread, ensure_ws
// records the workspace a call needs and makes the call return kDryRun before
// any GPU work is queued.
constexpr hess_status kDryRun = static_cast<hess_status>(100);
extern thread_local size_t* g_dry_bytes;

// Brackets launches with CUDA events when the handle's timing is enabled (a
// null handle times nothing).
class Tick {
 public:
  Tick(hess_mlp* h, int cls, double flops, double bytes);
  void set_work(double flops, double bytes) {
    rec_.flops = flops;
    rec_.bytes = bytes;
  }
  // the bracketed launches run on sms SMs (persistent grids confined to part
  // of the GPU)
  void set_sms(int sms) { rec_.sms = sms; }
  void stop();
  ~Tick() { stop(); }

 private:
  hess_mlp* h_;
  TimingRec rec_{};
  bool live_ = false;
};

// ------------------------------------------------------- SIMT launchers ----
// Generic strided GEMM: C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n),
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C(m,n) = C[m*scm + n*scn],
// batched over blockIdx.z with element strides bsa/bsb/bsc.  upper: M == N and
// only the tiles on or above the diagonal are computed.
template <typename T>
struct Gemm {
  int M = 0, N = 0, K = 0;
  T alpha = 1, beta = 0;
  const T* A = nullptr;
  int64_t sam = 0, sak = 0, bsa = 0;
  const T* B = nullptr;
  int64_t sbk = 0, sbn = 0, bsb = 0;
  T* C = nullptr;
  int64_t scm = 0, scn = 0, bsc = 0;
  int batch = 1;
  int upper = 0;
};
template <typename T>
hess_status gemm(const Gemm<T>& g, cudaStream_t s);

// Scratch for split-K partial tiles of the SIMT GEMM, set by each entry point
// from its workspace for the duration of the call (none: no split).  Guards
// nest: a call made inside another's scope restores the outer scratch.
struct SplitScratch {
  void* p = nullptr;
  size_t bytes = 0;
  int sms = 0;
};
extern thread_local SplitScratch g_split;
struct SplitGuard {
  explicit SplitGuard(void* p, size_t bytes, int sms) : prev_(g_split) { g_split = SplitScratch{p, bytes, sms}; }
  ~SplitGuard() { g_split = prev_; }

 private:
  SplitScratch prev_;
};
constexpr size_t kSplitBytes = (size_t)64 << 20;

// out[r] = alpha * sum_{n < K} A[n * lda + r]  for r < R (deterministic)
template <typename T>
hess_status colsum(const T* A, int64_t lda, int64_t R, int64_t K, T alpha, T* out, int64_t ostride,
                   cudaStream_t s);

// Forward/backward caches of one call (all device, row-major N x T_l).
template <typename T>
struct Caches {
  int64_t N = 0;
  const T* a[kMaxLayers] = {};  // a[j] j = 0..L-2 (a[0] = X)
  T* s1[kMaxLayers] = {};       // sigma' for hidden positions j = 1..L-2
  T* s2[kMaxLayers] = {};       // sigma''
  T* d[kMaxLayers] = {};        // delta for positions j = 1..L-1
  T* e[kMaxLayers] = {};        // W^T delta before sigma' for hidden j
  T* p = nullptr;               // softmax output N x T_L
  T* ysum = nullptr;            // row sums of Y (N)
  T* z = nullptr;               // scratch for pre-activations (N x max T)
};
template <typename T>
void plan_caches(Arena& ar, const Net& net, int64_t N, Caches<T>& c);
// df_wide (FP64 only): the products of layers with 128 or more inputs in
// double-float arithmetic (the eigen step's pass, whose later arithmetic is
// double-float too).
template <typename T>
hess_status forward_backward(const Net& net, const T* omega, const T* X, const T* Y, Caches<T>& c,
                             cudaStream_t s, bool df_wide = false);
template <typename T>
hess_status write_grads(const Net& net, const Caches<T>& c, T* G, int64_t ldg, cudaStream_t s);
template <typename T>
hess_status mirror_upper(T* C, int64_t n, int64_t ldc, cudaStream_t s);
template <typename T>
hess_status fill(T* p, int64_t n, T v, cudaStream_t s);
template <typename Ti, typename To>
hess_status convert(const Ti* in, To* out, int64_t n, cudaStream_t s);

// R-operator over a block of B unit directions d0..d0+B-1, all inside the
// parameters of weight layer jm (1-based, W^(jm) and b^(jm+1)).
template <typename T>
struct RopBufs {
  int B = 0;
  std::vector<T*> rz;  // positions j >= jm: B x N x T
  std::vector<T*> ra;  // hidden positions j >= jm
  std::vector<T*> rd;  // positions j >= jm
  T* tmp = nullptr;    // B x N x max T
  T* ones = nullptr;   // N ones (filled by the first hvp_block on these buffers)
  bool ones_ready = false;
};
template <typename T>
void plan_rop(Arena& ar, const Net& net, int64_t N, int jm, int B, RopBufs<T>& r);
template <typename T>
hess_status rop_block(const Net& net, const T* omega, const Caches<T>& c, int jm, int64_t d0, int B,
                      RopBufs<T>& r, cudaStream_t s);
// H v_d for B general directions (v_d = V + d ldv, result HV + d ldh); r
// planned with jm = 1.
template <typename T>
hess_status hvp_block(const Net& net, const T* omega, const Caches<T>& c, const T* V, int64_t ldv, int B,
                      RopBufs<T>& r, T* HV, int64_t ldh, cudaStream_t s);
// H[d][c] for the block's rows and the columns of weight layer jl (>= jm),
// kept where c >= d and mirrored to H[c][d] where c > d.  tmp: B x P_l.
template <typename T>
hess_status contract_layer(const Net& net, const Caches<T>& c, const RopBufs<T>& r, int jm, int jl,
                           int64_t d0, T* tmp, T* H, cudaStream_t s);
template <typename T>
hess_status scatter_sym(const T* tmp, int B, int64_t cols, int64_t c0, int64_t d0, T* H, int64_t P,
                        cudaStream_t s);

// -------------------------------------------------------- eigensolver ----
struct EigResult {
  int converged = 0;
  int rank_deficient = 0;
  int lanczos_steps = 0;
  double flops = 0.0;  // algorithmic FP64 flops of the Gram matrix, Lanczos and back-projection
};
// Top-k eigenpairs of the symmetric tridiagonal matrix with diagonal a[0..m-1]
// and off-diagonal b[0..m-2]: theta[c] = c-th largest eigenvalue (Sturm
// bisection), row c of Y (stride ldy) its unit eigenvector (inverse
// iteration; clusters closer than 1e-6 |theta_0| orthogonalised), res[c] =
// |beta_last y_c[m-1]| (the Lanczos residual bound), mx = {max res, |theta_0|}.
// scratch: tridiag_scratch_doubles(m, k) doubles (null when that is 0).
int64_t tridiag_scratch_doubles(int64_t mcap, int k);
hess_status tridiag_topk(const double* a, const double* b, int m, int k, double* theta, int* cstart, double* Y,
                         int64_t ldy, const double* beta_last, double* res, double* mx, uint64_t key,
                         double* scratch, cudaStream_t s);
// Blocks (one per SM) the Lanczos launches of the OPG eigen step take for N
// examples and k eigenpairs.
int eig_lanczos_blocks(hess_mlp* h, int64_t n, int k);
// after_gram (optional) runs once the Gram matrix's kernels and the first
// Lanczos launch are queued, before the host waits for that launch's result:
// the fused call queues its contractions there, behind side->gram_done.
// side (optional): a second stream with four events, for the parts of the
// eigen step that need not wait in line on the handle's stream (the
// back-projection's split of the activations into digits, which needs
// nothing but the forward pass, and the narrow layers' back-projection
// beside the wide layers'); gram_done (optional) is recorded on the
// handle's stream behind the Gram matrix.
struct EigSide {
  cudaStream_t s = nullptr;
  cudaEvent_t ev[4] = {};
  cudaEvent_t gram_done = nullptr;
};
hess_status topk_eig_gram(hess_mlp* h, const Net& net, const Caches<double>& c, int64_t N, int k,
                          double* evals_d, double* evecs_d, Arena& ar, bool dry, EigResult* res,
                          const std::function<hess_status()>* after_gram = nullptr, const EigSide* side = nullptr);
// Top-k eigenpairs of a resident symmetric n x n FP64 matrix M (row-major):
// the same Lanczos, tridiagonal eigensolver and checks as the Gram route;
// evecs_d row c = the unit eigenvector of evals_d[c] (sign canonicalised;
// zero when evals_d[c] <= 1e-13 evals_d[0], flagged in res->rank_deficient).
hess_status topk_eig_dense(hess_mlp* h, const double* M, int64_t n, int k, double* evals_d, double* evecs_d,
                           Arena& ar, bool dry, EigResult* res);

// ------------------------------------------------------ tensor cores ----
namespace tc {
// One contraction of the persistent tcgen05 kernel: its four operand tensor
// maps (bf16 hi/lo planes of A: M x K and B: Nn x K, K-major), K, and where its
// tiles land in a symmetric output.  A launch walks a list of tiles (job, row
// tile, column tile), so one launch serves many contractions of different
// shapes and networks.
struct Job {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  int64_t M;      // valid rows of A
  int64_t Nn;     // valid rows of B (= columns of the product)
  int BN;         // tile columns (multiple of 16, <= 256)
  int nkb;        // k-blocks of 64
  uint32_t idesc; // instruction descriptor (N = BN)
  int mode;       // 0: symmetric rank-K update (orow = m, ocol = n)
                  // 1: Hessian rows of one weight layer, W columns
                  // 2: Hessian rows of one weight layer (W rows and, from the
                  //    ones row of A, bias rows), columns after W
                  // 3: a general product (orow = m, ocol = n, no mirror)
  float scale;
  float* out;
  int64_t ldo;
  int64_t woff;   // modes 1, 2: offset of W in omega
  int64_t boff;   // mode 2: first column (the layer's bias)
  int Tin, Tout, p0;
  int64_t R0;     // mode 1: first concatenated row of unit p0
  int ntn;        // mode 2: column tiles per unit
  int64_t brow;   // mode 2: B rows per unit
  int chunk_kb;   // k-blocks per TMEM accumulation chunk (0: CHUNK_KB; exact
                  // integer products take the whole K in one chunk)
};
}  // namespace tc

// Scratch of an exact-digit FP64 product A A^T on the tensor cores (n rows,
// K columns): digit planes, row exponents, the FP32 results of a group of
// digit pairs, and the launch tables.
struct F64SyrkScratch {
  int64_t n = 0, ldk = 0;
  __nv_bfloat16* D = nullptr;  // digits side by side along K, and reversed
  __nv_bfloat16* R = nullptr;
  int* ex = nullptr;
  float* T = nullptr;
  int group = 1;
  tc::Job* jobs = nullptr;
  int4* tiles = nullptr;
};
// Usable when the tensor-core path is (sm_103, tensor-map encoder),
// 128 <= K <= 4096 (exact FP32 sums of the digit products) and
// 128 <= n <= 16384.
bool f64_syrk_tc_eligible(hess_mlp* h, int64_t n, int64_t K);
void plan_f64_syrk(Arena& ar, int64_t n, int64_t K, F64SyrkScratch& fs);
// The digit planes of the last group of an exact-digit A A^T, left for the
// caller to combine: entry (r, c), c >= r, of the product is
//   part[r ldp + c] (when part is set) + 2^(ex[r] + ex[c]) s,
//   s = fma(T_j, w_j, s) over j = 0 .. count - 1 in turn from s = 0,
// T_j = T[j n^2 + r n + c] (exact FP32 integers).
constexpr int kMaxSyrkPlanes = 36;  // digit pairs with d + d' <= 7
struct F64SyrkPlanes {
  const float* T = nullptr;
  int count = 0;
  double w[kMaxSyrkPlanes] = {};
  int wexp[kMaxSyrkPlanes] = {};  // w[j] = 2^(-12 - 7 wexp[j]); equal wexp adjacent
  const int* ex = nullptr;
  const double* part = nullptr;  // the earlier groups, combined (C)
  int64_t ldp = 0;
};
// Upper triangle (and diagonal) of C = A A^T for row-major FP64 A (n x K,
// stride lda), accurate to FP64 rounding; C's lower triangle is not written.
// With defer set, the last group of digit planes is not combined: its planes
// are described there instead (C then holds the earlier groups only, and
// defer->part points to it when there were any).
hess_status f64_syrk_tc(hess_mlp* h, const double* A, int64_t lda, int64_t K, double* C, int64_t ldc,
                        const F64SyrkScratch& fs, cudaStream_t s, F64SyrkPlanes* defer = nullptr);

// Scratch of an exact-digit FP64 product C = G^T B^T on the tensor cores
// (G: K x M row-major, B rows of length K): digits of the rows of G^T
// (side by side along K) and of B (reversed), exponents, the FP32 results of
// a group of contractions, and the launch tables.
struct F64GemmScratch {
  int64_t M = 0, Nn = 0, Nt = 0, ldk = 0;
  __nv_bfloat16* DA = nullptr;
  __nv_bfloat16* RB = nullptr;
  int *exA = nullptr, *exB = nullptr;
  unsigned long long* mxA = nullptr;  // column maxima of G (bits)
  float* T = nullptr;
  int64_t Mcap = 0;   // rows of A the plan has room for
  int64_t tsize = 0;  // floats of T
  int group = 1;      // room for digit jobs
  int64_t ntiles = 0; // room for tiles
  tc::Job* jobs = nullptr;
  int4* tiles = nullptr;
};
// The scratch several products need (the largest of each part): add each
// product with f64_gemm_nt_need, then take it with plan_f64_gemm_nt.  A
// product run on the plan sets the scratch's M and Nn to its own.
struct F64GemmNeed {
  int64_t M = 0, Nt = 0, ldk = 0, t = 0, jobs = 0, tiles = 0;
};
// Usable when the tensor-core path is, K >= 128 (in segments of at most
// 4096, each with exact FP32 sums), M >= 128 and 1 <= Nn <= 256 (one tile
// column per group of columns), and the FP32 results of the Nt columns
// (default Nn) fit their bound.
bool f64_gemm_nt_tc_eligible(hess_mlp* h, int64_t M, int64_t Nn, int64_t K, int64_t Nt = -1);
void f64_gemm_nt_need(int64_t M, int64_t Nn, int64_t K, int64_t Nt, F64GemmNeed& nd);
void plan_f64_gemm_nt(Arena& ar, const F64GemmNeed& nd, F64GemmScratch& fs);
// C(m, c) = sum_k G[k][m] B(c, k), B(c, k) = B[c b_rs + k b_ks], written to
// C[m scm + c scn], accurate to FP64 rounding; c < Nn_total (default: the
// plan's Nn; at most its Nt), in groups of the plan's Nn columns, all in one
// tensor-core launch.  With Mg < M, G has Mg columns and the rows m >= Mg of
// G^T are all ones (C's row m then sums B's row over k).
// a_split: A's digits were formed by f64_gemm_nt_split_a (same G, K, fs, Mg)
// earlier in stream order.
hess_status f64_gemm_nt_tc(hess_mlp* h, const double* G, int64_t ldg, const double* B, int64_t b_rs, int64_t b_ks,
                           int64_t K, double* C, int64_t scm, int64_t scn, const F64GemmScratch& fs, cudaStream_t s,
                           int64_t Nn_total = -1, int64_t Mg = -1, bool a_split = false);
// The digit split of A = G^T alone (fs.DA, fs.exA), on stream s.
hess_status f64_gemm_nt_split_a(const double* G, int64_t ldg, int64_t K, const F64GemmScratch& fs, cudaStream_t s,
                                int64_t Mg = -1);

// Jobs and tiles gathered for one persistent launch.
struct TcPlan {
  std::vector<tc::Job> jobs;
  std::vector<int64_t> caps;  // per job: its tiles at the narrowest candidate width
  std::vector<int4> tiles;    // (job, row tile, column tile, 0)
  int64_t tiles_cap = 0;      // tiles at the narrowest candidate width (table room)
  double syrk_flops = 0.0, hess_flops = 0.0;
};
// The first `nfirst` jobs of `both` (with their tiles and the SYRK flops) and
// the others (re-indexed, with the Hessian flops), for separate launches.
void tc_split_plan(const TcPlan& both, int nfirst, TcPlan& first, TcPlan& rest);

// One network's request: device X (N x T_1), Y (N x T_L) and the P x P
// device outputs of the requested matrices (the pointers are not consulted to
// decide what is requested: a planning pass may pass placeholders).
struct TcItem {
  const float* X = nullptr;
  const float* Y = nullptr;
  int64_t N = 0;
  bool want_opg = false, want_hess = false;
  float* opg = nullptr;
  float* hess = nullptr;
  bool x3 = true;  // split-BF16 (three products) or BF16 (one)
};

hess_status tc_available(hess_mlp* h);
// Lays out (live = false) or builds (live = true, on stream s) everything the
// item's contractions read: forward/backward caches, split-BF16 operands, and
// the Hessian entries outside the tensor-core blocks; appends the item's
// jobs to the plan.  The caller provides the split-K scratch (SplitGuard).
// With a fork (live calls), the Hessian's part runs on fork->s: it waits
// for the forward/backward pass on s (event after_fb), and 'done' is recorded
// behind it, so that the OPG's contraction need not wait for it.
struct TcFork {
  cudaStream_t s = nullptr;
  cudaEvent_t after_fb = nullptr;
  cudaEvent_t done = nullptr;
};
hess_status tc_prep(hess_mlp* h, const TcItem& it, Arena& ar, bool live, TcPlan& plan, cudaStream_t s,
                    const TcFork* fork = nullptr);
// Takes arena memory for the plan's job and tile tables; when live, copies
// them there and starts one persistent launch over all tiles (longest first).
hess_status tc_launch_plan(int sm_count, const TcPlan& plan, Arena& ar, bool live, bool x3, int* err,
                           PinnedStage& stage, cudaStream_t s);

}  // namespace hm
