/*
 * hessmlp.h -- C ABI of the GB300 curvature-matrix library.
 *
 * Computes, for a dense feed-forward network with softmax cross-entropy cost
 * (Nilsen et al., "Efficient Computation of Hessian Matrices in TensorFlow",
 * Sec. 2: Eq. modelfunc, Eq. cost), the per-example gradient matrix G, the
 * outer product of gradients OPG = G^T G / N (Sec. 3, Eq. hesseq2/hesseq3),
 * the exact Hessian H (Sec. 3, Eq. hesseq1; built from Hessian-vector
 * products with unit directions, Sec. 5.1 and Appendix A.1) and the top-k
 * eigenpairs of the OPG (Sec. 4.1, Sec. 5.4, Eq. J).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Network:   layers l = 1..L with widths T_1..T_L; weight layer l-1 maps
 *            layer l-1 to layer l: z^(l) = W^(l-1) a^(l-1) + b^(l), with
 *            W^(l-1) of shape T_l x T_{l-1}; hidden layers apply sigma^(l),
 *            the output layer applies softmax (Sec. 2).
 * Parameters: omega has P = sum_{l=2..L} (T_{l-1} T_l + T_l) entries, laid out
 *            layer by layer as W^(l-1) row-major (entry (i,j) at offset
 *            i*T_{l-1} + j) followed by b^(l) (Sec. 2, Eq. flatten, read as a
 *            row-wise flatten of each matrix).  Every row and column index of
 *            G, OPG, H and of the eigenvectors follows this order.
 * Inputs:    X is N x T_1 row-major, Y is N x T_L row-major one-hot labels.
 *            Rows may be any non-negative label vector: the library computes
 *            dC_n/dz^(L) = p_n (sum_m y_nm) - y_n and scales the softmax
 *            curvature diag(p_n) - p_n p_n^T by sum_m y_nm, which is the
 *            exact derivative of C_n = (sum_m y_nm) logsumexp(z^(L)) - y_n . z^(L)
 *            (Eq. cost) and equals p_n - y_n for one-hot rows.
 * Precision: HESS_FP64 -- X, Y and outputs are double; all arithmetic FP64.
 *            HESS_FP32 -- X, Y and outputs are float; arithmetic FP32 (the
 *                         softmax log-sum-exp in FP64).
 *            HESS_BF16, HESS_BF16X3 -- X, Y and outputs are float; forward and
 *                         backward passes in FP32; the OPG and Hessian
 *                         contractions on the tensor cores with BF16 operands
 *                         (one product) or split-BF16 operands
 *                         (hi*hi + hi*lo + lo*hi) and FP32 accumulation.
 * Memory:    every data pointer may point to host or device memory; the
 *            library asks the CUDA runtime which.  Device pointers must be on
 *            the handle's device.  The caller owns every buffer it passes;
 *            the handle owns omega's device copy and all workspace.
 * Streams:   work is queued on the handle's stream.  A call whose pointers are
 *            all device pointers returns without waiting; a call with any host
 *            pointer waits for its own work before returning.
 * Errors:    every entry point returns a hess_status; nothing aborts or
 *            throws.  Arguments are checked before any work is queued.
 *            hess_last_error() gives a message for the calling thread's most
 *            recent failure.  The tensor-core kernels bound every pipeline
 *            wait; one that gives up sets a flag on the handle that the call
 *            reports as HESS_ERR_TIMEOUT when it waits for its work, and
 *            otherwise the next call on the handle reports.
 * Threads:   a handle must not be used by two threads at once.
 */
#ifndef HESSMLP_H
#define HESSMLP_H

#include <stdint.h>

#if defined(__GNUC__)
#define HESS_API __attribute__((visibility("default")))
#else
#define HESS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HESS_OK = 0,
  HESS_ERR_INVALID_ARG = 1,    /* bad pointer, size, enum or layout */
  HESS_ERR_OOM = 2,            /* device allocation failed */
  HESS_ERR_CUDA = 3,           /* a CUDA runtime or kernel error */
  HESS_ERR_RANK_DEFICIENT = 4, /* opg_topk_eig: some of the k eigenvalues are
                                  null (results still written) */
  HESS_ERR_NOT_CONVERGED = 5,  /* opg_topk_eig: iteration limit reached */
  HESS_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  HESS_ERR_ADMISSION = 7,      /* request exceeds the memory budget */
  HESS_ERR_UNSUPPORTED = 8     /* valid request the library cannot serve (e.g. a precision the call lacks) */
} hess_status;

typedef enum { HESS_ACT_SIGMOID = 0, HESS_ACT_TANH = 1, HESS_ACT_RELU = 2 } hess_act;

typedef enum { HESS_FP64 = 0, HESS_FP32 = 1, HESS_BF16 = 2, HESS_BF16X3 = 3 } hess_precision;

typedef struct hess_mlp hess_mlp;

/* Network description (Sec. 2).  widths: L entries T_1..T_L (L >= 2, each
 * T_l >= 1, T_L >= 2); act: L-2 hidden activations (may be NULL when L == 2).
 * The arrays are copied at create time. */
typedef struct {
  int L;
  const int* widths;
  const int* act; /* hess_act values */
} hess_mlp_desc;

/* Create a handle for the network and parameter point omega (P doubles, host or
 * device, order of Eq. flatten).  omega is copied to the device (FP64 and FP32
 * copies); the caller keeps ownership of its buffer.  stream: a cudaStream_t
 * (NULL = the legacy default stream).  The current CUDA device becomes the
 * handle's device.  Errors: INVALID_ARG (bad desc, NULL out/omega),
 * OOM, CUDA. */
HESS_API hess_status hess_mlp_create(const hess_mlp_desc* desc, const double* omega, void* stream,
                            hess_mlp** out);

/* Release the handle and its device memory (waits for its stream first).
 * NULL is accepted and ignored. */
HESS_API hess_status hess_mlp_destroy(hess_mlp* h);

/* P, the number of parameters (Sec. 2, after Eq. flatten); -1 for NULL. */
HESS_API int64_t hess_mlp_num_params(const hess_mlp* h);

/* Replace the parameter point (P doubles, host or device). */
HESS_API hess_status hess_mlp_set_params(hess_mlp* h, const double* omega);

/* Change the stream used by later calls. */
HESS_API hess_status hess_mlp_set_stream(hess_mlp* h, void* stream);

/* Device bytes of split-BF16 operands above which the tensor-core Hessian
 * (BF16/BF16X3) is built and contracted in chunks, one launch per chunk,
 * instead of all at once in one launch (default 4 GiB; at least 1 MiB).
 * Results do not depend on it. */
HESS_API hess_status hess_mlp_set_operand_limit(hess_mlp* h, int64_t bytes);

/* Blocks (one per SM) the Lanczos kernel of the OPG eigen step uses when the
 * Gram matrix's rows fit shared memory (0, the default: 8/15 of the SMs).
 * The kernel is bound by the latency of its grid barriers rather than by
 * arithmetic, so a grid smaller than the GPU costs it little and leaves SMs
 * to work that overlaps it: hess_curvature runs its contractions there.
 * Results depend on it only through the rounding of the Lanczos sums (the
 * same setting gives the same bits). */
HESS_API hess_status hess_mlp_set_eig_blocks(hess_mlp* h, int blocks);

/* Per-example gradient matrix (Sec. 3.1 and Sec. 5.2 "get_J_op"; the matrix J
 * of Eq. hesseq3 read with one example per ROW): G is N x P row-major,
 * G[n, :] = dC_n/domega^T with C_n the per-example cross-entropy of Eq. cost.
 * Precision FP64 (double X, Y, G) or FP32 (float X, Y, G); BF16/BF16X3 are
 * accepted and compute as FP32.  N >= 1.  Errors: INVALID_ARG, OOM, CUDA. */
HESS_API hess_status per_example_grads(hess_mlp* h, const void* X, const void* Y, int64_t N,
                              hess_precision prec, void* G);

/* OPG = (1/N) sum_n g_n g_n^T = G^T G / N (Sec. 3, Eq. hesseq2 and hesseq3),
 * written in full (both triangles) as a P x P row-major matrix, double for
 * FP64 and float otherwise.  The contraction is a symmetric rank-N update:
 * FP64/FP32 on the SIMT pipes, BF16/BF16X3 on the tensor cores.  The 1/N
 * weighting always uses the true N.  Errors: INVALID_ARG, OOM, CUDA. */
HESS_API hess_status opg(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec,
                void* OPG);

/* Exact Hessian H = (1/N) sum_n d^2 C_n / domega domega^T (Sec. 3, Eq.
 * hesseq1), P x P row-major, both triangles, double for FP64 and float
 * otherwise.  Computed as in Sec. 5.1 from Hessian-vector products with the
 * unit vectors of R^P, batched over blocks of directions: each block runs the
 * forward-over-reverse R-operator (Pearlmutter; Appendix A.1 shows the
 * product equals the second derivative applied to the direction) and a
 * contraction over the N examples.  Errors: INVALID_ARG, OOM, CUDA. */
HESS_API hess_status exact_hessian(hess_mlp* h, const void* X, const void* Y, int64_t N,
                          hess_precision prec, void* H);

/* Top-k eigenpairs of the OPG (Sec. 4.1 low-rank factors, Sec. 5.4 Eq. J):
 * with M = G G^T / N (N x N), the OPG eigenvalues are the eigenvalues mu of M
 * and the eigenvectors are q = G^T u / sqrt(N mu).  evals: k doubles in
 * descending (algebraic) order; evecs: P x k column-major doubles (column c is
 * q_c, unit norm, sign chosen so that its largest-magnitude entry is
 * positive).  X and Y are double for FP64 and float otherwise; for every
 * precision the Gram matrix, the eigensolver (Lanczos with full
 * reorthogonalisation, tridiagonal eigenpairs) and the back-projection are
 * held to FP64 accuracy: exact-digit FP64 products on the tensor cores for
 * the wide layers, and, where the Gram matrix's rows fit shared memory
 * (N up to about 2048), double-float arithmetic (pairs of FP32 numbers,
 * about 48 significant bits) for the Gram matrix, the Lanczos vectors and
 * the wide layer's forward product, the eigenvalues then refined in FP64.
 * Requires 1 <= k <=
 * min(N, P).  Returns HESS_ERR_RANK_DEFICIENT (after writing every output)
 * when mu_c <= 1e-13 mu_1 for some c; those columns are zero.  Errors:
 * INVALID_ARG, OOM, CUDA, NOT_CONVERGED. */
HESS_API hess_status opg_topk_eig(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                         hess_precision prec, double* evals, double* evecs);

/* Top-k OPG eigenpairs for data sets whose N x P gradient matrix is not held
 * at once (Sec. 5.4 works through mini-batches of examples; here uncentred,
 * as Eq. J states).  The examples are taken in chunks of `chunk`; each
 * chunk's OPG comes from opg() in precision prec (so at most one chunk's
 * gradients exist at a time) and is added, weighted by its share of the
 * examples, into a P x P FP64 sum, whose top-k eigenpairs come from the same
 * FP64 Lanczos, tridiagonal eigensolver and checks as opg_topk_eig.  Needs
 * P^2 doubles of device memory (a second workspace the handle keeps) but no
 * N x N Gram matrix, so N may exceed what opg_topk_eig accepts.  X, Y in the
 * precision's dtype, host or device (host chunks are staged one at a time);
 * evals/evecs as in opg_topk_eig.  Requires 1 <= k <= min(N, P).  Waits for
 * its work.  Errors: those of opg() and opg_topk_eig. */
HESS_API hess_status opg_topk_eig_streaming(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                            hess_precision prec, int64_t chunk, double* evals, double* evecs);

/* Top-k OPG eigenpairs in O(k P) device memory (Sec. 5.4 and Sec. 6: the
 * OPG eigenpairs from passes over mini-batches of examples with memory
 * O(K P); here uncentred, as Eq. J states, and converged rather than
 * truncated).  Neither G (N x P), nor the Gram matrix (N x N), nor the OPG
 * (P x P) is formed: each pass over the examples, in chunks of `chunk`,
 * applies OPG = (1/N) sum G_c^T G_c to a block of `block` vectors (0: the
 * default, min(max(k, 16), 128)) through per-layer GEMMs with the chunk's
 * forward/backward quantities; a block Krylov method with Rayleigh-Ritz
 * extraction and thick restarts keeps at most max(6 block, k + 3 block)
 * basis vectors and stops when every one of the top k Ritz residuals
 * ||OPG q - mu q|| is at most tol mu_1 (tol = 1e-10 for HESS_FP64, 1e-5 for
 * HESS_FP32, the precision of the products; the basis and the projected
 * eigenproblem are FP64 in both).  Device memory: about 2 (6 block + k) P
 * doubles plus one chunk's caches and two chunk x (T_out block) arrays.
 * X, Y in the precision's dtype, host or device (host data is staged chunk
 * by chunk, every pass); evals/evecs as in opg_topk_eig; *passes (may be
 * NULL) receives the number of passes over the data.  Requires 1 <= k <=
 * min(N, P).  Waits for its work.  Errors: INVALID_ARG (also for BF16
 * precisions), OOM, CUDA, NOT_CONVERGED (after 300 passes),
 * RANK_DEFICIENT (as opg_topk_eig), TIMEOUT. */
HESS_API hess_status opg_topk_eig_lowmem(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                         hess_precision prec, int64_t chunk, int block, double* evals,
                                         double* evecs, int* passes);


/* OPG (Eq. hesseq2, hesseq3), exact Hessian (Eq. hesseq1) and top-k OPG
 * eigenpairs (Sec. 5.4, Eq. J) of one data set in one call (any of them may
 * be left out: OPG or H NULL, k = 0).  The same results as
 * opg(), exact_hessian() and opg_topk_eig() with the same arguments, but
 * scheduled across five streams for BF16/BF16X3: the tensor-core operands and
 * contractions on the handle's stream, the FP64 eigen step (Gram matrix,
 * Lanczos, back-projection) concurrently on a second, higher-priority stream,
 * the copies of host outputs behind their contractions, each matrix in two
 * halves on a third and a fourth stream, and the Hessian's operands and the
 * eigen step's side work on a fifth; all of it is ordered before the
 * handle's stream's later work.
 * X, Y float (double for HESS_FP64), host or device; OPG and H as in
 * opg()/exact_hessian(); evals/evecs as in opg_topk_eig().  Other precisions,
 * or nothing to overlap, run the single calls in turn.  When every buffer is
 * device memory the call waits only for the Lanczos process's convergence
 * flags (and the Ritz values that decide HESS_ERR_RANK_DEFICIENT), not for
 * the rest of the work.  Errors: those of the three calls. */
HESS_API hess_status hess_curvature(hess_mlp* h, const void* X, const void* Y, int64_t N, hess_precision prec,
                                    void* OPG, void* H, int k, double* evals, double* evecs);

/* Hessian-vector products H v_d for b directions (Sec. 5.1: the exact
 * Hessian's columns are its products with the unit vectors; here any
 * directions).  Each product applies the R-operator (Appendix A) to the
 * forward pass and to the per-example back-propagation of every example and
 * averages over the N examples, without forming H.  V and HV: b x P row-major
 * (direction d is the P-vector V + d P, in the parameter order of Eq.
 * flatten), host or device.  X, Y, V and HV are double for HESS_FP64, float
 * for HESS_FP32 (the arithmetic's precision); BF16 precisions return
 * HESS_ERR_UNSUPPORTED.  Directions are processed in blocks sized to the
 * workspace.  Waits for its work when a buffer is host memory.  Errors:
 * INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
HESS_API hess_status hessian_vector_products(hess_mlp* h, const void* X, const void* Y, int64_t N,
                                             hess_precision prec, const void* V, int b, void* HV);

/* The k algebraically largest eigenpairs of the exact Hessian (Sec. 5.3:
 * Lanczos on the operator v -> H v, never forming H).  FP64 Lanczos with full
 * reorthogonalisation, extended until every top-k Ritz pair's residual bound
 * is below 1e-10 ||T_m||; the products H q run in FP64 (HESS_FP64: X, Y
 * double) or FP32 (HESS_FP32: X, Y float).  evals: k doubles, descending;
 * evecs: P x k column-major doubles (column c unit norm, largest-magnitude
 * entry positive).  steps (may be NULL) receives the Krylov dimension used.
 * Requires 1 <= k <= P.  Waits for its work.  Errors: INVALID_ARG,
 * UNSUPPORTED (BF16 precisions), OOM, CUDA, NOT_CONVERGED (Krylov dimension
 * cap min(P, 8k + 1024) reached; the outputs then hold the current Ritz
 * pairs). */
HESS_API hess_status hessian_topk_eig(hess_mlp* h, const void* X, const void* Y, int64_t N, int k,
                                      hess_precision prec, double* evals, double* evecs, int* steps);

/* Mini-batch (bs > 1) or per-example (bs = 1) Hessians (Sec. 5.1: feeding a
 * mini-batch, or one example, to the Hessian operation yields the average of
 * the per-example Hessians over it): H_b = (1/n_b) sum over examples n of
 * batch b of d^2 C_n / d omega d omega^T for the consecutive batches of bs
 * examples (n_b = bs except the last).  H: ceil(N / bs) row-major P x P
 * matrices back to back, dtype of the precision.  For BF16/BF16X3 with every
 * buffer in device memory the batches run through a batch object the handle
 * keeps (waves of one persistent tensor-core launch; each matrix
 * bit-identical to exact_hessian on its slice); otherwise one exact_hessian
 * call per batch.  Waits for its work.  Errors: those of exact_hessian. */
HESS_API hess_status hessian_minibatches(hess_mlp* h, const void* X, const void* Y, int64_t N, int64_t bs,
                                         hess_precision prec, void* H);

/* Low-rank and full-rank approximations of a curvature matrix from K of its
 * eigenpairs (Sec. 4.1: H~ = Q diag(lam) Q^T; Sec. 4.2: H~~ = H~ +
 * lam_tilde (I - Q Q^T), the other P - K eigenvalues replaced by lam_tilde,
 * positive definite when lam_tilde > 0).  evals: K doubles; evecs: P x K
 * column-major doubles with orthonormal columns (the outputs of
 * hessian_topk_eig or opg_topk_eig), host or device.  full = 0 for H~, 1 for
 * H~~; lam_tilde = NaN takes lam_K (the paper's choice).  P is the handle's.
 *
 * hess_approx_form writes the P x P matrix (row-major, exactly symmetric):
 * double for HESS_FP64, float for HESS_FP32 (computed in that precision);
 * BF16 precisions return HESS_ERR_UNSUPPORTED.
 *
 * hess_approx_apply applies the operator without forming it (Sec. 5.5, 5.6):
 * for each row x of X (b x P row-major doubles), HX row = H~ x (or H~~ x) and
 * quad = x^T H~ x (or x^T H~~ x); HX or quad may be NULL.  FP64.
 *
 * Both wait for their work when a buffer is host memory.  Errors:
 * INVALID_ARG (K outside 1 .. P, b < 1, NULL buffers), UNSUPPORTED, OOM,
 * CUDA. */
HESS_API hess_status hess_approx_form(hess_mlp* h, int K, const double* evals, const double* evecs, int full,
                                      double lam_tilde, hess_precision prec, void* out);
HESS_API hess_status hess_approx_apply(hess_mlp* h, int K, const double* evals, const double* evecs, int full,
                                       double lam_tilde, const double* X, int b, double* HX, double* quad);

/* Host helper: perm[i] = the index in the order of Eq. flatten of the i-th
 * parameter in "augmented row" order, where each output unit's weight row is
 * followed by its bias ([W_i,: , b_i] for every layer).  perm has P entries. */
HESS_API hess_status hess_param_permutation(int L, const int* widths, int64_t* perm);

/* Allocation-free per-example gradients (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc -- their device memory belongs to
 * another allocator (a framework's caching allocator, a fixed pool with a hard
 * budget), or they run a latency-bound loop where an allocation, with its
 * implicit synchronisation and possible failure, is not acceptable.  Computes
 * the same G as per_example_grads in FP64 (N x P row-major, one row per
 * example) without a handle and without allocating: desc describes the
 * network (validated as in hess_mlp_create); omega (at least P doubles), X
 * (at least N x T_1), Y (at least N x T_L) and G (at least N x P) must all be
 * device memory on the current device.  The call checks each pointer's
 * device and that its allocation extends far enough past it; a buffer carved
 * out of a larger allocation (a caching allocator's segment) cannot be
 * checked more closely than that, so its size is the caller's promise.
 * The forward/backward caches live in a file-scope device array of 32 MiB
 * that every GPU loading the library holds until the process exits; a request
 * whose caches exceed it, N * (4 (T_2 + ... + T_{L-1}) + (T_2 + ... + T_L) +
 * T_L + max_l T_l + 1) doubles plus alignment, is rejected with
 * HESS_ERR_INVALID_ARG before any GPU work.  The array's device address
 * belongs to a CUDA context: the first call under each context (the device's
 * primary context, a new one after cudaDeviceReset, or a caller's own
 * driver-API context) looks it up with cudaGetSymbolAddress while that
 * context is current and caches it under the context's handle; make that
 * first call before any stream capture.  Work is queued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call returns
 * without waiting.  All calls share the array: calls whose work overlaps on
 * the GPU (on different streams or from different threads) race on it. */
HESS_API hess_status per_example_grads_noalloc(const hess_mlp_desc* desc, const double* omega,
                                               const double* X, const double* Y, int64_t N,
                                               double* G, void* stream);

/* ----------------------------------------------------------------------
 * Request server (no counterpart in the paper: the paper computes one matrix
 * per call).  Continuous batching on one GPU: requests for Hessians, OPGs and
 * top-k OPG eigenpairs of registered networks are admitted in arrival order
 * as soon as a slot is free and their workspace fits the memory budget; each
 * slot runs on its own CUDA stream, so admitted requests overlap on the
 * device.  Network weights stay on the device.  Results are the same as the
 * single calls above (same kernels, deterministic).
 * -------------------------------------------------------------------- */
typedef struct hess_server hess_server;

typedef enum { HESS_REQ_HESSIAN = 0, HESS_REQ_OPG = 1, HESS_REQ_EIG = 2 } hess_request_kind;

typedef struct {
  int kind;         /* hess_request_kind */
  int net;          /* id returned by hess_server_add_network */
  const void* X;    /* N x T_1, host or device; must stay valid until the wait returns */
  const void* Y;    /* N x T_L */
  int64_t N;
  int prec;         /* hess_precision */
  int k;            /* HESS_REQ_EIG: number of eigenpairs */
  void* out;        /* P x P (Hessian, OPG) or P x k column-major doubles (eigenvectors) */
  double* evals;    /* HESS_REQ_EIG: k doubles */
} hess_request;

/* slots: concurrent requests (1..64); budget_bytes: device memory the slots'
 * workspaces may hold together.  The current device becomes the server's. */
HESS_API hess_status hess_server_create(int slots, int64_t budget_bytes, hess_server** out);

/* Copy a network and its parameter point to the device; net_id names it in
 * requests.  Errors as hess_mlp_create. */
HESS_API hess_status hess_server_add_network(hess_server* s, const hess_mlp_desc* desc,
                                             const double* omega, int* net_id);

/* Queue a request.  Its arguments are checked and its workspace planned at
 * once: HESS_ERR_ADMISSION if it alone exceeds the budget, the usual errors
 * for bad arguments.  ticket identifies it for hess_server_wait. */
HESS_API hess_status hess_server_submit(hess_server* s, const hess_request* req, int64_t* ticket);

/* Wait up to timeout_seconds (< 0: no limit) for a request; *result is the
 * status the request's call returned.  HESS_ERR_TIMEOUT if it is not done
 * (the ticket stays valid); a finished ticket is released by this call. */
HESS_API hess_status hess_server_wait(hess_server* s, int64_t ticket, double timeout_seconds,
                                      hess_status* result);

/* hess_server_wait, and the request's device times: *gpu_start_ms and
 * *gpu_end_ms (either may be NULL) receive the times, in ms since the server
 * was created, of CUDA events recorded on the request's slot stream just
 * before and just after its work was queued (so the interval spans the
 * request's kernels on the device); -1 if they could not be read. */
HESS_API hess_status hess_server_wait_timed(hess_server* s, int64_t ticket, double timeout_seconds,
                                            hess_status* result, double* gpu_start_ms, double* gpu_end_ms);

/* Finish the running requests, fail the queued ones, release everything. */
HESS_API hess_status hess_server_destroy(hess_server* s);

/* ----------------------------------------------------------------------
 * Tile-width autotuning of the tensor-core contractions (no counterpart in
 * the paper).  By default each contraction's tile width comes from a cost
 * model.  With tuning on, the first contraction of each shape (mode, output
 * columns, K blocks, BF16 or split-BF16) that a call meets is run alone at
 * every candidate width (64 .. 256) on its real operands -- its output is
 * written each time, with the same values -- and the fastest width is kept
 * for the rest of the process.  Tuning synchronises the calling stream and
 * is skipped inside a CUDA-graph capture.  The table can be saved and loaded
 * (text, one "mode columns kblocks products3 width" line per shape).
 * -------------------------------------------------------------------- */
HESS_API hess_status hess_autotune(int enable);
HESS_API int hess_autotune_entries(void);
HESS_API hess_status hess_autotune_save(const char* path);
/* Errors: INVALID_ARG for an unreadable file or malformed lines (the valid
 * lines are still loaded). */
HESS_API hess_status hess_autotune_load(const char* path);

/* ----------------------------------------------------------------------
 * Batched curvature matrices (no counterpart in the paper, which computes the
 * matrices of one network per call).  The OPG and/or exact Hessian of many
 * networks, each with its own data, in waves: a wave builds the operands of
 * as many items (in list order) as fit the batch's workspace, then contracts
 * every item of the wave in ONE persistent tensor-core launch.  An item whose
 * operands exceed the workspace alone runs by itself through opg() and
 * exact_hessian().  Each matrix is bit-identical to the single-network call
 * at the same precision.
 * -------------------------------------------------------------------- */
typedef struct hess_batch hess_batch;

typedef struct {
  hess_mlp* net;      /* network and parameter point (its stream is not used) */
  const float* X;     /* N x T_1 row-major, device */
  const float* Y;     /* N x T_L row-major one-hot, device */
  int64_t N;          /* >= 1 */
  float* opg;         /* P x P row-major device output, or NULL */
  float* hessian;     /* P x P row-major device output, or NULL */
} hess_batch_item;

typedef struct {
  int waves;          /* persistent tensor-core launches */
  int items_chunked;  /* items run alone (larger than the workspace) */
  int64_t tiles;      /* output tiles of the wave launches */
  double flops;       /* tensor-core flops of the wave launches (3 products for BF16X3) */
  double launch_ms;   /* summed device time of the wave launches (CUDA events) */
  int graph_replayed; /* 1 when the run replayed a captured CUDA graph */
} hess_batch_info;

/* workspace_bytes: device memory the batch allocates now and reuses for every
 * wave (at least 65 MiB; the wave size follows from it).  stream: cudaStream_t
 * for all batch work.  The current device becomes the batch's.  Errors:
 * INVALID_ARG, OOM, CUDA. */
HESS_API hess_status hess_batch_create(int64_t workspace_bytes, void* stream, hess_batch** out);

/* Computes every requested matrix of items[0..count).  All buffers must be
 * device memory on the batch's device; at least one output per item.
 * Precision BF16 or BF16X3 (INVALID_ARG otherwise).  Every item is checked
 * before any work is queued.  Waits for its work before returning; info (may
 * be NULL) receives the wave statistics.  Errors: INVALID_ARG, OOM, CUDA,
 * TIMEOUT (a pipeline wait of the tensor-core kernel gave up). */
HESS_API hess_status hess_batch_run(hess_batch* b, const hess_batch_item* items, int count,
                                    hess_precision prec, hess_batch_info* info);

/* CUDA graphs for repeated runs (off by default).  With graphs on, the second
 * run of an item list (the same handles, buffers, N and precision; buffer
 * contents may change) captures all of its waves -- every forward/backward
 * pass, operand builder and persistent launch -- into one CUDA graph, and
 * later runs of that list replay it with a single launch.  The graphs of the
 * 8 most recently used lists are kept.  Lists with an item too large for the
 * workspace run directly.  Errors: INVALID_ARG, CUDA. */
HESS_API hess_status hess_batch_set_graphs(hess_batch* b, int enable);

/* Waits for the batch stream and releases the workspace.  NULL is ignored. */
HESS_API hess_status hess_batch_destroy(hess_batch* b);

/* ----------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper).  When timing is enabled
 * the library brackets every launch of the kernel classes below with CUDA
 * events on the handle's stream, and records the algorithmic work of each
 * launch (flops of the contraction, or bytes that must cross HBM).
 * hess_timing_read waits for the handle's stream, returns the totals since
 * the last read for one class and resets them.
 * -------------------------------------------------------------------- */
typedef enum {
  HESS_K_SYRK = 0,      /* OPG contraction G^T G / N */
  HESS_K_HCONTRACT = 1, /* Hessian contraction over the N examples */
  HESS_K_GRADS = 2,     /* per-example gradient rows (HBM write) */
  HESS_K_ROP = 3,       /* R-operator over a block of directions */
  HESS_K_EIG = 4,       /* Gram matrix, Lanczos and back-projection */
  HESS_K_HREST = 5,     /* Hessian columns outside the tensor-core blocks */
  HESS_K_HVP = 6,       /* Hessian-vector products over a block of directions */
  HESS_K_HLANCZOS = 7,  /* Lanczos steps on the Hessian operator (products,
                           reorthogonalisation) and its Ritz vectors */
  HESS_K_APPROX = 8,    /* low-/full-rank approximations: forming, applying */
  /* parts of the OPG eigen step (HESS_K_EIG brackets the whole step; these
   * bracket pieces of it): */
  HESS_K_GRAM = 9,      /* Gram matrix: SIMT FP64 products, digit splitting
                           and FP64 combines of the exact-digit products,
                           Hadamard updates; flops = FP64 work of the Gram
                           matrix */
  HESS_K_DIGITS = 10,   /* the exact-digit products' tensor-core launches
                           (Gram term and back-projection); flops = BF16
                           digit-product flops */
  HESS_K_LANCZOS = 11,  /* the Lanczos launches on the Gram matrix; flops =
                           sum over steps j of 2 N^2 + 8 N (j + 1) */
  HESS_K_TRIDIAG = 12,  /* eigenpairs of the tridiagonal T_m */
  HESS_K_BACKPROJ = 13, /* Ritz vectors and back-projection; flops =
                           2 N m k + 2 P N k */
  HESS_K_LOWMEM = 14,   /* opg_topk_eig_lowmem: the passes over the data
                           (flops 4 N P b per pass); its basis updates and
                           projected eigenproblems count as HESS_K_EIG */
  HESS_K_COUNT = 15
} hess_kernel_class;

typedef struct {
  int64_t launches;
  double ms;    /* summed device time of the bracketed launches */
  double flops; /* summed algorithmic flops */
  double bytes; /* summed algorithmic HBM bytes */
  double sm_ms; /* summed device time x SMs the launches were given (the
                   whole GPU unless a launch was confined to fewer) */
} hess_kernel_stats;

HESS_API hess_status hess_timing_enable(hess_mlp* h, int enable);
HESS_API hess_status hess_timing_read(hess_mlp* h, int kernel_class, hess_kernel_stats* out);

/* Test hooks (no counterpart in the paper).
 *
 * hess_check_devmath: for n device doubles x, writes six rows of n device
 * doubles to out (6 n entries, row-major): the refined FP64 reciprocal the
 * eigensolvers use (hardware estimate plus two Newton-Raphson steps; within
 * one ulp of 1/x), CUDA's correctly rounded 1.0 / x, the refined reciprocal
 * square root (within two ulps), and 1.0 / sqrt(x) (the last two 0 where
 * x <= 0); then the hi and lo FP32 words of the double-float split that the
 * double-float kernels take from the bits of an FP64 input (hi: x with its
 * significand cut to 24 bits; hi + lo = x to 2^-48 relative for |x| in
 * [2^-74, 2^128); both 0 for |x| below 2^-126).  The refined forms are meant
 * for |x| in [2^-1022, 2^1022]: the estimate flushes subnormal inputs and
 * results to zero, so outside that range they return 0 (|x| > 2^1022) or a
 * value that is not finite (subnormal x).  Queued on `stream`; returns
 * without waiting.  Errors: INVALID_ARG.
 *
 * hess_debug_set_barrier_limit: the number of SM clock cycles a block of the
 * OPG eigen step's cooperative Lanczos kernel waits at a grid barrier before
 * it gives up (the kernel then stops and the call returns HESS_ERR_TIMEOUT);
 * cycles <= 0 restores the default of 4e9 cycles (about 2 s).  Process-wide;
 * affects launches queued after it returns.  Meant for tests that make the
 * wait run out.  Errors: none.
 *
 * hess_probe_fp64: a measurement kernel of the current device, 4 blocks of
 * 256 threads per SM, each thread running eight independent chains of iters
 * FP64 fused multiply-adds; *flops receives the launch's flop count (2 per
 * FMA), so that flops over the launch's duration (timed by the caller with
 * events on `stream`) is the device's FP64 issue rate.  sink: device memory
 * for one double, never written in practice.  Queued on `stream`; returns
 * without waiting.  Errors: INVALID_ARG, CUDA. */
HESS_API hess_status hess_check_devmath(const double* x, int64_t n, double* out, void* stream);
HESS_API hess_status hess_debug_set_barrier_limit(int64_t cycles);
HESS_API hess_status hess_probe_fp64(int64_t iters, double* flops, double* sink, void* stream);

/* Number of kernels this library has launched in the process so far. */
HESS_API int64_t hess_launch_count(void);

/* Message for the calling thread's most recent error ("" if none). */
HESS_API const char* hess_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HESSMLP_H */
