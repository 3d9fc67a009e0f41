/*
 * ruqlp.h -- C ABI of the GB300 RU-QLP library (libruqlp.so).
 *
 * Randomized Unpivoted QLP (arXiv 2209.12464, Section III, Algorithms 1-2),
 * in the right-sketch orientation: for A (m x n) and a Gaussian test matrix
 * Omega (n x d, d = k + p) the library computes
 *
 *     Y = A Omega;  Q = orth(Y);
 *     q times:  Z = A^T Q;  Q~ = orth(Z);  Y = A Q~;  Q = orth(Y);   (Alg. 2)
 *     B^T = A^T Q;  [P, R_B] = qr(B^T);  L = R_B^T                   (Alg. 1)
 *
 * so that A ~= Q L P^T with Q (m x d), P (n x d) orthonormal and L (d x d)
 * lower triangular; |diag(L)| estimate sigma_1..sigma_d of A (Section III-A,
 * Theorem 1).  This is the paper's Algorithm 1 + 2 applied to A^T with
 * Phi = Omega, stopped before its d x d QR of R^T (Algorithm 1, step 5);
 * that last QR is available with ruqlp_params.finish_paper.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  Sizes are element counts.  "Device" pointers
 *     are CUDA device memory on the handle's device; "host" pointers are CPU
 *     memory (pinned or pageable).
 *   - The caller owns every buffer it passes (A, Omega, outputs); the
 *     library owns only its workspace arena.  Buffers must stay valid until
 *     the call returns (ruqlp_decompose*) or until ruqlp_poll reports
 *     completion (ruqlp_submit).
 *   - Errors are returned as ruqlp_status; nothing is thrown or aborted
 *     across the ABI.  Invalid arguments give RUQLP_ERR_INVALID and leave the
 *     outputs untouched; ruqlp_last_error(h) returns a message.
 *   - A handle is not reentrant: one thread at a time per handle, except
 *     ruqlp_submit / ruqlp_poll, which are thread-safe.
 */
#ifndef RUQLP_H
#define RUQLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ruqlp_ctx* ruqlp_handle;

typedef enum {
  RUQLP_OK = 0,
  RUQLP_NOT_READY = 1,      /* ruqlp_poll: request still running */
  RUQLP_ERR_INVALID = 2,    /* bad argument (sizes, pointers, dtype) */
  RUQLP_ERR_BUDGET = 3,     /* workspace would exceed the HBM budget */
  RUQLP_ERR_CUDA = 4,       /* a CUDA runtime / launch error */
  RUQLP_ERR_BREAKDOWN = 5,  /* orth() failed even after its fallbacks (not
                               returned since the TSQR fallback exists) */
  RUQLP_ERR_TIMEOUT = 6     /* a bounded device wait ran out */
} ruqlp_status;

typedef enum {
  RUQLP_F64 = 0,   /* IEEE binary64 */
  RUQLP_F32 = 1,   /* IEEE binary32 */
  RUQLP_BF16 = 2   /* bfloat16 (8-bit exponent, 7-bit mantissa) */
} ruqlp_dtype;

/* Output flags (ruqlp_outputs.flags), OR-ed over all orth() calls. */
#define RUQLP_FLAG_SHIFTED 0x1u    /* a Cholesky broke down; the shifted
                                      CholeskyQR3 path was taken */
#define RUQLP_FLAG_RANKDEF 0x2u    /* CholeskyQR could not orthonormalise a
                                      sketch: a pivot failed even after the
                                      shift, or the last pass of a final basis
                                      met a Gram far from I (a pivot outside
                                      [1/2, 2]) -- the sketch is numerically
                                      rank deficient at the working precision
                                      (e.g. an exactly rank-k A with d > k).
                                      The decomposition was then redone with
                                      Householder TSQR (RUQLP_FLAG_TSQR). */
#define RUQLP_FLAG_TSQR 0x4u       /* every orth() of the returned result was
                                      a Householder TSQR (Section II-A's
                                      unpivoted QR; Demmel et al. 2012): after
                                      RUQLP_FLAG_RANKDEF, or with the
                                      "orth_tsqr" option */

typedef struct {
  int device;               /* CUDA device ordinal */
  size_t hbm_budget_bytes;  /* cap on the workspace arena (0 = no cap) */
  int max_slots;            /* serving: requests in flight at once (0 = 8) */
  void* cuda_stream;        /* cudaStream_t the work is ordered on (NULL =
                               the legacy default stream) */
} ruqlp_config;

/* Dense A, row-major, leading dimension ld >= n (elements). */
typedef struct {
  int64_t m, n, ld;
  ruqlp_dtype dtype;
  const void* data;
} ruqlp_dense;

/* Sparse A in CSR: rowptr[m+1] non-decreasing from 0 to nnz, colidx[nnz] in
 * [0, n) and strictly increasing inside each row, values[nnz] of dtype (F32
 * or BF16; products are accumulated in FP32).  m, n and nnz must fit int32.
 * The library checks this structure on the device and returns INVALID when
 * it fails; the transposed products use a CSC copy built in the workspace,
 * which allows at most 1024 nonzeros per column. */
typedef struct {
  int64_t m, n, nnz;
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* values;
  ruqlp_dtype dtype;
} ruqlp_csr;

/* Low-rank term of a sparse input (is_csr = 2): A = S + X D Y^T with S the
 * CSR part, X (m x r), D (r x r), Y (n x r), FP32, row-major with leading
 * dimension r, device memory, 1 <= r <= 4096.  The term is applied through
 * products -- A W = S W + X (D (Y^T W)), A^T W = S^T W + Y (D^T (X^T W)) --
 * and never formed, keeping the sparse path's O(sd) cost (Section III-D)
 * plus O((m + n) r d).  Not accepted by ruqlp_decompose_host. */
typedef struct {
  int64_t r;
  const float* X;
  const float* D;
  const float* Y;
} ruqlp_lowrank;

typedef struct {
  int is_csr;          /* 0: dense, 1: csr, 2: csr plus a low-rank term */
  ruqlp_dense dense;
  ruqlp_csr csr;
  ruqlp_lowrank lr;
} ruqlp_matrix;

/* k >= 1 (target rank), p >= 0 (oversampling), d = k + p with
 * d <= min(m, n) (Section III-A asks d < n; d = n is accepted and exact),
 * q >= 0 power steps (Algorithm 2; q = 0 is Algorithm 1 alone).
 * compute: precision A is streamed in.  F64: everything in FP64.  F32: A,
 * sketches and Q/P in FP32.  BF16: A in BF16 through the tensor cores with
 * FP32 accumulation; sketches and Q/P kept in FP32.  d x d Grams and R_B are
 * accumulated in FP64 in every mode; the Cholesky factorisations are FP64 on
 * the FP64 path and FP32 (shifted CholeskyQR3) on the FP32/BF16 paths unless
 * the "orth_fp64" option is set.  compute must equal A's dtype.
 * BF16 inputs use the tensor cores when A's leading dimension is a multiple
 * of 8 elements and A is 16-byte aligned (sketches wider than 256 columns
 * run as column chunks, one pass over A each); otherwise CUDA cores.
 * omega: n x d row-major FP64 Gaussian test matrix (device memory for
 * ruqlp_decompose / ruqlp_submit; host memory for ruqlp_decompose_host), or
 * NULL: then the library generates it on the device from omega_seed with
 * the counter-based generator of ruqlp_omega (no host copy of Omega).
 * finish_paper: 1 = also take the d x d QR of L, [P~, R~] = qr(L)
 * (Algorithm 1, step 5, in the paper's orientation).  On return Q holds
 * Q P~ and L holds R~ (UPPER triangular), so A ~= Q L P^T still holds and
 * diag(L) are the paper's L-values of A^T (Corollary 1).
 * 2 = the SVD-like finish of Section III-C (Remark 1): L = U S V^T by
 * one-sided Jacobi (in the work precision, on one SM); on return Q holds
 * Q U, P holds P V and L holds diag(S) (descending), so A ~= Q L P^T is an
 * approximate truncated SVD.  d <= 512. */
typedef struct {
  int k, p, q;
  ruqlp_dtype compute;
  const double* omega;
  int finish_paper;
  uint64_t omega_seed;
} ruqlp_params;

/* Q: m x d, L: d x d (dense, zero upper triangle), P: n x d, all row-major
 * with leading dimension d, in out_dtype (F64 or F32).  flags: written by
 * the library (RUQLP_FLAG_*). */
typedef struct {
  void* Q;
  void* L;
  void* P;
  ruqlp_dtype out_dtype;
  uint32_t flags;
} ruqlp_outputs;

/* Create a handle on cfg->device.  No workspace is allocated until the first
 * decomposition (or ruqlp_reserve).  Errors: INVALID (NULL args, bad
 * device), CUDA. */
ruqlp_status ruqlp_create(ruqlp_handle* h, const ruqlp_config* cfg);

/* Free the handle and its workspace (waits for its work to finish). */
ruqlp_status ruqlp_destroy(ruqlp_handle h);

/* Point the handle at another stream (cudaStream_t as void*). */
ruqlp_status ruqlp_set_stream(ruqlp_handle h, void* cuda_stream);

/* Set a tuning option of the handle.  Known names:
 *   "orth_fp64": 1 = on the FP32/BF16 paths, orth() runs CholeskyQR2 with
 *   FP64 products in the Gram and an FP64 Cholesky (slow on GB300's FP64
 *   units); 0 (default) = shifted CholeskyQR3 in FP32 with FP64 sums across
 *   row slabs.  The FP64 path always uses the FP64 form.
 *   "orth_full": 1 = on the FP32/BF16 paths every orth() of the power loop
 *   takes three CholeskyQR passes (shifted CholeskyQR3); 0 (default) =
 *   orth() results that only feed the next product take two (shifted, then
 *   plain; same span, and in exact arithmetic the final Q, L, P are
 *   identical because the bases differ by upper-triangular factors); the
 *   last Q and P always take three.
 *   "bf16_simt": 1 = run BF16 products on the CUDA cores instead of the
 *   tensor cores (comparison baseline); 0 (default) = tensor cores.
 *   "orth_simt": 1 = orth() of tall matrices (>= 8192 rows) forms its Grams
 *   and Q = Y R^{-1} on the CUDA cores (FP32 Gram tiles, blocked triangular
 *   solve); 0 (default) = on the tensor cores (three-way BF16 split of the
 *   FP32 operands, FP32 accumulation: FP32-level results).
 *   "batch_orth_tc": 1 = in ruqlp_decompose_batch, BF16 items with
 *   k + p <= 80 run their CholeskyQR passes (Grams, Q = Y R^{-1}) on the
 *   tensor cores, as tall single matrices do (ignored with "orth_simt" or
 *   "bf16_simt" = 1); 0 (default) = on the CUDA cores.
 *   "profile": 1 = bracket every phase with CUDA events on the handle's
 *   stream and accumulate their durations (read with ruqlp_profile); setting
 *   it (to 0 or 1) also zeroes the accumulators.
 * Errors: INVALID (unknown name). */
ruqlp_status ruqlp_set_option(ruqlp_handle h, const char* name, int64_t value);
/* (continued) "test_withhold_stage": test hook, off by default.  1 = in each
 *   tensor-core product that follows, the first CTA never loads its first
 *   shared-memory stage, so the MMA warp's bounded wait (2 s) runs out and the
 *   call returns RUQLP_ERR_TIMEOUT after the CTA has drained its copies and
 *   freed its tensor memory; the handle stays usable.  Exercises the timeout
 *   path without faulting or hanging the GPU.
 * (continued) "tc_nsplit": column split of the tensor-core products: 0
 *   (default) = chosen per product shape by the library's tuner (below);
 *   1, 2, 4 = that split (each 128-row tile of the output taken as that many
 *   items of dp / split columns by consecutive CTAs; needs dp / split to be a
 *   multiple of 16, else the product returns RUQLP_ERR_CUDA).
 * (continued) "orth_tsqr": 1 = every orth() is a Householder TSQR (leaf QRs
 *   of row blocks, a binary tree of stacked-R QRs, explicit Q; Demmel,
 *   Grigori, Hoemmen, Langou 2012) -- the unpivoted QR of Section II-A taken
 *   literally, stable whatever the sketch's conditioning or rank, slower
 *   than CholeskyQR; 0 (default) = CholeskyQR, with TSQR as the automatic
 *   fallback for sketches flagged RUQLP_FLAG_RANKDEF. */

/* Grow the workspace arena now for problems up to m x n with d columns in
 * the given compute dtype (nnz < 0: dense A; nnz >= 0: CSR A with that many
 * nonzeros), so that later calls allocate nothing.
 * Errors: INVALID, BUDGET, CUDA. */
ruqlp_status ruqlp_reserve(ruqlp_handle h, int64_t m, int64_t n, int d,
                           ruqlp_dtype compute, int64_t nnz);

/* Workspace bytes a problem needs (0 on invalid sizes); nnz as for
 * ruqlp_reserve. */
size_t ruqlp_workspace_bytes(int64_t m, int64_t n, int d, ruqlp_dtype compute,
                             int64_t nnz);

/* One RU-QLP decomposition (Section III-A; Algorithms 1 and 2), all buffers
 * in device memory.  Work is ordered on the handle's stream; the call
 * returns when it has completed (it synchronises that stream once to read
 * the device status word).  On RUQLP_OK, out->Q/L/P hold Q, L = R_B^T, P
 * (or, with finish_paper, Q P~, R~ and P, where [P~, R~] = qr(R_B^T)) and
 * out->flags the fallbacks taken.  Errors: INVALID, BUDGET, CUDA,
 * BREAKDOWN. */
ruqlp_status ruqlp_decompose(ruqlp_handle h, const ruqlp_matrix* A,
                             const ruqlp_params* prm, ruqlp_outputs* out);

/* `count` independent decompositions in one call (the batched workload:
 * many dense matrices of uneven shapes).  A[i], prm[i], out[i] as for
 * ruqlp_decompose (device memory); every item must be dense, share one
 * compute dtype (F32 or BF16) and one q, have d <= 288 and finish_paper = 0.
 * Each phase of the method (sketch products, Grams, Cholesky factorisations,
 * triangular solves) is one launch over all items; the launch sequence is
 * captured in a CUDA graph the second time a batch signature (shapes, q,
 * dtype) is seen and replayed afterwards (option "batch_graph" = 0 turns
 * this off).  BF16 items whose rows start on 16-byte boundaries take their
 * products on the tensor cores (option "bf16_simt" = 1: the CUDA cores);
 * option "batch_orth_tc" moves the CholeskyQR passes of narrow BF16 items
 * there too.  Every item gives bitwise
 * its result in a batch of one; an FP32 item also bitwise the result of
 * ruqlp_decompose on it (for BF16: with option "bf16_simt" = 1).  Returns
 * after completion; out[i].flags per item.
 * Errors: INVALID (with the failing item's index in ruqlp_last_error),
 * BUDGET, CUDA. */
ruqlp_status ruqlp_decompose_batch(ruqlp_handle h, int count, const ruqlp_matrix* A,
                                   const ruqlp_params* prm, ruqlp_outputs* out);

/* Serving (the paper has no counterpart: a request loop around the
 * decomposition of Section III).  ruqlp_submit queues one decomposition
 * (arguments as for ruqlp_decompose, device memory) and returns at once with
 * a ticket; A, omega, the output buffers and *out must stay valid until
 * ruqlp_poll reports completion, and A and omega must already hold their
 * values (the loop's streams do not wait on the caller's stream).  A scheduler thread of the handle admits
 * queued requests in arrival order as execution slots (config.max_slots,
 * each with its own stream and workspace) and HBM free up: the workspaces of
 * all slots together stay within config.hbm_budget_bytes (0 = no limit).
 * Consecutive batchable requests (dense, F32/BF16, d <= 256, at most 2^25
 * elements, same compute dtype and q, no finish_paper) are launched together
 * through the batched path; others run alone; requests arriving while earlier ones run are
 * admitted into the next free slot, so their work overlaps on the device.
 * A request's result is bitwise the one it gets alone (batch invariance).
 * Errors at submit: INVALID (arguments), BUDGET (its workspace alone exceeds
 * the budget).  ruqlp_submit and ruqlp_poll are thread-safe; ruqlp_destroy
 * waits for every submitted request. */
ruqlp_status ruqlp_submit(ruqlp_handle h, const ruqlp_matrix* A, const ruqlp_params* prm,
                          ruqlp_outputs* out, uint64_t* ticket);

/* Seconds since the handle's request loop started. */
typedef struct {
  double submit_s;  /* ruqlp_submit returned */
  double start_s;   /* admitted and launched */
  double done_s;    /* completion observed by the loop */
} ruqlp_request_times;

/* NOT_READY while the request is queued or running; afterwards its status
 * (OK, or the error of its decomposition; out->flags set) -- once: the
 * ticket is released.  ruqlp_poll_times also reports the request's times
 * (times may be NULL).  Unknown tickets: INVALID. */
ruqlp_status ruqlp_poll(ruqlp_handle h, uint64_t ticket);
ruqlp_status ruqlp_poll_times(ruqlp_handle h, uint64_t ticket, ruqlp_request_times* times);

/* The same decomposition with A, prm->omega and the outputs in HOST memory:
 * the library copies A and Omega into its arena, runs ruqlp_decompose's
 * path and copies Q, L, P back.  Errors as ruqlp_decompose. */
ruqlp_status ruqlp_decompose_host(ruqlp_handle h, const ruqlp_matrix* A,
                                  const ruqlp_params* prm, ruqlp_outputs* out);

/* One pass over A, the O(mnd) product step of RU-QLP (Algorithm 1 step 3,
 * the products of Algorithm 2, B^T = A^T Q; Section III-D):
 *   trans = 0:  Y (m x d) = A X,    X: n x d;
 *   trans = 1:  Y (n x d) = A^T X,  X: m x d.
 * A is dense (device memory, any dtype) or CSR (F32 or BF16 values); X and
 * Y are row-major device buffers (leading dimensions ldx, ldy >= d) in FP64
 * when A is FP64, else FP32.  The kernel is the one ruqlp_decompose uses for A's dtype (BF16:
 * X rounded to BF16, tensor cores, FP32 accumulation).  Returns after
 * completion.  Errors: INVALID, BUDGET, CUDA, TIMEOUT. */
ruqlp_status ruqlp_sketch(ruqlp_handle h, const ruqlp_matrix* A, int trans, const void* X,
                          int64_t ldx, int d, void* Y, int64_t ldy);

/* orth() of Section II-A as used by the path: Q (M x d) with orthonormal
 * columns spanning range(Y), Y = Q R with R upper triangular and positive
 * diagonal (the unique thin-QR Q when Y has full column rank).  Y and Q:
 * device memory, row-major, ld >= d, dtype F64 (CholeskyQR2 in FP64) or F32
 * (shifted CholeskyQR3 in FP32, or CholeskyQR2 with FP64 Gram and Cholesky
 * under the "orth_fp64" option).  Q may alias Y.  Returns after completion.
 * Errors: INVALID (NULL, d outside 1..512, M < d, ld < d, dtype), BUDGET,
 * CUDA. */
ruqlp_status ruqlp_orth(ruqlp_handle h, const void* Y, int64_t M, int d, int64_t ldy,
                        ruqlp_dtype dtype, void* Q, int64_t ldq);

/* Gram matrix of a tall-skinny matrix, the l x l product that orth()'s
 * CholeskyQR factors (Section II-A orth(); Algorithm 2):
 *   G (d x d, FP64, row-major, ld d) = Y^T Y,
 * Y: M x d row-major with leading dimension ldy >= d, dtype F64 or F32, all
 * in device memory on the handle's device.  Products and sums are FP64 (the
 * products of FP32 inputs are exact).  The M range is split into slabs whose
 * FP64 partial Grams go to the handle's workspace arena and are summed in a
 * fixed order, so repeated calls give bitwise-equal results.  Ordered on the
 * handle's stream; returns after completion.  Errors: INVALID (NULL
 * pointers, M < 1, d outside 1..512, ldy < d, other dtype), BUDGET, CUDA. */
ruqlp_status ruqlp_gram(ruqlp_handle h, const void* Y, int64_t M, int d, int64_t ldy,
                        ruqlp_dtype dtype, double* G);

/* ruqlp_gram for callers that cannot allocate device memory -- for example
 * code recording a CUDA graph (allocation is refused inside stream capture),
 * host programs whose own allocator owns all device memory, or loops that
 * cannot afford cudaMalloc's implicit synchronisation.  The paper has no
 * counterpart; it is a deployment variant of the Gram above.
 *   G (d x d, FP64, ld d) = Y^T Y, Y: M x d, ld ldy >= d, F64 or F32.
 * Y and G are device memory on the calling thread's current device; the work
 * is ordered on cuda_stream (cudaStream_t, NULL = legacy default stream) and
 * the call returns after enqueueing it (no synchronisation).  The library
 * allocates nothing: the FP64 partial sums live in one fixed 4 MiB device
 * array that every GPU loading the library keeps until the process exits, so
 * d is limited to 256 (larger d returns RUQLP_ERR_BUDGET).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress),
 * and so does the first call after that device's context has changed (a
 * cudaDeviceReset); make those first calls before any stream capture.  All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and give wrong results -- order them on one stream.  Each
 * call overwrites what it uses, so no clearing is needed between calls.
 * Errors: INVALID (NULL pointers, M < 1, d < 1, ldy < d, other dtype),
 * BUDGET (d > 256), CUDA. */
ruqlp_status ruqlp_gram_noalloc(const void* Y, int64_t M, int d, int64_t ldy,
                                ruqlp_dtype dtype, double* G, void* cuda_stream);

/* Message of the last error on this handle (never NULL; "" if none). */
const char* ruqlp_last_error(ruqlp_handle h);

/* Omega for a NULL params.omega (Section III-A step 1: iid N(0,1)), written
 * to out (device, n x d row-major FP64, ld d): Philox4x32-10 (Salmon et al.,
 * SC 2011) with key (seed mod 2^32, seed / 2^32) and counter
 * (j, i mod 2^32, i / 2^32, 0) for entry (i, j); its words x0, x1 give
 * u = (x + 1/2) 2^-32 and Omega_ij = sqrt(-2 ln u1) cos(2 pi u2) in FP64.
 * Errors: INVALID (n < 1, d < 1, NULL out), CUDA. */
ruqlp_status ruqlp_omega(ruqlp_handle h, int64_t n, int d, uint64_t seed, double* out);

/* Kernels launched by this library in this process so far (all handles). */
int64_t ruqlp_launch_count(void);

/* Tile tuner of the tensor-core products (the sketch / power / B^T passes
 * of Section III-D, the bulk of the O(mnd) work): the first product of each
 * shape (orientation, two-part operand, output rows, K, dp) outside stream
 * capture times every valid column split (1, 2, 4; each with the deepest
 * shared-memory ring that fits) twice with CUDA events and keeps the fastest
 * for the process; that configuration computes the result, so results are
 * deterministic from then on.  ruqlp_tune_file(path) loads earlier choices
 * from a text file (one "tc_gemm trans two_part rows K dp split stages us"
 * line each) and appends every new choice to it; NULL or "" stops the
 * mirroring.  Returns the number of entries loaded.  Process-wide (all
 * handles); thread-safe. */
int ruqlp_tune_file(const char* path);

/* With the "profile" option on: number of spans and their summed device time
 * (milliseconds, CUDA events on the handle's stream) of a phase:
 *   "ax"   sketch products A X (Algorithm 1 step 3 / Algorithm 2),
 *   "atx"  transposed products A^T Y (Algorithm 2; B^T = A^T Q),
 *   "orth" whole orth() calls (Gram, Cholesky, triangular solve passes),
 *   "step" whole decompositions,
 *   "tc_ax" / "tc_atx" the tensor-core product kernel launches alone
 *   (BF16 path; without operand transposes and the stream-K fix-up),
 *   "tc_atx2" those of the two-part last product B^T = A^T Q (the skinny
 *   operand as two BF16 parts: two MMAs per A tile),
 *   "gram" / "chol" / "trsm" the FP32 orth() passes' Gram (with its slab
 *   reduction), blocked Cholesky and triangular solve (single-matrix path).
 * Errors: INVALID (unknown phase, NULL pointers). */
ruqlp_status ruqlp_profile(ruqlp_handle h, const char* phase, int64_t* count, double* total_ms);

/* Library version string. */
const char* ruqlp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RUQLP_H */
