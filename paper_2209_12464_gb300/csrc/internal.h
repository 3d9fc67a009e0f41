// Internal launchers of the RU-QLP CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <functional>

#include "common.cuh"

namespace ruqlp {

// How a SIMT product accumulates.
enum class Mul : int {
  F64 = 0,        // products and sums in FP64 (exact products for FP32/BF16 inputs)
  F32 = 1,        // products and sums in FP32
  F32_ACC64 = 2,  // FP32 products summed in FP32 over 16-row chunks, chunks summed in FP64
};

// C[M x N] = A[M x K] B[K x N]; all row-major with the given leading dims.
cudaError_t simt_gemm_nn(Ty ta, Ty tb, Ty tc, Mul mul, const void* A, int64_t lda,
                         const void* B, int64_t ldb, void* C, int64_t ldc, int64_t M,
                         int64_t K, int64_t N, cudaStream_t st);

// C[M x N] = A^T B with A (K x M) and B (K x N) row-major.  With splits > 1
// the K range is cut into `splits` slabs whose FP64 partial products go to
// `partial` ([splits][M][N], FP64) and are summed in slab order into C.
// A non-null `gate` makes the launch a no-op unless *gate != 0 (device word).
cudaError_t simt_gemm_tn(Ty ta, Ty tb, Ty tc, Mul mul, const void* A, int64_t lda,
                         const void* B, int64_t ldb, void* C, int64_t ldc, int64_t M,
                         int64_t K, int64_t N, int splits, double* partial,
                         const int32_t* gate, cudaStream_t st);

// Number of K slabs simt_gemm_tn should use for a small M x N output.
int tn_splits(int64_t M, int64_t K, int64_t N, int max_splits);

// Cholesky G = R^T R of the d x d FP64 Gram G (row-major, full symmetric),
// in one CTA, in FP64.  On a non-positive pivot it retries once on
// G + shift I with shift = shift_rel * trace(G) and sets status->shifted
// (and RUQLP_FLAG_SHIFTED); a second breakdown sets RUQLP_FLAG_RANKDEF and
// replaces the failed pivots by shift-sized ones so the output stays finite.
// Writes R (upper, FP64, ld d, zero lower part) and Rw = R in type tw.
// A non-null `gate` makes it a no-op unless *gate != 0.  tf: arithmetic of
// the factorisation (F64 or F32); force_shift: factor G + shift I directly.
// check: 1 = the last pass of a CholeskyQR (its Gram should be close to I:
// a pivot outside [1/2, 2] raises RUQLP_FLAG_RANKDEF); 2 = the same while
// status->shifted is 0 (no third pass will follow); 0 = no check.
cudaError_t chol_upper(const double* G, int d, double shift_rel, double* R, void* Rw,
                       Ty tw, DevStatus* status, const int32_t* gate, cudaStream_t st,
                       Ty tf = Ty::F64, bool force_shift = false, int check = 0);

// FP32 blocked Cholesky of a d x d FP64 Gram in one CTA (d <= 256):
// G + shift I = R^T R (shift = shift_rel * trace(G) when force_shift or after
// a breakdown).  `tiles` (chol_tiles_bytes(d)) receives the packed 32 x 32
// upper tiles of R and the inverses of its diagonal tiles, which
// trsm_tiles_f32 uses to form X = Y R^{-1} (X may alias Y).
bool chol_tiles_supported(int d);
size_t chol_tiles_bytes(int d);
// check: as chol_upper's check = 1.
cudaError_t chol_tiles_f32(const float* G, int d, double shift_rel, bool force_shift,
                           float* tiles, DevStatus* status, const int32_t* gate, cudaStream_t st,
                           bool check = false);
// Bt (optional): also X^T in BF16 (dp x ldbt, zero rows d..dp), the next
// tensor-core product's B operand; Btl (optional) its low part
// bf16(x - bf16(x)) for the two-part product.
cudaError_t trsm_tiles_f32(const float* Y, int64_t ldy, const float* tiles, float* X, int64_t ldx,
                           int64_t M, int d, cudaStream_t st, void* Bt = nullptr,
                           int64_t ldbt = 0, void* Btl = nullptr);

// C (d1 x d2, FP64, ld d2) = X^T W for FP32 X (M x d1, ld ldx) and W (M x d2,
// ld ldw): FP32 products summed in FP32 within a row slab, slabs summed in
// FP64 in order.  X == W computes only the upper tiles and mirrors them.
// partial: max_slabs * d1 * d2 doubles of scratch.  Cf (optional): the same
// result rounded to FP32 (the Cholesky's input).
cudaError_t gram_f32(const float* X, int64_t ldx, const float* W, int64_t ldw, int64_t M, int d1,
                     int d2, double* C, double* partial, int max_slabs, const int32_t* gate,
                     cudaStream_t st, float* Cf = nullptr);

// X[M x d] <- Y[M x d] R^{-1} for upper-triangular R (type ty, ld d): each
// row solves x R = y by forward substitution.  X may alias Y.  A non-null
// `gate` makes it a no-op unless *gate != 0.
cudaError_t trsm_right_upper(Ty ty, const void* Y, int64_t ldy, const void* R, void* X,
                             int64_t ldx, int64_t M, int d, const int32_t* gate,
                             cudaStream_t st);

// dst[rows x cols] (type td, ld lds) <- src (type ts, ld lds), zeroing nothing else.
cudaError_t copy_cast_2d(Ty ts, const void* src, int64_t lds, Ty td, void* dst, int64_t ldd,
                         int64_t rows, int64_t cols, cudaStream_t st);

// dst[rows x cols] (FP32, ld ldd) <- src (F32 or F64) rounded to the sum of
// its two BF16 parts, h + bf16(v - h) with h = bf16(v) (the skinny operand of
// the two-part BF16 product on the CUDA cores).
cudaError_t round2_bf16_2d(Ty ts, const void* src, int64_t lds, float* dst, int64_t ldd,
                          int64_t rows, int64_t cols, cudaStream_t st);

// L (d x d, type tl, ld ldl (0: d)) <- transpose of the upper triangle of R
// (FP64, ld d), zeros above the diagonal.  With `upper` the upper triangle is
// copied as is instead (finish_paper output).
cudaError_t write_L(const double* R, int d, Ty tl, void* L, bool upper, cudaStream_t st,
                    int ldl = 0);

// Tensor-core BF16 products (k_tc.cu).  trans = false: out[m x dp] = A Bt^T;
// trans = true: out[n x dp] = A^T Bt^T, with A (m x n, BF16, ld lda) and
// Bt (dp x K, BF16, ld ldb, K = n or m).  frag: tc_frag_bytes(dp) of scratch
// for the stream-K fragments; err: device word set on a wait timeout.
// mark(true) / mark(false) are called right before / after the main kernel
// launch (used to bracket it with profiling events); may be empty.
// Btl (optional, same layout as Bt): the low BF16 part of the skinny operand;
// then out = A (Bt + Btl)^T (or A^T ...), two MMAs per A tile.
// force_ns > 0: that column split (dp / force_ns a multiple of 16); 0: the
// configuration the tuner measured fastest for this shape.  withhold (test
// hook): CTA 0 never loads its first ring stage, so its bounded waits run
// out and the launch ends on the timeout path (err set, TMEM freed).
cudaError_t tc_gemm(bool trans, const void* A, int64_t lda, int64_t m, int64_t n, const void* Bt,
                    int64_t ldb, int dp, float* out, int64_t ldo, float* frag, int* err,
                    cudaStream_t st, const std::function<void(bool)>& mark = {},
                    const void* Btl = nullptr, int force_ns = 0, int withhold = 0);
// Mirror the product tuner's choices in a text file (loaded now, appended
// to as shapes are tuned); returns the entries loaded.
int tune_file(const char* path);
size_t tc_frag_bytes(int dp);
// Whether tc_gemm accepts these operands (alignment / size rules).
bool tc_supported(const void* A, int64_t lda, int dp);

// dst[dp x rows] (BF16, ld ldd) = transpose of src[rows x cols] (ld lds), rows
// cols..dp-1 of dst zero; lo (optional, same layout) the low BF16 parts.
cudaError_t transpose_to_bf16(Ty ts, const void* src, int64_t lds, int64_t rows, int cols, int dp,
                              void* dst, int64_t ldd, cudaStream_t st, void* lo = nullptr);

// CSR products (k_csr.cu), values FP32 or BF16, dense operands FP32.
// csr_validate ORs into *flag: 1 bad rowptr, 2 bad / unsorted / duplicate
// column index.  csr_transpose builds the CSR of A^T (colptr n+1, rowidx and
// cvals nnz) with rows sorted inside each column (deterministic); scratch:
// 2n ints; *flag |= 4 if a column has more than 1024 nonzeros.
cudaError_t csr_validate(const int32_t* rowptr, const int32_t* colidx, int64_t m, int64_t n,
                         int64_t nnz, int* flag, cudaStream_t st);
cudaError_t csr_transpose(Ty tv, const int32_t* rowptr, const int32_t* colidx, const void* vals,
                          int64_t m, int64_t n, int64_t nnz, int32_t* colptr, int32_t* rowidx,
                          void* cvals, int32_t* scratch, int* flag, cudaStream_t st);
// Y[rows x d] (ld ldy) = A X with A given by (ptr, idx, vals), X FP32 (ld ldx).
cudaError_t spmm_csr(Ty tv, const int32_t* ptr, const int32_t* idx, const void* vals, int64_t rows,
                     const float* X, int64_t ldx, int d, float* Y, int64_t ldy, cudaStream_t st);

// ---- batched execution (ruqlp_decompose_batch) ----------------------------
// One entry of the device problem table: matrix A_i, its FP32 work buffers
// (ld dp) and its outputs.
enum BufId : int { B_X = 0, B_Y = 1, B_Z = 2, B_P = 3 };
struct BMat {
  const void* A;
  int64_t lda, m, n;
  int d, dp, ot, pad;
  float* X;  // n x dp
  float* Y;  // m x dp
  float* Z;  // n x dp
  float* P;  // n x dp
  double* partial;
  double* G;
  float* Gf;       // the Gram in FP32 (Cholesky input)
  float* tiles;
  const double* omega;  // NULL: generated from seed (philox.cuh)
  uint64_t seed;
  void* Bt;        // dp x ldbt BF16 (tensor-core items): the transposed skinny operand
  void* Btl;       // its low BF16 part (same layout), for the two-part B^T = A^T Q
  int64_t ldbt;
  // orth_tc: this item's CholeskyQR runs on the tensor cores (bgram_tc,
  // btrinv, bqmul_tc); St then holds the three BF16 parts of (R^{-1})^T,
  // 3 x dp x 128
  void* St;
  int use_tc, orth_tc;
  // q_direct: the last solve of the final orth of Y writes Q straight into
  // Qout (FP32, leading dimension d) instead of the Y buffer (tensor-core
  // items with the CUDA-core solve and FP32 outputs: nothing reads Y after
  // that solve, the last product taking its BF16 parts)
  int q_direct, pad2;
  void* Qout;
  void* Lout;
  void* Pout;
  DevStatus* status;
};
__host__ __device__ inline float* bbuf(const BMat& b, int id) {
  return id == B_X ? b.X : (id == B_Y ? b.Y : (id == B_Z ? b.Z : b.P));
}
// Row slabs of a Gram over M rows (a function of the shape only, so a matrix
// gets the same summation order alone and inside a batch).
__host__ __device__ inline int64_t gram_slabs(int64_t M, int max_slabs, int64_t* slab_rows) {
  int64_t slabs = (M + 511) / 512;
  if (slabs > max_slabs) slabs = max_slabs;
  if (slabs < 1) slabs = 1;
  int64_t slab = (M + slabs - 1) / slabs;
  slab = (slab + 31) / 32 * 32;
  *slab_rows = slab;
  return (M + slab - 1) / slab;
}
int bgemm_tiles(int64_t rows, int d);
// split2 (BF16 A): the skinny operand is rounded to the sum of its two BF16
// parts (the two-part B^T = A^T Q), else to BF16.
cudaError_t bgemm(bool trans, Ty ta, Ty tb, const BMat* T, const int* prefix, int total, int count,
                  int src, int dst, cudaStream_t st, bool split2 = false);
int bgram_tiles(int64_t M, int d, bool sym, int max_slabs);
// Symmetric batched Grams of the items with round16(d) <= 80 (k_bgram_sym:
// one CTA per row slab, upper-triangle blocks only); bgram_sym_ctas is an
// item's CTA count (0 for wider items, whose tiles go to bgram).
int bgram_sym_ctas(int64_t M, int d, int max_slabs);
cudaError_t bgram_sym(const BMat* T, const int* prefix, int total, int count, int src,
                      int max_slabs, cudaStream_t st);
// Batched CholeskyQR passes on the tensor cores (k_borth.cu, k_qmul.cu) for
// items with orth_tc (dp <= BO_DPMAX).  Work comes as units (a row range of
// one item); CTA c of a launch takes units uoff[c] .. uoff[c + 1] - 1, the
// host having balanced their rows over the CTAs.
//  * bgram_tc: one unit = one row slab of gram_slabs(); its FP32 sum of the
//    three-way BF16 split products (tcgen05) goes to the item's partial[slab]
//    as FP64, lower triangle (row j >= column i); bgram_reduce then adds the
//    slabs in order into G and Gf;
//  * btrinv: St = parts of (R^{-1})^T from the Cholesky's tiles (d <= 128);
//  * bqmul_tc: buf[dst] = buf[src] R^{-1} over the units' rows (the same
//    six-part-product rule as qmul_tc); make_bt as btrsm's.
constexpr int BO_DPMAX = 80;
struct BoUnit {
  int item, rows;  // table index; rows of the unit
  int64_t row0;    // first row
};
constexpr int BO_KP = 128;  // K padding of the St parts
constexpr int BO_MAXU = 64;  // units a CTA of bgram_tc / bqmul_tc takes at most
size_t bo_st_bytes(int d);
cudaError_t bgram_tc(const BMat* T, const BoUnit* units, const int* uoff, int grid, int src,
                     int max_slabs, int* err, cudaStream_t st);
cudaError_t btrinv(const BMat* T, const int* list, int n, int dmax, cudaStream_t st);
cudaError_t bqmul_tc(const BMat* T, const BoUnit* units, const int* uoff, int grid, int src,
                     int dst, int make_bt, int* err, cudaStream_t st);
// reduce = false: only the CUDA-core tiles (bgram_reduce adds the slabs
// later, e.g. together with bgram_tc's)
cudaError_t bgram(const BMat* T, const int* prefix, int total, int count, int src, int src2,
                  int max_slabs, int dmax, cudaStream_t st, bool reduce = true);
cudaError_t bgram_reduce(const BMat* T, int count, int src, int src2, int max_slabs, int dmax,
                         cudaStream_t st);
int btrsm_blocks(int64_t M);
cudaError_t bchol(const BMat* T, int count, double shift_rel, bool force_shift, int dmax,
                  cudaStream_t st, bool check = false);
// make_bt: 1 = also write the result transposed in BF16 to each tensor-core
// item's Bt (the next product's B operand); 2 = and its low part to Btl.
cudaError_t btrsm(const BMat* T, const int* prefix, int total, int count, int src, int dst,
                  int dmax, cudaStream_t st, int make_bt = 0);
// Tensor-core Gram C = Y^T Y of a tall FP32 Y (M >= 8192, d <= 256, ld a
// multiple of 4, 16-byte aligned) via a three-way BF16 split; part holds
// the FP32 slab sums (gram_tc_part_bytes(d) bytes at most); C (FP64) and Cf
// (FP32) the result.
bool gram_tc_supported(int64_t M, int d, int64_t ldy, const void* Y);
int gram_tc_ctas(int64_t M);
size_t gram_tc_part_bytes(int d);
// The upper triangle of C = X^T Y (same shape and rules as gram_tc; the
// strictly lower triangle of C is set to zero): R_B = P^T B^T.
cudaError_t gram_tc_upper(const float* X, const float* Y, int64_t ld, int64_t M, int d,
                          float* part, double* C, int* err, cudaStream_t st);
// Q = Y R^{-1} on the tensor cores (tall FP32 Y, M >= 8192, d <= 256): the
// blocked Cholesky's tiles are inverted into St (qmul_st_bytes(d) bytes,
// S^T as three BF16 parts), then Q (may alias Y) = Y S; Bt (optional)
// receives Q^T in BF16 with leading dimension ldbt, Btl (optional) its low
// BF16 part.  err: timeout word.
size_t qmul_st_bytes(int d);
bool qmul_supported(int64_t M, int d, int64_t ldy, const void* Y, int64_t ldq, const void* Q);
cudaError_t qmul_tc(const float* Y, int64_t ldy, const float* tiles, int64_t M, int d, void* St,
                    float* Q, int64_t ldq, void* Bt, int64_t ldbt, int* err, cudaStream_t st,
                    void* Btl = nullptr);
// 2-D BF16 tensor map (128-byte swizzle) over a row-major [outer][inner]
// array with leading dimension ld_elems; box box_inner x box_outer.
bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld_elems,
              uint32_t box_inner, uint32_t box_outer);
int sm_count();
cudaError_t gram_tc(const float* Y, int64_t ldy, int64_t M, int d, float* part, double* C,
                    float* Cf, int* err, cudaStream_t st);
// SVD of a d x d matrix by one-sided Jacobi in one CTA (type t: F32/F64):
// W (column-major) holds the matrix on entry; outputs Uo, Vo (d x d row-major,
// ld ldo, columns sorted by decreasing singular value) and s (descending).
cudaError_t svd_jacobi(Ty t, void* W, void* V, void* s, int d, int max_sweeps, int* order,
                       void* tmpcol, int* sweeps, void* Uo, void* Vo, int64_t ldo,
                       cudaStream_t st);
// L (d x d, type to) = diag(s) (s of type t).
cudaError_t write_diag(Ty t, const void* s, int d, Ty to, void* L, cudaStream_t st);

// out += t for a rows x d FP32 block (the low-rank term of a CSR input).
cudaError_t add_rows_f32(float* out, int64_t ldo, const float* t, int64_t ldt, int64_t rows, int d,
                         cudaStream_t st);

// Householder TSQR (k_tsqr.cu): Q (M x d, ld ldq, may alias Y) = the
// orthonormal factor of Y (M x d, ld ldy) with diag(R) >= 0, F32 or F64,
// M >= d; work: tsqr_work_bytes(t, M, d) bytes of device memory.
size_t tsqr_work_bytes(Ty t, int64_t M, int d);
bool tsqr_supported(Ty t, int64_t M, int d);
cudaError_t tsqr(Ty t, const void* Y, int64_t ldy, int64_t M, int d, void* Q, int64_t ldq,
                 void* work, cudaStream_t st);

// Omega (n x d, FP64, row-major with ld ldo) from the counter-based generator
// of philox.cuh.
cudaError_t omega_philox(uint64_t seed, int64_t n, int d, double* out, int64_t ldo,
                         cudaStream_t st);

// Batched tensor-core products (BF16 A): tile list entries and launcher.
struct BTcTile {
  int mat, tile;
};
// Encode the four tensor maps of one matrix (A, Bt over n, Bt over m, Btl
// over m) into maps4 (btc_map_bytes() bytes, 64-byte aligned); a_only
// re-encodes A alone.
bool btc_encode(void* maps4, const void* A, int64_t lda, int64_t m, int64_t n, const void* Bt,
                const void* Btl, int64_t ldbt, int dp, bool a_only);
// Bytes of one matrix's tensor maps.
size_t btc_map_bytes();
// buf[dst] = A Bt^T (trans: A^T Bt^T) for the tile list's matrices; b2
// (trans only): A^T (Bt + Btl)^T, the two-part product.
cudaError_t btc_gemm(bool trans, const BMat* T, int count, const BTcTile* list, int n,
                     const void* maps, int src, int dst, int dpmax, int* err, cudaStream_t st,
                     bool b2 = false);
cudaError_t bcast_omega(const BMat* T, int count, int64_t max_elems, cudaStream_t st);
cudaError_t boutputs(const BMat* T, int count, int64_t max_elems, cudaStream_t st);

// Zero the status word.
cudaError_t status_reset(DevStatus* s, cudaStream_t st);
// Clear only the per-orth `shifted` field.
cudaError_t status_clear_shift(DevStatus* s, cudaStream_t st);

}  // namespace ruqlp
