// C ABI of the RU-QLP library: handle, validation, workspace arena and the
// host-side orchestration of Algorithm 1 + Algorithm 2 (Section III) in the
// right-sketch orientation.  Every arithmetic step runs in the kernels of
// this library; the host only validates, carves the arena and launches.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <stdio.h>
#include <functional>
#include <vector>
#include <stdarg.h>
#include <string.h>
#include <string>

#include "../../include/ruqlp.h"
#include "ctx.h"
#include "internal.h"

using namespace ruqlp;

namespace ruqlp {
static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ruqlp

namespace {

const char* kVersion = "ruqlp-gb300 0.1 (sm_103a)";

ruqlp_status fail(ruqlp_ctx* h, ruqlp_status s, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return s;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(h, RUQLP_ERR_CUDA, "%s failed: %s (%s:%d)", #call,               \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

// Profile categories: sketch products A X, transposed products A^T Y (whole
// product phases), orth(), the whole decomposition, and the tensor-core
// product kernel launches alone (k_tc_gemm, without operand transposes or the
// stream-K fix-up) for A X, for A^T Y with a one-part skinny operand and for
// the two-part last product B^T = A^T Q.
enum {
  PROF_AX = 0, PROF_ATX = 1, PROF_ORTH = 2, PROF_STEP = 3, PROF_TC_AX = 4, PROF_TC_ATX = 5,
  PROF_GRAM = 6, PROF_CHOL = 7, PROF_TRSM = 8, PROF_TC_ATX2 = 9
};
const int kProfN = ruqlp_ctx::kProfPhases;
const char* kProfNames[] = {"ax", "atx", "orth", "step", "tc_ax", "tc_atx",
                            "gram", "chol", "trsm", "tc_atx2"};
static_assert(sizeof(kProfNames) / sizeof(kProfNames[0]) == kProfN, "profile phases");

cudaEvent_t ev_get(ruqlp_ctx* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  ruqlp_ctx* h;
  int cat;
  cudaEvent_t a = nullptr;
  ProfScope(ruqlp_ctx* h_, int c) : h(h_), cat(c) {  // h == nullptr: no span
    if (h && h->profile) {
      a = ev_get(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~ProfScope() {
    if (h && h->profile && a) {
      cudaEvent_t b = ev_get(h);
      cudaEventRecord(b, h->stream);
      h->spans.push_back({cat, a, b});
    }
  }
};

void prof_collect(ruqlp_ctx* h) {
  for (auto& sp : h->spans) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
      h->prof_count[sp.cat] += 1;
      h->prof_ms[sp.cat] += ms;
    }
    h->pool.push_back(sp.a);
    h->pool.push_back(sp.b);
  }
  h->spans.clear();
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int round16(int d) { return (d + 15) / 16 * 16; }

bool ty_of(ruqlp_dtype d, Ty* t) {
  if (d == RUQLP_F64) { *t = Ty::F64; return true; }
  if (d == RUQLP_F32) { *t = Ty::F32; return true; }
  if (d == RUQLP_BF16) { *t = Ty::BF16; return true; }
  return false;
}

// Work type of the tall-skinny matrices (Y, Z, Q, P) for a compute dtype.
Ty work_ty(Ty ct) { return ct == Ty::F64 ? Ty::F64 : Ty::F32; }

constexpr int kMaxSplits = 64;

// Workspace layout for one problem.
struct Layout {
  size_t X, Y, Z, P, partial, G, Gf, R, Rw, St, Bt, Btl, frag, colptr, rowidx, cvals, cscratch, T, Om,
      lrT1, lrT2, lrTmp, lrPart, svdW, svdV, svdS, svdOrd, svdTmp, svdU, svdVs, Ts, total;
};

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// nnz >= 0: A is CSR with nnz nonzeros of val_bytes each (CSC copy kept too).
// finish: room for Algorithm 1 step 5 (an m x dp buffer for Q P~).
// tsqr: room for the Householder TSQR orth() (the rank-deficiency fallback).
Layout layout_of(int64_t m, int64_t n, int d, Ty ct, int64_t nnz = -1, size_t val_bytes = 0,
                 int finish = 0, bool gen_omega = false, int64_t lr_r = 0, bool tsqr = false) {
  Layout L{};
  const int dp = round16(d);
  const size_t wes = ty_size(work_ty(ct));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.X = take((size_t)n * dp * wes);
  L.Y = take((size_t)m * dp * wes);
  L.Z = take((size_t)n * dp * wes);
  L.P = take((size_t)n * dp * wes);
  // Gram scratch: FP64 slab partials (SIMT Gram) or FP32 slab sums of the
  // tensor-core Gram (one per SM, at most 160)
  L.partial = take(std::max((size_t)d * d * std::max<size_t>(kMaxSplits * sizeof(double), 160 * sizeof(float)),
                             gram_tc_part_bytes(d)));
  L.G = take((size_t)d * d * sizeof(double));
  L.Gf = take((size_t)d * d * sizeof(float));
  L.R = take((size_t)d * d * sizeof(double));
  {
    size_t rw = (size_t)d * d * sizeof(double);
    if (chol_tiles_supported(d) && chol_tiles_bytes(d) > rw) rw = chol_tiles_bytes(d);
    L.Rw = take(rw);
  }
  // S = R^{-1} as three BF16 parts for the tensor-core Q = Y S
  if (work_ty(ct) == Ty::F32 && dp <= 256) L.St = take(qmul_st_bytes(d));
  if (ct == Ty::BF16 && nnz < 0) {
    // the transposed BF16 skinny operand, then its low BF16 part (the
    // two-part B^T = A^T Q); the CUDA-core kernel's rounded FP32 operand
    // (K x d) fits the two together
    const size_t one = (size_t)dp * round8(m > n ? m : n) * 2;
    L.Bt = take(2 * one);
    L.Btl = L.Bt + one;
    L.frag = take(tc_frag_bytes(dp <= 256 ? dp : 256));  // per column chunk
  }
  if (finish) L.T = take((size_t)m * dp * wes);
  if (finish == 2) {  // Jacobi SVD of L: W, V, S, order, norms, sweep count, sorted U and V
    L.svdW = take((size_t)d * d * wes);
    L.svdV = take((size_t)d * d * wes);
    L.svdS = take((size_t)d * wes);
    L.svdOrd = take((size_t)d * sizeof(int) + 16);
    L.svdTmp = take((size_t)d * wes);
    L.svdU = take((size_t)d * dp * wes);
    L.svdVs = take((size_t)d * dp * wes);
  }
  if (gen_omega) L.Om = take((size_t)n * d * sizeof(double));
  if (lr_r > 0) {  // low-rank term of a CSR input
    L.lrT1 = take((size_t)lr_r * dp * sizeof(float));
    L.lrT2 = take((size_t)lr_r * dp * sizeof(float));
    L.lrTmp = take((size_t)(m > n ? m : n) * dp * sizeof(float));
    L.lrPart = take((size_t)kMaxSplits * lr_r * dp * sizeof(double));
  }
  if (nnz >= 0) {
    L.colptr = take((size_t)(n + 1) * sizeof(int32_t));
    L.rowidx = take((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    L.cvals = take((size_t)(nnz > 0 ? nnz : 1) * val_bytes);
    L.cscratch = take((size_t)2 * n * sizeof(int32_t));
  }
  if (tsqr) L.Ts = take(tsqr_work_bytes(work_ty(ct), std::max<int64_t>(std::max(m, n), d), d));
  L.total = off;
  return L;
}

ruqlp_status ensure_arena(ruqlp_ctx* h, size_t bytes) {
  if (bytes <= h->arena_bytes) return RUQLP_OK;
  if (h->budget && bytes > h->budget)
    return fail(h, RUQLP_ERR_BUDGET, "workspace of %zu bytes exceeds the budget of %zu bytes",
                bytes, h->budget);
  CK(cudaSetDevice(h->device));
  if (h->arena) {
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaFree(h->arena));
    h->arena = nullptr;
    h->arena_bytes = 0;
  }
  CK(cudaMalloc(&h->arena, bytes));
  h->arena_bytes = bytes;
  for (auto& g : h->batches)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->batches.clear();
  return RUQLP_OK;
}

ruqlp_status validate_params(ruqlp_ctx* h, int64_t m, int64_t n, Ty at, const ruqlp_params* prm,
                             const ruqlp_outputs* out, int* d) {
  Ty ct;
  if (!ty_of(prm->compute, &ct)) return fail(h, RUQLP_ERR_INVALID, "unknown compute dtype");
  if (at != ct) return fail(h, RUQLP_ERR_INVALID, "compute dtype must equal A's dtype");
  if (prm->k < 1) return fail(h, RUQLP_ERR_INVALID, "k must be >= 1 (got %d)", prm->k);
  if (prm->p < 0) return fail(h, RUQLP_ERR_INVALID, "p must be >= 0 (got %d)", prm->p);
  if (prm->q < 0) return fail(h, RUQLP_ERR_INVALID, "q must be >= 0 (got %d)", prm->q);
  if (prm->finish_paper < 0 || prm->finish_paper > 2)
    return fail(h, RUQLP_ERR_INVALID, "finish_paper must be 0, 1 or 2");
  const int64_t dd = (int64_t)prm->k + prm->p;
  if (dd > m || dd > n)
    return fail(h, RUQLP_ERR_INVALID, "d = k + p = %lld exceeds min(m, n) = %lld",
                (long long)dd, (long long)(m < n ? m : n));
  if (dd > 512) return fail(h, RUQLP_ERR_INVALID, "d = %lld exceeds the maximum of 512",
                            (long long)dd);
  if (!out->Q || !out->L || !out->P) return fail(h, RUQLP_ERR_INVALID, "NULL output buffer");
  if (out->out_dtype != RUQLP_F64 && out->out_dtype != RUQLP_F32)
    return fail(h, RUQLP_ERR_INVALID, "out_dtype must be F64 or F32");
  *d = (int)dd;
  return RUQLP_OK;
}

ruqlp_status validate(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                      const ruqlp_outputs* out, int64_t* m, int64_t* n, int* d) {
  if (!A || !prm || !out) return fail(h, RUQLP_ERR_INVALID, "NULL argument");
  Ty at;
  if (A->is_csr) {
    const ruqlp_csr& C = A->csr;
    if (C.m < 1 || C.n < 1) return fail(h, RUQLP_ERR_INVALID, "A must be at least 1 x 1");
    if (C.nnz < 0 || C.nnz >= (int64_t)1 << 31)
      return fail(h, RUQLP_ERR_INVALID, "nnz must be in [0, 2^31)");
    if (C.m >= (int64_t)1 << 31 || C.n >= (int64_t)1 << 31)
      return fail(h, RUQLP_ERR_INVALID, "CSR dimensions must fit int32 indices");
    if (!C.rowptr || (C.nnz > 0 && (!C.colidx || !C.values)))
      return fail(h, RUQLP_ERR_INVALID, "NULL CSR array");
    if (!ty_of(C.dtype, &at) || at == Ty::F64)
      return fail(h, RUQLP_ERR_INVALID, "CSR values must be F32 or BF16");
    if (A->is_csr == 2) {
      const ruqlp_lowrank& R = A->lr;
      if (R.r < 1 || R.r > 4096) return fail(h, RUQLP_ERR_INVALID, "low-rank r must be in [1, 4096]");
      if (!R.X || !R.D || !R.Y) return fail(h, RUQLP_ERR_INVALID, "NULL low-rank factor");
    } else if (A->is_csr != 1) {
      return fail(h, RUQLP_ERR_INVALID, "is_csr must be 0, 1 or 2");
    }
    *m = C.m;
    *n = C.n;
  } else {
    const ruqlp_dense& D = A->dense;
    if (D.m < 1 || D.n < 1) return fail(h, RUQLP_ERR_INVALID, "A must be at least 1 x 1");
    if (D.ld < D.n) return fail(h, RUQLP_ERR_INVALID, "ld (%lld) < n (%lld)", (long long)D.ld,
                                (long long)D.n);
    if (!D.data) return fail(h, RUQLP_ERR_INVALID, "A.data is NULL");
    if (!ty_of(D.dtype, &at)) return fail(h, RUQLP_ERR_INVALID, "unknown dtype");
    *m = D.m;
    *n = D.n;
  }
  return validate_params(h, *m, *n, at, prm, out, d);
}

// Everything the orchestration needs for one decomposition.
struct Job {
  const void* A;
  int64_t lda, m, n;
  int d, dp, q;
  Ty ct, wt;
  const double* omega;  // device, n x d; NULL: generated from seed
  uint64_t seed = 0;
  void* Qout;
  void* Lout;
  void* Pout;
  Ty ot;
  int finish_paper;  // 0 none, 1 qr(L) (Algorithm 1 step 5), 2 SVD of L (Remark 1)
  bool use_tc;  // BF16 products on the tensor cores (k_tc.cu)
  // CSR input (work type FP32): A's arrays and the CSC copy in the arena
  bool csr = false;
  const int32_t* rowptr = nullptr;
  const int32_t* colidx = nullptr;
  const void* vals = nullptr;
  int64_t nnz = 0;
  Ty tv = Ty::F32;
  int32_t* colptr = nullptr;
  int32_t* rowidx = nullptr;
  void* cvals = nullptr;
  // low-rank term A = S + X D Y^T of a CSR input (lr_r = 0: none)
  int64_t lr_r = 0;
  const float* lrX = nullptr;
  const float* lrD = nullptr;
  const float* lrY = nullptr;
};

// orth() of Section II-A: Q = Yin R^{-1} with R from Cholesky factorisations
// of Gram matrices (CholeskyQR, Fukaya et al. 2020).
//  * FP64 work type (and the "orth_fp64" option): CholeskyQR2 with FP64
//    products and an FP64 Cholesky; a third pass runs only when a Cholesky of
//    this orth had to shift (status->shifted gates the launches).
//  * FP32 work type (default for FP32/BF16): shifted CholeskyQR3 in FP32 --
//    the first Cholesky always factors G + s I, s = 64 u_32 trace(G), so it
//    cannot break down for kappa(Y) up to about 1/u_32; two more unshifted
//    passes restore orthonormality.  FP32 Grams are summed across row slabs
//    in FP64 (CUDA-core Gram) or with compensated FP32 sums (tensor-core
//    Gram).  (A single-SM FP64 Cholesky of a 220 x 220 Gram costs ~0.45 ms on
//    GB300, whose FP64 rate is 1/58 of FP32.)
// make_bt: the last solve also writes Q^T in BF16 to the arena's Bt (the
// next tensor-core product's operand), and with split2 its low BF16 part to
// Btl (the two-part B^T = A^T Q); returns whether it did.
ruqlp_status orth(ruqlp_ctx* h, const Layout& Lo, const Job& J, const void* Yin, void* Qout,
                  int64_t M, bool final_basis = true, bool make_bt = false,
                  bool* bt_made = nullptr, bool split2 = false) {
  if (bt_made) *bt_made = false;
  ProfScope ps(h, PROF_ORTH);
  char* base = (char*)h->arena;
  double* partial = (double*)(base + Lo.partial);
  double* G = (double*)(base + Lo.G);
  float* Gf = (float*)(base + Lo.Gf);
  double* R = (double*)(base + Lo.R);
  void* Rw = base + Lo.Rw;
  const int d = J.d, dp = J.dp;
  const Ty wt = J.wt;
  cudaStream_t st = h->stream;
  if (h->tsqr_now || h->orth_tsqr) {
    // Householder TSQR: the unpivoted QR itself, stable whatever the rank
    // (the fallback when a CholeskyQR pass flagged the sketch as numerically
    // rank deficient); the next tensor-core product transposes Q itself
    if (Lo.Ts == 0 || !tsqr_supported(wt, M, d))
      return fail(h, RUQLP_ERR_INVALID, "internal: no TSQR workspace for %lld x %d",
                  (long long)M, d);
    CK(tsqr(wt, Yin, dp, M, d, Qout, dp, base + Lo.Ts, st));
    return RUQLP_OK;
  }
  if (wt == Ty::F32 && !h->orth_fp64) {
    const double s1 = 64.0 * 5.960464477539063e-08;
    const bool blocked = chol_tiles_supported(d);
    const int passes = (final_basis || h->orth_full) ? 3 : 2;
    for (int pass = 0; pass < passes; ++pass) {
      const float* src = (const float*)(pass == 0 ? Yin : Qout);
      {
        ProfScope pg(h, PROF_GRAM);
        if (!h->orth_simt && gram_tc_supported(M, d, dp, src))
          CK(gram_tc(src, dp, M, d, (float*)partial, G, Gf, &h->status->timeout, st));
        else
          CK(gram_f32(src, dp, src, dp, M, d, d, G, partial, kMaxSplits, nullptr, st, Gf));
      }
      if (blocked) {
        {
          ProfScope pc(h, PROF_CHOL);
          // the last pass of a final basis sees a Gram close to I, or flags
          // the sketch as numerically rank deficient
          CK(chol_tiles_f32(Gf, d, s1, pass == 0, (float*)Rw, h->status, nullptr, st,
                            pass == 2));
        }
        ProfScope pt(h, PROF_TRSM);
        const bool bt = make_bt && pass == passes - 1;
        void* btl = (bt && split2) ? base + Lo.Btl : nullptr;
        if (!h->orth_simt && Lo.St != 0 && qmul_supported(M, d, dp, src, dp, Qout))
          CK(qmul_tc(src, dp, (const float*)Rw, M, d, base + Lo.St, (float*)Qout, dp,
                     bt ? base + Lo.Bt : nullptr, round8(M), &h->status->timeout, st, btl));
        else
          CK(trsm_tiles_f32(src, dp, (const float*)Rw, (float*)Qout, dp, M, d, st,
                            bt ? base + Lo.Bt : nullptr, round8(M), btl));
        if (bt && bt_made) *bt_made = true;
      } else {
        CK(chol_upper(G, d, s1, R, Rw, Ty::F32, h->status, nullptr, st, Ty::F32, pass == 0,
                      pass == 2 ? 1 : 0));
        CK(trsm_right_upper(Ty::F32, src, dp, Rw, Qout, dp, M, d, nullptr, st));
      }
    }
    return RUQLP_OK;
  }
  const Mul g = Mul::F64;  // FP64 products (exact for FP32 data)
  const double srel =
      11.0 * ((double)M * d + (double)d * (d + 1)) * 1.1102230246251565e-16;
  const int S = tn_splits(d, M, d, kMaxSplits);
  const int32_t* gate = &h->status->shifted;
  CK(status_clear_shift(h->status, st));  // this orth's shift flag gates pass 3
  // pass 1
  CK(simt_gemm_tn(wt, wt, Ty::F64, g, Yin, dp, Yin, dp, G, d, d, M, d, S, partial, nullptr, st));
  CK(chol_upper(G, d, srel, R, Rw, wt, h->status, nullptr, st));
  CK(trsm_right_upper(wt, Yin, dp, Rw, Qout, dp, M, d, nullptr, st));
  // pass 2 (the last one unless pass 1 shifted: then its Gram must be close
  // to I, else the sketch is numerically rank deficient)
  CK(simt_gemm_tn(wt, wt, Ty::F64, g, Qout, dp, Qout, dp, G, d, d, M, d, S, partial, nullptr, st));
  CK(chol_upper(G, d, srel, R, Rw, wt, h->status, nullptr, st, Ty::F64, false, 2));
  CK(trsm_right_upper(wt, Qout, dp, Rw, Qout, dp, M, d, nullptr, st));
  // pass 3 (only after a shift; the last pass)
  CK(simt_gemm_tn(wt, wt, Ty::F64, g, Qout, dp, Qout, dp, G, d, d, M, d, S, partial, gate, st));
  CK(chol_upper(G, d, srel, R, Rw, wt, h->status, gate, st, Ty::F64, false, 1));
  CK(trsm_right_upper(wt, Qout, dp, Rw, Qout, dp, M, d, gate, st));
  return RUQLP_OK;
}

// One pass over A (Algorithm 1 step 3, Algorithm 2, B^T = A^T Q):
//   trans = false: out[m x dp] = A Xin, Xin n x d;
//   trans = true:  out[n x dp] = A^T Xin, Xin m x d;
// Xin has type xt and leading dimension ldx; out is the work type, ld dp.
// split2 (BF16 A): the skinny operand is taken as the sum of its two BF16
// parts, h + bf16(x - h), instead of bf16(x) -- the last product B^T = A^T Q,
// whose rounding of Q would otherwise enter L directly (Q dQ^T A with
// ||dQ^T A|| about 2^-9 sqrt(d / m) ||A||); the sketch products only need
// the span of their operand.
ruqlp_status product(ruqlp_ctx* h, const Layout& Lo, const Job& J, bool trans, Ty xt,
                     const void* Xin, int64_t ldx, void* out, bool bt_ready = false,
                     bool split2 = false) {
  ProfScope p(h, trans ? PROF_ATX : PROF_AX);
  cudaStream_t st = h->stream;
  char* base = (char*)h->arena;
  const int64_t K = trans ? J.m : J.n;
  const int64_t Mout = trans ? J.n : J.m;
  if (J.csr) {
    if (xt != Ty::F32) return fail(h, RUQLP_ERR_INVALID, "internal: CSR operand type");
    if (!trans)
      CK(spmm_csr(J.tv, J.rowptr, J.colidx, J.vals, J.m, (const float*)Xin, ldx, J.d,
                  (float*)out, J.dp, st));
    else
      CK(spmm_csr(J.tv, J.colptr, J.rowidx, J.cvals, J.n, (const float*)Xin, ldx, J.d,
                  (float*)out, J.dp, st));
    if (J.lr_r > 0) {
      // + X (D (Y^T W))  or  + Y (D^T (X^T W)): two thin products and a
      // K = r product, FP32 with FP64 split-K partials over the long dimension
      const int64_t r = J.lr_r;
      const float* F1 = trans ? J.lrX : J.lrY;  // contracted with W
      const float* F2 = trans ? J.lrY : J.lrX;  // expands back to rows
      float* T1 = (float*)(base + Lo.lrT1);
      float* T2 = (float*)(base + Lo.lrT2);
      float* tmp = (float*)(base + Lo.lrTmp);
      double* lrp = (double*)(base + Lo.lrPart);
      CK(simt_gemm_tn(Ty::F32, Ty::F32, Ty::F32, Mul::F32, F1, r, Xin, ldx, T1, J.dp, r, K, J.d,
                      tn_splits(r, K, J.d, kMaxSplits), lrp, nullptr, st));
      if (!trans)
        CK(simt_gemm_nn(Ty::F32, Ty::F32, Ty::F32, Mul::F32, J.lrD, r, T1, J.dp, T2, J.dp, r, r,
                        J.d, st));
      else
        CK(simt_gemm_tn(Ty::F32, Ty::F32, Ty::F32, Mul::F32, J.lrD, r, T1, J.dp, T2, J.dp, r, r,
                        J.d, 1, nullptr, nullptr, st));
      CK(simt_gemm_nn(Ty::F32, Ty::F32, Ty::F32, Mul::F32, F2, r, T2, J.dp, tmp, J.dp, Mout, r,
                      J.d, st));
      CK(add_rows_f32((float*)out, J.dp, tmp, J.dp, Mout, J.d, st));
    }
    return RUQLP_OK;
  }
  if (J.use_tc) {
    // the MMA's N is at most 256: wider sketches run as column chunks of
    // equal width (multiples of 16), each one pass over A
    void* Bt = base + Lo.Bt;
    void* Btl = split2 ? base + Lo.Btl : nullptr;
    const int64_t ldb = round8(K);
    const int nch = (J.dp + 255) / 256;
    const int w = round16((J.dp + nch - 1) / nch);
    const size_t xes = ty_size(xt);
    for (int c0 = 0; c0 < J.dp; c0 += w) {
      const int wc = std::min(w, J.dp - c0);
      const int cols = std::max(0, std::min(J.d - c0, wc));
      if (!(bt_ready && nch == 1))  // else the last solve of orth() wrote it
        CK(transpose_to_bf16(xt, (const char*)Xin + (size_t)c0 * xes, ldx, K, cols, wc, Bt, ldb,
                             st, Btl));
      CK(tc_gemm(trans, J.A, J.lda, J.m, J.n, Bt, ldb, wc, (float*)out + c0, J.dp,
                 (float*)(base + Lo.frag), &h->status->timeout, st,
                 h->profile ? [&](bool begin) {
                   static thread_local cudaEvent_t a;
                   if (begin) { a = ev_get(h); cudaEventRecord(a, st); }
                   else {
                     cudaEvent_t b = ev_get(h);
                     cudaEventRecord(b, st);
                     h->spans.push_back(
                         {trans ? (split2 ? PROF_TC_ATX2 : PROF_TC_ATX) : PROF_TC_AX, a, b});
                   }
                 } : std::function<void(bool)>(), Btl, h->tc_nsplit, h->test_withhold));
    }
    return RUQLP_OK;
  }
  const Mul mul = (J.ct == Ty::F64) ? Mul::F64 : Mul::F32;
  if (J.ct == Ty::BF16 && split2) {
    // the two-part operand, rounded as the tensor cores use it (h + l is exact
    // in FP32)
    float* Xr = (float*)(base + Lo.Bt);
    CK(round2_bf16_2d(xt, Xin, ldx, Xr, J.d, K, J.d, st));
    Xin = Xr;
    xt = Ty::F32;
    ldx = J.d;
  } else if (J.ct == Ty::BF16) {
    // BF16 compute rounds the skinny operand to BF16 on either kernel, so the
    // CUDA-core kernel computes the same product as the tensor cores
    void* Xb = base + Lo.Bt;
    CK(copy_cast_2d(xt, Xin, ldx, Ty::BF16, Xb, J.d, K, J.d, st));
    Xin = Xb;
    xt = Ty::BF16;
    ldx = J.d;
  }
  if (!trans)
    CK(simt_gemm_nn(J.ct, xt, J.wt, mul, J.A, J.lda, Xin, ldx, out, J.dp, Mout, K, J.d, st));
  else
    CK(simt_gemm_tn(J.ct, xt, J.wt, mul, J.A, J.lda, Xin, ldx, out, J.dp, Mout, K, J.d, 1,
                    nullptr, nullptr, st));
  return RUQLP_OK;
}

// Job fields shared by the device and host entry points.
void fill_job(const ruqlp_matrix* A, const ruqlp_params* prm, const ruqlp_outputs* out, int64_t m,
              int64_t n, int d, Job& J) {
  J.m = m;
  J.n = n;
  J.d = d;
  J.dp = round16(d);
  J.q = prm->q;
  ty_of(prm->compute, &J.ct);
  J.wt = work_ty(J.ct);
  J.omega = prm->omega;
  J.seed = prm->omega_seed;
  ty_of(out->out_dtype, &J.ot);
  J.finish_paper = prm->finish_paper;
  if (A->is_csr) {
    J.csr = true;
    J.rowptr = A->csr.rowptr;
    J.colidx = A->csr.colidx;
    J.vals = A->csr.values;
    J.nnz = A->csr.nnz;
    ty_of(A->csr.dtype, &J.tv);
    J.wt = Ty::F32;
    if (A->is_csr == 2) {
      J.lr_r = A->lr.r;
      J.lrX = A->lr.X;
      J.lrD = A->lr.D;
      J.lrY = A->lr.Y;
    }
  } else {
    J.A = A->dense.data;
    J.lda = A->dense.ld;
  }
}

// CSR inputs: check the structure on the device and build the CSC copy in
// the arena (used by the A^T products); one synchronisation to read the
// check result.  Jm receives the CSC pointers.
ruqlp_status prepare_csr(ruqlp_ctx* h, const Layout& Lo, Job& J) {
  char* base = (char*)h->arena;
  J.colptr = (int32_t*)(base + Lo.colptr);
  J.rowidx = (int32_t*)(base + Lo.rowidx);
  J.cvals = base + Lo.cvals;
  int* flag = &h->status->invalid;
  // the structure is checked (and the result read) before any kernel indexes
  // with the column indices
  CK(csr_validate(J.rowptr, J.colidx, J.m, J.n, J.nnz, flag, h->stream));
  CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int f = h->status_host->invalid;
  if (f & 1) return fail(h, RUQLP_ERR_INVALID, "CSR rowptr is not a valid prefix array");
  if (f & 2)
    return fail(h, RUQLP_ERR_INVALID,
                "CSR column index out of range or not strictly increasing within a row");
  CK(csr_transpose(J.tv, J.rowptr, J.colidx, J.vals, J.m, J.n, J.nnz, J.colptr, J.rowidx,
                   J.cvals, (int32_t*)(base + Lo.cscratch), flag, h->stream));
  return RUQLP_OK;
}

ruqlp_status run_dense(ruqlp_ctx* h, const Job& J0) {
  Job J = J0;
  const bool gen = J.omega == nullptr;
  const bool ts = h->tsqr_now || h->orth_tsqr;
  const Layout Lo = J.csr ? layout_of(J.m, J.n, J.d, J.ct, J.nnz, ty_size(J.tv), J.finish_paper,
                                      gen, J.lr_r, ts)
                          : layout_of(J.m, J.n, J.d, J.ct, -1, 0, J.finish_paper, gen, 0, ts);
  ruqlp_status s = ensure_arena(h, Lo.total);
  if (s != RUQLP_OK) return s;
  CK(status_reset(h->status, h->stream));
  if (gen) {  // a1: Omega from the counter-based generator, on the device
    double* Om = (double*)((char*)h->arena + Lo.Om);
    CK(omega_philox(J.seed, J.n, J.d, Om, J.d, h->stream));
    J.omega = Om;
  }
  if (J.csr) {
    s = prepare_csr(h, Lo, J);
    if (s != RUQLP_OK) return s;
  }
  char* base = (char*)h->arena;
  void* X = base + Lo.X;
  void* Y = base + Lo.Y;
  void* Z = base + Lo.Z;
  void* Pb = base + Lo.P;
  double* partial = (double*)(base + Lo.partial);
  double* G = (double*)(base + Lo.G);
  const int d = J.d, dp = J.dp;
  const Ty wt = J.wt;
  const size_t wes = ty_size(wt);
  cudaStream_t st = h->stream;

  ProfScope pstep(h, PROF_STEP);
  // a1 + a2: Y = A Omega (Omega is FP64 n x d; the tensor-core path transposes
  // it straight to BF16, the other paths cast it to the work type first)
  if (J.use_tc) {
    s = product(h, Lo, J, false, Ty::F64, J.omega, d, Y);
  } else {
    CK(cudaMemsetAsync(X, 0, (size_t)J.n * dp * wes, st));
    CK(copy_cast_2d(Ty::F64, J.omega, d, wt, X, dp, J.n, d, st));
    s = product(h, Lo, J, false, wt, X, dp, Y);
  }
  if (s != RUQLP_OK) return s;
  // a3: Q = orth(Y).  orth() outputs that only feed the next product enter
  // the result through their span: Y R^{-1} for any upper-triangular R with
  // positive diagonal gives, after the later orth()s, exactly the same Q in
  // exact arithmetic.  On the FP32/BF16 paths those take two CholeskyQR
  // passes (shifted, then plain: orthonormal to about kappa(Y)^2 u, enough to
  // keep the next sketch well conditioned); the last Q and P take three.
  // the orth() before a tensor-core product hands it the transposed BF16 Q
  const bool fuse_bt = J.use_tc && J.dp <= 256;
  bool btY = false, btZ = false;
  s = orth(h, Lo, J, Y, Y, J.m, J.q == 0, fuse_bt, &btY, J.q == 0);
  if (s != RUQLP_OK) return s;
  // a4: power iteration with orthonormalisation (Algorithm 2)
  for (int it = 0; it < J.q; ++it) {
    s = product(h, Lo, J, true, wt, Y, dp, Z, btY);
    if (s != RUQLP_OK) return s;
    s = orth(h, Lo, J, Z, Z, J.n, false, fuse_bt, &btZ);
    if (s != RUQLP_OK) return s;
    s = product(h, Lo, J, false, wt, Z, dp, Y, btZ);
    if (s != RUQLP_OK) return s;
    s = orth(h, Lo, J, Y, Y, J.m, it == J.q - 1, fuse_bt, &btY, it == J.q - 1);
    if (s != RUQLP_OK) return s;
  }
  // a5: B^T = A^T Q (BF16 A: Q as two BF16 parts)
  s = product(h, Lo, J, true, wt, Y, dp, Z, btY, true);
  if (s != RUQLP_OK) return s;
  // a6: [P, R_B] = qr(B^T): P = orth(B^T), R_B = P^T B^T
  s = orth(h, Lo, J, Z, Pb, J.n);
  if (s != RUQLP_OK) return s;
  if (wt == Ty::F64)
    CK(simt_gemm_tn(wt, wt, Ty::F64, Mul::F64, Pb, dp, Z, dp, G, d, d, J.n, d,
                    tn_splits(d, J.n, d, kMaxSplits), partial, nullptr, st));
  else if (!h->orth_simt && gram_tc_supported(J.n, d, dp, Pb) && gram_tc_supported(J.n, d, dp, Z))
    // R_B is upper triangular: its upper triangle on the tensor cores
    CK(gram_tc_upper((const float*)Pb, (const float*)Z, dp, J.n, d, (float*)partial, G,
                     &h->status->timeout, st));
  else
    CK(gram_f32((const float*)Pb, dp, (const float*)Z, dp, J.n, d, d, G, partial, kMaxSplits,
                nullptr, st));
  if (J.finish_paper == 2) {
    // Remark 1: L = U S V^T (one-sided Jacobi on one SM), A ~= (Q U) S (P V)^T;
    // the column-major copy of L is R_B row-major
    void* W = base + Lo.svdW;
    void* Us = base + Lo.svdU;
    void* Vs = base + Lo.svdVs;
    void* QP = base + Lo.T;
    const Mul mm = wt == Ty::F64 ? Mul::F64 : Mul::F32;
    CK(copy_cast_2d(Ty::F64, G, d, wt, W, d, d, d, st));
    CK(svd_jacobi(wt, W, base + Lo.svdV, base + Lo.svdS, d, 40, (int*)(base + Lo.svdOrd),
                  base + Lo.svdTmp, (int*)(base + Lo.svdOrd + (size_t)d * sizeof(int)), Us, Vs,
                  dp, st));
    CK(simt_gemm_nn(wt, wt, wt, mm, Y, dp, Us, dp, QP, dp, J.m, d, d, st));
    CK(simt_gemm_nn(wt, wt, wt, mm, Pb, dp, Vs, dp, X, dp, J.n, d, d, st));
    CK(write_diag(wt, base + Lo.svdS, d, J.ot, J.Lout, st));
    CK(copy_cast_2d(wt, QP, dp, J.ot, J.Qout, d, J.m, d, st));
    CK(copy_cast_2d(wt, X, dp, J.ot, J.Pout, d, J.n, d, st));
    return RUQLP_OK;
  }
  if (J.finish_paper) {
    // Algorithm 1 step 5 in this orientation: [P~, R~] = qr(L), L = R_B^T;
    // Q <- Q P~, middle factor R~ (upper triangular): A ~= (Q P~) R~ P^T.
    void* Lw = X;   // d x dp: L, then P~
    void* Lc = Z;   // d x dp: a copy of L for R~ = P~^T L
    void* QP = base + Lo.T;
    CK(write_L(G, d, wt, Lw, false, st, dp));
    CK(write_L(G, d, wt, Lc, false, st, dp));
    s = orth(h, Lo, J, Lw, Lw, d);
    if (s != RUQLP_OK) return s;
    if (wt == Ty::F64)
      CK(simt_gemm_tn(wt, wt, Ty::F64, Mul::F64, Lw, dp, Lc, dp, G, d, d, d, d,
                      tn_splits(d, d, d, kMaxSplits), partial, nullptr, st));
    else
      CK(gram_f32((const float*)Lw, dp, (const float*)Lc, dp, d, d, d, G, partial, kMaxSplits,
                  nullptr, st));
    CK(simt_gemm_nn(wt, wt, wt, wt == Ty::F64 ? Mul::F64 : Mul::F32, Y, dp, Lw, dp, QP, dp, J.m,
                    d, d, st));
    CK(write_L(G, d, J.ot, J.Lout, true, st));
    CK(copy_cast_2d(wt, QP, dp, J.ot, J.Qout, d, J.m, d, st));
    CK(copy_cast_2d(wt, Pb, dp, J.ot, J.Pout, d, J.n, d, st));
    return RUQLP_OK;
  }
  // a7: outputs
  CK(write_L(G, d, J.ot, J.Lout, false, st));
  CK(copy_cast_2d(wt, Y, dp, J.ot, J.Qout, d, J.m, d, st));
  CK(copy_cast_2d(wt, Pb, dp, J.ot, J.Pout, d, J.n, d, st));
  return RUQLP_OK;
}

ruqlp_status finish(ruqlp_ctx* h, ruqlp_outputs* out) {
  CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profile) prof_collect(h);
  out->flags = (uint32_t)h->status_host->flags;
  if (h->tsqr_now || h->orth_tsqr) out->flags |= RUQLP_FLAG_TSQR;
  if (h->status_host->timeout)
    return fail(h, RUQLP_ERR_TIMEOUT, "a bounded device wait ran out in a tensor-core product");
  if (h->status_host->invalid & 4)
    return fail(h, RUQLP_ERR_INVALID, "a CSR column has more than 1024 nonzeros");
  if (h->status_host->breakdown)
    return fail(h, RUQLP_ERR_BREAKDOWN, "orth() broke down after its fallbacks");
  return RUQLP_OK;
}

}  // namespace


namespace ruqlp {

ruqlp_status single_begin(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                          const ruqlp_outputs* out) {
  int64_t m, n;
  int d;
  ruqlp_status s = validate(h, A, prm, out, &m, &n, &d);
  if (s != RUQLP_OK) return s;
  h->last_A = *A;
  h->last_prm = *prm;
  h->last_out = *out;
  CK(cudaSetDevice(h->device));
  Job J{};
  fill_job(A, prm, out, m, n, d, J);
  J.Qout = out->Q;
  J.Lout = out->L;
  J.Pout = out->P;
  J.use_tc = !J.csr && J.ct == Ty::BF16 && !h->bf16_simt &&
             tc_supported(J.A, J.lda, std::min(J.dp, 256));
  return run_dense(h, J);
}

// A decomposition whose CholeskyQR flagged a numerically rank-deficient
// sketch (RUQLP_FLAG_RANKDEF) is run again with every orth() a Householder
// TSQR, the paper's unpivoted QR taken literally; its flags then carry both
// RUQLP_FLAG_RANKDEF and RUQLP_FLAG_TSQR.
ruqlp_status single_end(ruqlp_ctx* h, ruqlp_outputs* out) {
  ruqlp_status s = finish(h, out);
  if (s != RUQLP_OK || !(out->flags & RUQLP_FLAG_RANKDEF) || h->tsqr_now || h->orth_tsqr)
    return s;
  h->tsqr_now = true;
  s = single_begin(h, &h->last_A, &h->last_prm, &h->last_out);
  if (s == RUQLP_OK) s = finish(h, out);
  h->tsqr_now = false;
  out->flags |= RUQLP_FLAG_RANKDEF;
  return s;
}

ruqlp_status check_request(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                           const ruqlp_outputs* out, int* d) {
  int64_t m, n;
  return validate(h, A, prm, out, &m, &n, d);
}

size_t single_bytes(const ruqlp_matrix* A, const ruqlp_params* prm) {
  Ty ct;
  if (!ty_of(prm->compute, &ct)) return 0;
  const int d = prm->k + prm->p;
  if (A->is_csr) {
    Ty tv;
    if (!ty_of(A->csr.dtype, &tv)) return 0;
    return layout_of(A->csr.m, A->csr.n, d, ct, A->csr.nnz, ty_size(tv), prm->finish_paper,
                     prm->omega == nullptr, A->is_csr == 2 ? A->lr.r : 0)
        .total;
  }
  return layout_of(A->dense.m, A->dense.n, d, ct, -1, 0, prm->finish_paper,
                   prm->omega == nullptr)
      .total;
}

size_t batch_item_bytes(const ruqlp_matrix* A, const ruqlp_params* prm) {
  const int64_t m = A->dense.m, n = A->dense.n;
  const int d = prm->k + prm->p, dp = round16(d);
  int64_t slab;
  const int64_t sl = std::max(gram_slabs(m, kMaxSplits, &slab), gram_slabs(n, kMaxSplits, &slab));
  const size_t per = (size_t)(3 * n + m) * dp * 4 + (size_t)sl * d * d * 8 + (size_t)d * d * 12 +
                     chol_tiles_bytes(d) + (size_t)2 * dp * std::max(m, n) * 2 + 8 * 256;
  // plus its share of the metadata (table entry, prefixes, tile lists, maps)
  return per + 4096 + (size_t)(ceil_div(m, 128) + ceil_div(n, 128)) * 8;
}

bool batchable(const ruqlp_matrix* A, const ruqlp_params* prm) {
  Ty ct;
  const int d = prm->k + prm->p;
  return !A->is_csr && ty_of(prm->compute, &ct) && ct != Ty::F64 && !prm->finish_paper &&
         round16(d) <= 256 && chol_tiles_supported(d) &&
         A->dense.m * A->dense.n <= ((int64_t)1 << 25);
}

void copy_options(const ruqlp_ctx* from, ruqlp_ctx* to) {
  to->orth_fp64 = from->orth_fp64;
  to->orth_full = from->orth_full;
  to->bf16_simt = from->bf16_simt;
  to->orth_simt = from->orth_simt;
  to->batch_orth_tc = from->batch_orth_tc;
  to->orth_tsqr = from->orth_tsqr;
  to->tc_nsplit = from->tc_nsplit;
}

ruqlp_status set_error(ruqlp_ctx* h, ruqlp_status s, const char* msg) {
  return fail(h, s, "%s", msg);
}

}  // namespace ruqlp

// ---------------------------------------------------------------------------
// Batched decompositions (many dense matrices of uneven shapes, FP32 or BF16,
// one q): every phase is one launch over a device problem table (BMat); the
// per-matrix Cholesky runs one CTA per matrix.  The sequence of launches
// depends only on the batch signature and is replayed from a CUDA graph.
// BF16 products run on the tensor cores (one persistent launch over a tile
// list of all matrices) when A's rows are 16-byte aligned, else on the CUDA
// cores; FP32 products on the CUDA cores.  Grams, Cholesky factorisations and
// triangular solves use the same device code and shape-only work splits as
// single decompositions, and every product tile is one K-ordered
// accumulation, so a matrix gets bitwise the same Q, L, P alone (a batch of
// one) and inside any batch; FP32 items (and BF16 with option bf16_simt) also
// equal ruqlp_decompose bitwise.
namespace {

enum { PF_NN = 0, PF_TN, PF_GY, PF_GN, PF_GPZ, PF_TY, PF_TN2, PF_GYW, PF_GNW, NPF };

struct BatchPlan {
  std::vector<BMat> table;
  // CUDA-core work per launch: NN, TN, gramY, gramN (narrow items), gramPZ,
  // trsmY, trsmN, gramY, gramN (wide items)
  std::vector<int> prefix[NPF];
  std::vector<BTcTile> tc_nn, tc_tn;  // tensor-core tile lists
  // tensor-core CholeskyQR items (orth_tc): their list (for k_btrinv) and,
  // over Y (m rows) and over Z (n rows), the Gram units (one row slab each)
  // and the Q = Y R^{-1} units with their per-CTA ranges
  struct BoPlan {
    std::vector<BoUnit> gu, qu;
    std::vector<int> goff, qoff;
    size_t o_gu, o_goff, o_qu, o_qoff;
  } bo[2];
  std::vector<int> bo_items;
  size_t off_bo_items;
  size_t off_meta, off_table, off_prefix[NPF], off_tc_nn, off_tc_tn, off_maps, meta_end;
  size_t off_status, off_err, total;
  int dmax, dpmax_tc, dmax_otc;
  int64_t max_omega, max_out;
};


ruqlp_status batch_launches(ruqlp_ctx* h, const BatchPlan& bp, int count, int q, Ty ct,
                            cudaStream_t st) {
  char* base = (char*)h->arena;
  const BMat* T = (const BMat*)(base + bp.off_table);
  auto pre = [&](int k) { return (const int*)(base + bp.off_prefix[k]); };
  auto tot = [&](int k) { return bp.prefix[k][count]; };
  int* err = (int*)(base + bp.off_err);
  const double s1 = 64.0 * 5.960464477539063e-08;
  // profiling spans only on the eager path (st is the handle's stream there)
  ruqlp_ctx* ph = (st == h->stream) ? h : nullptr;
  ProfScope step(ph, PROF_STEP);
  CK(cudaMemsetAsync(base + bp.off_status, 0, bp.total - bp.off_status, st));
  // make_bt: the last solve also writes the BF16 transposed operand of the
  // next tensor-core product (so that product needs no transpose launch)
  // (items with orth_tc take the tensor-core Gram and Q = Y R^{-1}, the
  // others the CUDA-core kernels; both share the Cholesky launch)
  auto orth_b = [&](int src, int dst, int passes, int make_bt) -> ruqlp_status {
    ProfScope sp(ph, PROF_ORTH);
    const bool y = src == B_Y;
    const int gp = y ? PF_GY : PF_GN, gw = y ? PF_GYW : PF_GNW;
    const int tp = y ? PF_TY : PF_TN2;
    const auto& bo = bp.bo[y ? 0 : 1];
    const int ng = (int)bo.goff.size() - 1, nq = (int)bo.qoff.size() - 1;
    auto dev = [&](size_t o) { return base + o; };
    for (int pass = 0; pass < passes; ++pass) {
      const int from = pass == 0 ? src : dst;
      const int mb = pass == passes - 1 ? make_bt : 0;
      CK(bgram_sym(T, pre(gp), tot(gp), count, from, kMaxSplits, st));
      CK(bgram(T, pre(gw), tot(gw), count, from, from, kMaxSplits, bp.dmax, st, false));
      CK(bgram_tc(T, (const BoUnit*)dev(bo.o_gu), (const int*)dev(bo.o_goff), ng, from,
                  kMaxSplits, err, st));
      if (tot(gp) > 0 || tot(gw) > 0 || ng > 0) CK(bgram_reduce(T, count, from, from, kMaxSplits, bp.dmax, st));
      CK(bchol(T, count, s1, pass == 0, bp.dmax, st, pass == 2));
      CK(btrsm(T, pre(tp), tot(tp), count, from, dst, bp.dmax, st, mb));
      CK(btrinv(T, (const int*)dev(bp.off_bo_items), (int)bp.bo_items.size(), bp.dmax_otc, st));
      CK(bqmul_tc(T, (const BoUnit*)dev(bo.o_qu), (const int*)dev(bo.o_qoff), nq, from, dst, mb,
                  err, st));
    }
    return RUQLP_OK;
  };
  // split2: the two-part skinny operand of B^T = A^T Q (as product() above)
  auto prod = [&](bool trans, int src, int dst, bool split2) -> ruqlp_status {
    ProfScope sp(ph, trans ? PROF_ATX : PROF_AX);
    const int pf = trans ? PF_TN : PF_NN;
    CK(bgemm(trans, ct, Ty::F32, T, pre(pf), tot(pf), count, src, dst, st, split2));
    const auto& list = trans ? bp.tc_tn : bp.tc_nn;
    if (!list.empty()) {  // Bt (and Btl) were written by the step that produced buf[src]
      ProfScope tc(ph, trans ? (split2 ? PROF_TC_ATX2 : PROF_TC_ATX) : PROF_TC_AX);
      CK(btc_gemm(trans, T, count, (const BTcTile*)(base + (trans ? bp.off_tc_tn : bp.off_tc_nn)),
                  (int)list.size(), base + bp.off_maps, src, dst, bp.dpmax_tc, err, st, split2));
    }
    return RUQLP_OK;
  };
  ruqlp_status s;
  CK(bcast_omega(T, count, bp.max_omega, st));
  if ((s = prod(false, B_X, B_Y, false)) != RUQLP_OK) return s;
  if ((s = orth_b(B_Y, B_Y, q == 0 ? 3 : 2, q == 0 ? 2 : 1)) != RUQLP_OK) return s;
  for (int it = 0; it < q; ++it) {
    if ((s = prod(true, B_Y, B_Z, false)) != RUQLP_OK) return s;
    if ((s = orth_b(B_Z, B_Z, 2, 1)) != RUQLP_OK) return s;
    if ((s = prod(false, B_Z, B_Y, false)) != RUQLP_OK) return s;
    if ((s = orth_b(B_Y, B_Y, it == q - 1 ? 3 : 2, it == q - 1 ? 2 : 1)) != RUQLP_OK) return s;
  }
  if ((s = prod(true, B_Y, B_Z, true)) != RUQLP_OK) return s;
  if ((s = orth_b(B_Z, B_P, 3, 0)) != RUQLP_OK) return s;
  CK(bgram(T, pre(PF_GPZ), tot(PF_GPZ), count, B_P, B_Z, kMaxSplits, bp.dmax, st));
  CK(boutputs(T, count, bp.max_out, st));
  return RUQLP_OK;
}

// tile list of the tensor-core items, longest contraction first (CTA c takes
// entries c, c + P, ...; sorting keeps each wave's tiles of similar cost)
void tc_list(const std::vector<BMat>& table, bool trans, std::vector<BTcTile>& out) {
  out.clear();
  std::vector<int> order;
  for (int i = 0; i < (int)table.size(); ++i)
    if (table[i].use_tc) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int64_t kx = trans ? table[x].m : table[x].n, ky = trans ? table[y].m : table[y].n;
    return kx > ky;
  });
  for (int i : order) {
    const int64_t rows = trans ? table[i].n : table[i].m;
    for (int t = 0; t < (int)ceil_div(rows, 128); ++t) out.push_back({i, t});
  }
}

}  // namespace

namespace ruqlp {

ruqlp_status batch_begin(ruqlp_ctx* h, int count, const ruqlp_matrix* A, const ruqlp_params* prm,
                         const ruqlp_outputs* out, bool graphs_ok, BatchRun* run) {
  if (count < 1 || !A || !prm || !out) return fail(h, RUQLP_ERR_INVALID, "empty or NULL batch");
  Ty ct0 = Ty::F32;
  int q0 = 0;
  std::vector<int> dd(count);
  for (int i = 0; i < count; ++i) {
    int64_t m, n;
    ruqlp_status s = validate(h, &A[i], &prm[i], &out[i], &m, &n, &dd[i]);
    if (s != RUQLP_OK) return fail(h, s, "batch item %d: %s", i, h->err.c_str());
    if (A[i].is_csr) return fail(h, RUQLP_ERR_INVALID, "batch item %d: CSR is not batched", i);
    Ty ct;
    ty_of(prm[i].compute, &ct);
    if (ct == Ty::F64) return fail(h, RUQLP_ERR_INVALID, "batches are FP32 or BF16");
    if (i == 0) {
      ct0 = ct;
      q0 = prm[i].q;
    } else if (ct != ct0 || prm[i].q != q0) {
      return fail(h, RUQLP_ERR_INVALID, "all items of a batch need the same dtype and q");
    }
    if (prm[i].finish_paper) return fail(h, RUQLP_ERR_INVALID, "finish_paper is not batched");
    if (!chol_tiles_supported(dd[i])) return fail(h, RUQLP_ERR_INVALID, "batched d must be <= 288");
  }
  CK(cudaSetDevice(h->device));
  // workspace: per-matrix buffers; the metadata block (table, prefix arrays,
  // tile lists, tensor maps: uploaded in one copy); statuses and an error word
  BatchPlan bp;
  bp.table.resize(count);
  bp.dmax = 0;
  bp.dpmax_tc = 0;
  bp.dmax_otc = 0;
  bp.max_omega = 0;
  bp.max_out = 0;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  std::vector<size_t> oX(count), oY(count), oZ(count), oP(count), oPa(count), oG(count),
      oT(count), oB(count), oGf(count), oS(count);
  for (int i = 0; i < count; ++i) {
    const ruqlp_dense& D = A[i].dense;
    const int64_t m = D.m, n = D.n;
    const int d = dd[i], dp = round16(d);
    BMat& b = bp.table[i];
    b.use_tc = (ct0 == Ty::BF16 && !h->bf16_simt && tc_supported(D.data, D.ld, dp)) ? 1 : 0;
    // option batch_orth_tc: BF16 items of width dp <= 80 run their
    // CholeskyQR passes on the tensor cores (a rule on the dtype, the
    // options and d only, so an item decides the same alone and in any
    // batch).  Off by default: at these widths the three-way BF16 split
    // costs the converter warps more per value than the CUDA-core Gram's d
    // multiply-adds (measured slower on the batched workload)
    b.orth_tc = (ct0 == Ty::BF16 && h->batch_orth_tc && !h->bf16_simt && !h->orth_simt &&
                 dp <= BO_DPMAX)
                    ? 1
                    : 0;
    b.ldbt = align_up((size_t)std::max(m, n), 8);
    int64_t slab;
    const int64_t sl = std::max(gram_slabs(m, kMaxSplits, &slab), gram_slabs(n, kMaxSplits, &slab));
    oX[i] = take((size_t)n * dp * 4);
    oY[i] = take((size_t)m * dp * 4);
    oZ[i] = take((size_t)n * dp * 4);
    oP[i] = take((size_t)n * dp * 4);
    oPa[i] = take((size_t)sl * d * d * 8);
    oG[i] = take((size_t)d * d * 8);
    oGf[i] = take((size_t)d * d * 4);
    oT[i] = take(chol_tiles_bytes(d));
    oB[i] = b.use_tc ? take((size_t)2 * dp * b.ldbt * 2) : 0;  // Bt, then Btl
    oS[i] = b.orth_tc ? take(bo_st_bytes(d)) : 0;
    if (b.orth_tc) bp.dmax_otc = std::max(bp.dmax_otc, d);
    bp.dmax = std::max(bp.dmax, d);
    if (b.use_tc) bp.dpmax_tc = std::max(bp.dpmax_tc, dp);
    bp.max_omega = std::max<int64_t>(bp.max_omega, n * dp);
    bp.max_out = std::max<int64_t>(bp.max_out, (m + n) * d + (int64_t)d * d);
  }
  // each prefix array: count + 1 tile offsets over the launch order, then
  // the order itself (count item indices)
  for (int k = 0; k < NPF; ++k) bp.prefix[k].assign(2 * count + 1, 0);
  bp.off_meta = off;
  bp.off_table = take(sizeof(BMat) * count);
  for (int k = 0; k < NPF; ++k) bp.off_prefix[k] = take(sizeof(int) * (2 * count + 1));
  // tile lists are sized below, after the table is filled
  size_t n_nn = 0, n_tn = 0;
  for (int i = 0; i < count; ++i)
    if (bp.table[i].use_tc) {
      n_nn += ceil_div(A[i].dense.m, 128);
      n_tn += ceil_div(A[i].dense.n, 128);
    }
  bp.off_tc_nn = take(sizeof(BTcTile) * std::max<size_t>(n_nn, 1));
  bp.off_tc_tn = take(sizeof(BTcTile) * std::max<size_t>(n_tn, 1));
  {
    // tensor-core CholeskyQR work: Gram units are the row slabs of
    // gram_slabs() (the summation order, a function of the shape), dealt to
    // at most one CTA per SM in contiguous runs of about equal rows; Q = Y
    // R^{-1} cuts the items' rows into one run per CTA, multiples of the
    // 128-row sub-tile (any cut gives the same rows of Q)
    const int G = sm_count();
    for (int i = 0; i < count; ++i)
      if (bp.table[i].orth_tc) bp.bo_items.push_back(i);
    for (int kind = 0; kind < 2; ++kind) {
      auto& bo = bp.bo[kind];
      auto rows = [&](int i) { return kind == 0 ? A[i].dense.m : A[i].dense.n; };
      int64_t R = 0;
      for (int i : bp.bo_items) {
        int64_t slab;
        gram_slabs(rows(i), kMaxSplits, &slab);
        for (int64_t r0 = 0; r0 < rows(i); r0 += slab)
          bo.gu.push_back({i, (int)std::min<int64_t>(slab, rows(i) - r0), r0});
        R += rows(i);
      }
      // (a run also ends at BO_MAXU units, the CTA's descriptor table)
      bo.goff.assign(1, 0);
      const int gg = std::min<int>(G, (int)bo.gu.size());
      int64_t acc = 0;
      for (int u = 0; u < (int)bo.gu.size(); ++u) {
        acc += bo.gu[u].rows;
        const int c = (int)bo.goff.size();
        if ((c < gg && acc * gg >= (int64_t)c * R) || u + 1 - bo.goff.back() == BO_MAXU)
          bo.goff.push_back(u + 1);
      }
      if (bo.goff.back() != (int)bo.gu.size()) bo.goff.push_back((int)bo.gu.size());
      bo.qoff.assign(1, 0);
      const int64_t quota = std::max<int64_t>(128, ceil_div(ceil_div(R, G), 128) * 128);
      int64_t fill = 0;
      for (int i : bp.bo_items) {
        for (int64_t r0 = 0; r0 < rows(i);) {
          const int64_t take_rows = std::min(rows(i) - r0, quota - fill);
          bo.qu.push_back({i, (int)take_rows, r0});
          r0 += take_rows;
          fill += take_rows;
          if (fill == quota || (int)bo.qu.size() - bo.qoff.back() == BO_MAXU) {
            bo.qoff.push_back((int)bo.qu.size());
            fill = 0;
          }
        }
      }
      if (bo.qoff.back() != (int)bo.qu.size()) bo.qoff.push_back((int)bo.qu.size());
      bo.o_gu = take(sizeof(BoUnit) * std::max<size_t>(bo.gu.size(), 1));
      bo.o_goff = take(sizeof(int) * bo.goff.size());
      bo.o_qu = take(sizeof(BoUnit) * std::max<size_t>(bo.qu.size(), 1));
      bo.o_qoff = take(sizeof(int) * bo.qoff.size());
    }
    bp.off_bo_items = take(sizeof(int) * std::max<size_t>(bp.bo_items.size(), 1));
  }
  const size_t map3 = btc_map_bytes();  // all tensor maps of one matrix
  bp.off_maps = take(map3 * count);
  bp.meta_end = off;
  bp.off_status = take(sizeof(DevStatus) * count);
  bp.off_err = take(sizeof(int));
  bp.total = off;
  ruqlp_status s = ensure_arena(h, bp.total);
  if (s != RUQLP_OK) return s;
  char* base = (char*)h->arena;
  std::vector<int> cnts[NPF];
  for (int k = 0; k < NPF; ++k) cnts[k].assign(count, 0);
  for (int i = 0; i < count; ++i) {
    BMat& b = bp.table[i];
    const ruqlp_dense& D = A[i].dense;
    b.A = D.data;
    b.lda = D.ld;
    b.m = D.m;
    b.n = D.n;
    b.d = dd[i];
    b.dp = round16(dd[i]);
    Ty ot;
    ty_of(out[i].out_dtype, &ot);
    b.ot = (int)ot;
    b.X = (float*)(base + oX[i]);
    b.Y = (float*)(base + oY[i]);
    b.Z = (float*)(base + oZ[i]);
    b.P = (float*)(base + oP[i]);
    b.partial = (double*)(base + oPa[i]);
    b.G = (double*)(base + oG[i]);
    b.Gf = (float*)(base + oGf[i]);
    b.tiles = (float*)(base + oT[i]);
    b.Bt = b.use_tc ? (void*)(base + oB[i]) : nullptr;
    b.Btl = b.use_tc ? (void*)(base + oB[i] + (size_t)b.dp * b.ldbt * 2) : nullptr;
    b.St = b.orth_tc ? (void*)(base + oS[i]) : nullptr;
    b.omega = prm[i].omega;
    b.seed = prm[i].omega_seed;
    b.Qout = out[i].Q;
    // (rows of Qout on 16 bytes, so the solve's 128-bit stores stay)
    b.q_direct = (b.use_tc && !b.orth_tc && ot == Ty::F32 && b.d % 4 == 0 &&
                  ((uintptr_t)b.Qout & 15) == 0) ? 1 : 0;
    b.Lout = out[i].L;
    b.Pout = out[i].P;
    b.status = (DevStatus*)(base + bp.off_status) + i;
    const bool cc = !b.orth_tc;  // CholeskyQR on the CUDA cores
    const bool narrow = bgram_sym_ctas(b.m, b.d, kMaxSplits) > 0;
    const int cnt[NPF] = {b.use_tc ? 0 : bgemm_tiles(b.m, b.d),
                          b.use_tc ? 0 : bgemm_tiles(b.n, b.d),
                          cc ? bgram_sym_ctas(b.m, b.d, kMaxSplits) : 0,
                          cc ? bgram_sym_ctas(b.n, b.d, kMaxSplits) : 0,
                          bgram_tiles(b.n, b.d, false, kMaxSplits),
                          cc ? btrsm_blocks(b.m) : 0,
                          cc ? btrsm_blocks(b.n) : 0,
                          cc && !narrow ? bgram_tiles(b.m, b.d, true, kMaxSplits) : 0,
                          cc && !narrow ? bgram_tiles(b.n, b.d, true, kMaxSplits) : 0};
    for (int k = 0; k < NPF; ++k) cnts[k][i] = cnt[k];
  }
  // the CUDA-core launches take their tiles widest item first (a tile's cost
  // grows with d^2), so the last wave holds the cheapest tiles; a tile's
  // result does not depend on when it runs
  {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      const BMat &a = bp.table[x], &b = bp.table[y];
      if (a.dp != b.dp) return a.dp > b.dp;
      return a.m + a.n > b.m + b.n;
    });
    for (int k = 0; k < NPF; ++k) {
      for (int pos = 0; pos < count; ++pos) {
        bp.prefix[k][pos + 1] = bp.prefix[k][pos] + cnts[k][order[pos]];
        bp.prefix[k][count + 1 + pos] = order[pos];
      }
    }
  }
  tc_list(bp.table, false, bp.tc_nn);
  tc_list(bp.table, true, bp.tc_tn);
  // signature: the launch sequence depends on shapes, q, dtype, product
  // kernels and the arena
  std::vector<int64_t> key = {count, q0, (int64_t)ct0, (int64_t)(uintptr_t)h->arena};
  for (int i = 0; i < count; ++i) {
    key.push_back(bp.table[i].m);
    key.push_back(bp.table[i].n);
    key.push_back(bp.table[i].d);
    key.push_back(bp.table[i].use_tc);
    key.push_back(bp.table[i].orth_tc);
  }
  ruqlp_ctx::BatchEntry* g = nullptr;
  for (auto& c : h->batches)
    if (c.key == key) g = &c;
  if (!g) {
    if (h->batches.size() >= 8) {
      if (h->batches.front().exec) cudaGraphExecDestroy(h->batches.front().exec);
      h->batches.erase(h->batches.begin());
    }
    h->batches.emplace_back();
    g = &h->batches.back();
    g->key = key;
    g->maps.assign(map3 * count, 0);
    g->aptr.assign(count, nullptr);
    g->alda.assign(count, 0);
  }
  // tensor maps: Bt maps depend on the signature only; A maps are re-encoded
  // when the caller's A pointer or stride changes
  for (int i = 0; i < count; ++i) {
    const BMat& b = bp.table[i];
    if (!b.use_tc || (g->aptr[i] == b.A && g->alda[i] == b.lda)) continue;
    if (!btc_encode(g->maps.data() + map3 * i, b.A, b.lda, b.m, b.n, b.Bt, b.Btl, b.ldbt, b.dp,
                    g->aptr[i] != nullptr))
      return fail(h, RUQLP_ERR_INVALID, "batch item %d: tensor map encoding failed", i);
    g->aptr[i] = b.A;
    g->alda[i] = b.lda;
  }
  // metadata image in pinned memory, one upload
  const size_t meta = bp.meta_end - bp.off_meta;
  if (h->stage_bytes < meta) {
    if (h->stage) cudaFreeHost(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    CK(cudaMallocHost(&h->stage, meta));
    h->stage_bytes = meta;
  }
  char* img = (char*)h->stage;
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (bytes) memcpy(img + (o - bp.off_meta), src, bytes);
  };
  put(bp.off_table, bp.table.data(), sizeof(BMat) * count);
  for (int k = 0; k < NPF; ++k)
    put(bp.off_prefix[k], bp.prefix[k].data(), sizeof(int) * (2 * count + 1));
  put(bp.off_tc_nn, bp.tc_nn.data(), sizeof(BTcTile) * bp.tc_nn.size());
  put(bp.off_tc_tn, bp.tc_tn.data(), sizeof(BTcTile) * bp.tc_tn.size());
  put(bp.off_maps, g->maps.data(), g->maps.size());
  for (const auto& bo : bp.bo) {
    put(bo.o_gu, bo.gu.data(), sizeof(BoUnit) * bo.gu.size());
    put(bo.o_goff, bo.goff.data(), sizeof(int) * bo.goff.size());
    put(bo.o_qu, bo.qu.data(), sizeof(BoUnit) * bo.qu.size());
    put(bo.o_qoff, bo.qoff.data(), sizeof(int) * bo.qoff.size());
  }
  put(bp.off_bo_items, bp.bo_items.data(), sizeof(int) * bp.bo_items.size());
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(base + bp.off_meta, img, meta, cudaMemcpyHostToDevice, st));
  const bool graphs = graphs_ok && h->batch_graphs && !h->profile;  // profiling runs eagerly
  if (graphs && g->exec) {
    CK(cudaGraphLaunch(g->exec, st));
    ruqlp::count_launch((int)g->launches);
  } else if (graphs && g->seen > 0) {  // second sighting of the signature: capture it
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = ruqlp::launch_count();
    s = batch_launches(h, bp, count, q0, ct0, h->cap_stream);
    g->launches = ruqlp::launch_count() - l0;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    if (s != RUQLP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    CK(ec);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    g->exec = exec;
    CK(cudaGraphLaunch(exec, st));
  } else {
    s = batch_launches(h, bp, count, q0, ct0, st);
    if (s != RUQLP_OK) return s;
  }
  g->seen++;
  run->count = count;
  run->off_status = bp.off_status;
  run->off_err = bp.off_err;
  run->A.assign(A, A + count);
  run->prm.assign(prm, prm + count);
  return RUQLP_OK;
}

ruqlp_status batch_end(ruqlp_ctx* h, const BatchRun& run, ruqlp_outputs* out) {
  char* base = (char*)h->arena;
  cudaStream_t st = h->stream;
  std::vector<DevStatus> stat(run.count);
  int derr = 0;
  CK(cudaMemcpyAsync(stat.data(), base + run.off_status, sizeof(DevStatus) * run.count,
                     cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&derr, base + run.off_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h->profile) prof_collect(h);
  for (int i = 0; i < run.count; ++i) out[i].flags = (uint32_t)stat[i].flags;
  if (derr) return fail(h, RUQLP_ERR_TIMEOUT, "a bounded device wait ran out in a batched kernel");
  // items whose sketch CholeskyQR could not orthonormalise: alone on the
  // single-matrix path, which reruns them with Householder TSQR (as it would
  // had they come alone)
  for (int i = 0; i < run.count; ++i) {
    if (!(out[i].flags & RUQLP_FLAG_RANKDEF) || i >= (int)run.A.size()) continue;
    ruqlp_outputs o = out[i];
    ruqlp_status s = single_begin(h, &run.A[i], &run.prm[i], &o);
    if (s == RUQLP_OK) s = single_end(h, &o);
    if (s != RUQLP_OK) return fail(h, s, "batch item %d (TSQR rerun): %s", i, h->err.c_str());
    out[i].flags = o.flags;
  }
  return RUQLP_OK;
}

}  // namespace ruqlp

extern "C" ruqlp_status ruqlp_decompose_batch(ruqlp_handle h, int count, const ruqlp_matrix* A,
                                              const ruqlp_params* prm, ruqlp_outputs* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  BatchRun run;
  ruqlp_status s = batch_begin(h, count, A, prm, out, true, &run);
  if (s != RUQLP_OK) return s;
  return batch_end(h, run, out);
}

extern "C" {

const char* ruqlp_version(void) { return kVersion; }

ruqlp_status ruqlp_create(ruqlp_handle* out, const ruqlp_config* cfg) {
  if (!out || !cfg) return RUQLP_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return RUQLP_ERR_CUDA;
  if (cfg->device < 0 || cfg->device >= ndev) return RUQLP_ERR_INVALID;
  ruqlp_ctx* h = new ruqlp_ctx();
  h->device = cfg->device;
  h->stream = (cudaStream_t)cfg->cuda_stream;
  h->budget = cfg->hbm_budget_bytes;
  h->max_slots = cfg->max_slots > 0 ? cfg->max_slots : 8;
  if (cudaSetDevice(h->device) != cudaSuccess ||
      cudaMalloc(&h->status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&h->status_host, sizeof(DevStatus)) != cudaSuccess) {
    if (h->status) cudaFree(h->status);
    delete h;
    return RUQLP_ERR_CUDA;
  }
  *out = h;
  return RUQLP_OK;
}

ruqlp_status ruqlp_destroy(ruqlp_handle h) {
  if (!h) return RUQLP_ERR_INVALID;
  server_shutdown(h);
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->batches)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int i = 0; i < ruqlp_ctx::kCopyStreams; ++i)
    if (h->copy_streams[i]) cudaStreamDestroy(h->copy_streams[i]);
  for (int i = 0; i <= ruqlp_ctx::kCopyStreams; ++i)
    if (h->copy_ev[i]) cudaEventDestroy(h->copy_ev[i]);
  if (h->stage) cudaFreeHost(h->stage);
  if (h->arena) cudaFree(h->arena);
  if (h->status) cudaFree(h->status);
  if (h->status_host) cudaFreeHost(h->status_host);
  delete h;
  return RUQLP_OK;
}

ruqlp_status ruqlp_set_stream(ruqlp_handle h, void* stream) {
  if (!h) return RUQLP_ERR_INVALID;
  h->stream = (cudaStream_t)stream;
  return RUQLP_OK;
}

ruqlp_status ruqlp_set_option(ruqlp_handle h, const char* name, int64_t value) {
  if (!h || !name) return RUQLP_ERR_INVALID;
  if (strcmp(name, "batch_graph") == 0) {
    h->batch_graphs = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "orth_full") == 0) {
    h->orth_full = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "orth_fp64") == 0) {
    h->orth_fp64 = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "bf16_simt") == 0) {
    h->bf16_simt = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "orth_simt") == 0) {
    h->orth_simt = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "batch_orth_tc") == 0) {
    h->batch_orth_tc = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "orth_tsqr") == 0) {
    h->orth_tsqr = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "test_withhold_stage") == 0) {
    h->test_withhold = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "tc_nsplit") == 0) {
    if (value != 0 && value != 1 && value != 2 && value != 4)
      return fail(h, RUQLP_ERR_INVALID, "tc_nsplit must be 0 (tuned), 1, 2 or 4");
    h->tc_nsplit = (int)value;
    return RUQLP_OK;
  }
  if (strcmp(name, "profile") == 0) {
    h->profile = value != 0;
    for (int i = 0; i < kProfN; ++i) {
      h->prof_count[i] = 0;
      h->prof_ms[i] = 0.0;
    }
    return RUQLP_OK;
  }
  return fail(h, RUQLP_ERR_INVALID, "unknown option '%s'", name);
}

size_t ruqlp_workspace_bytes(int64_t m, int64_t n, int d, ruqlp_dtype compute, int64_t nnz) {
  Ty ct;
  if (m < 1 || n < 1 || d < 1 || d > 512 || !ty_of(compute, &ct)) return 0;
  if (nnz >= 0) {
    if (ct == Ty::F64) return 0;
    return layout_of(m, n, d, Ty::F32, nnz, ty_size(ct)).total;
  }
  return layout_of(m, n, d, ct).total;
}

ruqlp_status ruqlp_reserve(ruqlp_handle h, int64_t m, int64_t n, int d, ruqlp_dtype compute,
                           int64_t nnz) {
  if (!h) return RUQLP_ERR_INVALID;
  const size_t b = ruqlp_workspace_bytes(m, n, d, compute, nnz);
  if (b == 0) return fail(h, RUQLP_ERR_INVALID, "invalid sizes for ruqlp_reserve");
  return ensure_arena(h, b);
}

ruqlp_status ruqlp_decompose(ruqlp_handle h, const ruqlp_matrix* A, const ruqlp_params* prm,
                             ruqlp_outputs* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  ruqlp_status s = single_begin(h, A, prm, out);
  if (s != RUQLP_OK) return s;
  return single_end(h, out);
}

// A 2-D copy (rows of `width` bytes) split by rows over the handle's copy
// streams, so that several copy engines share it; it starts once `st` reaches
// this point and `st` continues once every part has landed.  Contiguous
// blocks (both pitches equal to the width) go as 1-D copies.
static ruqlp_status copy_split(ruqlp_ctx* h, void* dst, size_t dpitch, const void* src,
                               size_t spitch, size_t width, size_t rows, cudaMemcpyKind kind,
                               cudaStream_t st) {
  constexpr int NS = ruqlp_ctx::kCopyStreams;
  if (!h->copy_streams[0]) {
    for (int i = 0; i < NS; ++i)
      CK(cudaStreamCreateWithFlags(&h->copy_streams[i], cudaStreamNonBlocking));
    for (int i = 0; i <= NS; ++i) CK(cudaEventCreateWithFlags(&h->copy_ev[i], cudaEventDisableTiming));
  }
  const int parts = (int)std::min<size_t>(NS, std::max<size_t>(1, rows * width >> 24));  // >= 16 MB each
  CK(cudaEventRecord(h->copy_ev[NS], st));
  const bool flat = dpitch == width && spitch == width;
  for (int i = 0; i < parts; ++i) {
    const size_t r0 = rows * i / parts, r1 = rows * (i + 1) / parts;
    cudaStream_t cs = h->copy_streams[i];
    CK(cudaStreamWaitEvent(cs, h->copy_ev[NS], 0));
    char* d = (char*)dst + r0 * dpitch;
    const char* s = (const char*)src + r0 * spitch;
    if (flat) CK(cudaMemcpyAsync(d, s, (r1 - r0) * width, kind, cs));
    else CK(cudaMemcpy2DAsync(d, dpitch, s, spitch, width, r1 - r0, kind, cs));
    CK(cudaEventRecord(h->copy_ev[i], cs));
    CK(cudaStreamWaitEvent(st, h->copy_ev[i], 0));
  }
  return RUQLP_OK;
}

static ruqlp_status decompose_host_once(ruqlp_handle h, const ruqlp_matrix* A,
                                       const ruqlp_params* prm, ruqlp_outputs* out);

ruqlp_status ruqlp_decompose_host(ruqlp_handle h, const ruqlp_matrix* A,
                                  const ruqlp_params* prm, ruqlp_outputs* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  ruqlp_status s = decompose_host_once(h, A, prm, out);
  if (s != RUQLP_OK || !(out->flags & RUQLP_FLAG_RANKDEF) || h->orth_tsqr) return s;
  // numerically rank-deficient sketch: again, with Householder TSQR orth()s
  h->tsqr_now = true;
  s = decompose_host_once(h, A, prm, out);
  h->tsqr_now = false;
  out->flags |= RUQLP_FLAG_RANKDEF;
  return s;
}

static ruqlp_status decompose_host_once(ruqlp_handle h, const ruqlp_matrix* A,
                                       const ruqlp_params* prm, ruqlp_outputs* out) {
  int64_t m, n;
  int d;
  ruqlp_status s = validate(h, A, prm, out, &m, &n, &d);
  if (s != RUQLP_OK) return s;
  if (A->is_csr == 2)
    return fail(h, RUQLP_ERR_INVALID, "a low-rank term needs the device entry points");
  CK(cudaSetDevice(h->device));
  Job J{};
  fill_job(A, prm, out, m, n, d, J);
  const size_t oes = ty_size(J.ot);
  // the workspace first, then staging for A, Omega and the outputs
  const bool gen = prm->omega == nullptr;  // run_dense's layout, which comes first
  const bool ts = h->tsqr_now || h->orth_tsqr;
  const Layout Lo = J.csr ? layout_of(m, n, d, J.ct, J.nnz, ty_size(J.tv), J.finish_paper, gen,
                                      0, ts)
                          : layout_of(m, n, d, J.ct, -1, 0, J.finish_paper, gen, 0, ts);
  size_t off = align_up(Lo.total, 256);
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  size_t oA = 0, oRp = 0, oCi = 0, oV = 0;
  int64_t lds = n;
  if (J.csr) {
    oRp = take((size_t)(m + 1) * sizeof(int32_t));
    oCi = take((size_t)(J.nnz > 0 ? J.nnz : 1) * sizeof(int32_t));
    oV = take((size_t)(J.nnz > 0 ? J.nnz : 1) * ty_size(J.tv));
  } else {
    lds = (J.ct == Ty::BF16) ? round8(n) : n;  // TMA needs a 16-byte row pitch
    oA = take((size_t)m * lds * ty_size(J.ct));
  }
  const size_t oOm = prm->omega ? take((size_t)n * d * sizeof(double)) : 0;
  const size_t oQ = take((size_t)m * d * oes);
  const size_t oL = take((size_t)d * d * oes);
  const size_t oP = take((size_t)n * d * oes);
  s = ensure_arena(h, off);
  if (s != RUQLP_OK) return s;
  char* base = (char*)h->arena;
  cudaStream_t st = h->stream;
  if (J.csr) {
    CK(cudaMemcpyAsync(base + oRp, A->csr.rowptr, (size_t)(m + 1) * sizeof(int32_t),
                       cudaMemcpyHostToDevice, st));
    if (J.nnz > 0) {
      CK(cudaMemcpyAsync(base + oCi, A->csr.colidx, (size_t)J.nnz * sizeof(int32_t),
                         cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(base + oV, A->csr.values, (size_t)J.nnz * ty_size(J.tv),
                         cudaMemcpyHostToDevice, st));
    }
    J.rowptr = (const int32_t*)(base + oRp);
    J.colidx = (const int32_t*)(base + oCi);
    J.vals = base + oV;
  } else {
    const size_t aes = ty_size(J.ct);
    s = copy_split(h, base + oA, (size_t)lds * aes, A->dense.data, (size_t)A->dense.ld * aes,
                   (size_t)n * aes, (size_t)m, cudaMemcpyHostToDevice, st);
    if (s != RUQLP_OK) return s;
    J.A = base + oA;
    J.lda = lds;
  }
  if (prm->omega) {
    CK(cudaMemcpyAsync(base + oOm, prm->omega, (size_t)n * d * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    J.omega = (const double*)(base + oOm);
  }  // else generated on the device by run_dense
  J.Qout = base + oQ;
  J.Lout = base + oL;
  J.Pout = base + oP;
  J.use_tc = !J.csr && J.ct == Ty::BF16 && !h->bf16_simt &&
             tc_supported(J.A, J.lda, std::min(J.dp, 256));
  s = run_dense(h, J);
  if (s != RUQLP_OK) return s;
  s = copy_split(h, out->Q, (size_t)d * oes, base + oQ, (size_t)d * oes, (size_t)d * oes,
                 (size_t)m, cudaMemcpyDeviceToHost, st);
  if (s != RUQLP_OK) return s;
  CK(cudaMemcpyAsync(out->L, base + oL, (size_t)d * d * oes, cudaMemcpyDeviceToHost, st));
  s = copy_split(h, out->P, (size_t)d * oes, base + oP, (size_t)d * oes, (size_t)d * oes,
                 (size_t)n, cudaMemcpyDeviceToHost, st);
  if (s != RUQLP_OK) return s;
  return finish(h, out);
}

ruqlp_status ruqlp_omega(ruqlp_handle h, int64_t n, int d, uint64_t seed, double* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  if (n < 1 || d < 1 || !out) return fail(h, RUQLP_ERR_INVALID, "invalid arguments to ruqlp_omega");
  CK(cudaSetDevice(h->device));
  CK(omega_philox(seed, n, d, out, d, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RUQLP_OK;
}

const char* ruqlp_last_error(ruqlp_handle h) { return h ? h->err.c_str() : "NULL handle"; }

int64_t ruqlp_launch_count(void) { return launch_count(); }

int ruqlp_tune_file(const char* path) { return tune_file(path); }

ruqlp_status ruqlp_sketch(ruqlp_handle h, const ruqlp_matrix* A, int trans, const void* X,
                          int64_t ldx, int d, void* Y, int64_t ldy) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  if (!A || !X || !Y) return fail(h, RUQLP_ERR_INVALID, "NULL argument");
  if (d < 1 || d > 512 || ldx < d || ldy < d)
    return fail(h, RUQLP_ERR_INVALID, "need 1 <= d <= 512, ldx >= d, ldy >= d");
  // reuse the decomposition's checks with a stand-in parameter set
  ruqlp_params prm{};
  prm.k = 1;
  prm.p = 0;
  prm.q = 0;
  prm.compute = A->is_csr ? A->csr.dtype : A->dense.dtype;
  prm.omega = (const double*)X;
  ruqlp_outputs o{};
  o.Q = o.L = o.P = Y;
  o.out_dtype = RUQLP_F32;
  int64_t m, n;
  int d1;
  ruqlp_status s = validate(h, A, &prm, &o, &m, &n, &d1);
  if (s != RUQLP_OK) return s;
  CK(cudaSetDevice(h->device));
  Job J{};
  fill_job(A, &prm, &o, m, n, 1, J);
  J.d = d;
  J.dp = round16(d);
  J.use_tc = !J.csr && J.ct == Ty::BF16 && !h->bf16_simt &&
             tc_supported(J.A, J.lda, std::min(J.dp, 256));
  const int64_t Mout = trans ? n : m;
  const Layout Lo = J.csr ? layout_of(m, n, d, J.ct, J.nnz, ty_size(J.tv), false, false, J.lr_r)
                          : layout_of(m, n, d, J.ct);
  s = ensure_arena(h, Lo.total);
  if (s != RUQLP_OK) return s;
  CK(status_reset(h->status, h->stream));
  if (J.csr) {
    s = prepare_csr(h, Lo, J);
    if (s != RUQLP_OK) return s;
  }
  void* stage = (char*)h->arena + (trans ? Lo.Z : Lo.Y);
  const void* Xuse = X;
  int64_t ldxu = ldx;
  if (J.csr && ((ldx % 4) || ((uintptr_t)X & 15))) {  // 128-bit gathers need aligned rows
    void* Xa = (char*)h->arena + (trans ? Lo.Y : Lo.X);  // m x dp or n x dp
    const int64_t K = trans ? m : n;
    CK(copy_cast_2d(J.wt, X, ldx, J.wt, Xa, J.dp, K, d, h->stream));
    Xuse = Xa;
    ldxu = J.dp;
  }
  s = product(h, Lo, J, trans != 0, J.wt, Xuse, ldxu, stage);
  if (s != RUQLP_OK) return s;
  CK(copy_cast_2d(J.wt, stage, J.dp, J.wt, Y, ldy, Mout, d, h->stream));
  ruqlp_outputs dummy{};
  return finish(h, &dummy);
}

ruqlp_status ruqlp_orth(ruqlp_handle h, const void* Y, int64_t M, int d, int64_t ldy,
                        ruqlp_dtype dtype, void* Q, int64_t ldq) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  if (!Y || !Q) return fail(h, RUQLP_ERR_INVALID, "NULL pointer");
  if (d < 1 || d > 512 || M < d || ldy < d || ldq < d)
    return fail(h, RUQLP_ERR_INVALID, "need 1 <= d <= 512, M >= d, ldy >= d, ldq >= d");
  if (dtype != RUQLP_F64 && dtype != RUQLP_F32)
    return fail(h, RUQLP_ERR_INVALID, "dtype must be F64 or F32");
  CK(cudaSetDevice(h->device));
  Job J{};
  J.m = M;
  J.n = d;
  J.d = d;
  J.dp = round16(d);
  J.ct = dtype == RUQLP_F64 ? Ty::F64 : Ty::F32;
  J.wt = J.ct;
  // CholeskyQR first; a numerically rank-deficient Y goes again through the
  // Householder TSQR
  ruqlp_outputs dummy{};
  for (int attempt = 0; attempt < 2; ++attempt) {
    h->tsqr_now = attempt == 1;
    const Layout Lo = layout_of(M, d, d, J.ct, -1, 0, 0, false, 0, h->tsqr_now || h->orth_tsqr);
    ruqlp_status s = ensure_arena(h, Lo.total);
    if (s == RUQLP_OK) {
      void* W = (char*)h->arena + Lo.Y;
      CK(status_reset(h->status, h->stream));
      CK(copy_cast_2d(J.wt, Y, ldy, J.wt, W, J.dp, M, d, h->stream));
      s = orth(h, Lo, J, W, W, M);
      if (s == RUQLP_OK) {
        CK(copy_cast_2d(J.wt, W, J.dp, J.wt, Q, ldq, M, d, h->stream));
        s = finish(h, &dummy);
      }
    }
    h->tsqr_now = false;
    if (s != RUQLP_OK || !(dummy.flags & RUQLP_FLAG_RANKDEF) || h->orth_tsqr) return s;
  }
  return RUQLP_OK;
}

ruqlp_status ruqlp_gram(ruqlp_handle h, const void* Y, int64_t M, int d, int64_t ldy,
                        ruqlp_dtype dtype, double* G) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  if (!Y || !G) return fail(h, RUQLP_ERR_INVALID, "NULL pointer");
  if (M < 1 || d < 1 || d > 512 || ldy < d)
    return fail(h, RUQLP_ERR_INVALID, "need M >= 1, 1 <= d <= 512, ldy >= d");
  if (dtype != RUQLP_F64 && dtype != RUQLP_F32)
    return fail(h, RUQLP_ERR_INVALID, "dtype must be F64 or F32");
  const Ty ty = dtype == RUQLP_F64 ? Ty::F64 : Ty::F32;
  const size_t bytes = (size_t)kMaxSplits * d * d * sizeof(double);
  ruqlp_status s = ensure_arena(h, bytes);
  if (s != RUQLP_OK) return s;
  CK(cudaSetDevice(h->device));
  CK(simt_gemm_tn(ty, ty, Ty::F64, Mul::F64, Y, ldy, Y, ldy, G, d, d, M, d,
                  tn_splits(d, M, d, kMaxSplits), (double*)h->arena, nullptr, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RUQLP_OK;
}

ruqlp_status ruqlp_profile(ruqlp_handle h, const char* phase, int64_t* count, double* total_ms) {
  if (!h || !phase || !count || !total_ms) return RUQLP_ERR_INVALID;
  for (int i = 0; i < kProfN; ++i) {
    if (strcmp(phase, kProfNames[i]) == 0) {
      *count = h->prof_count[i];
      *total_ms = h->prof_ms[i];
      return RUQLP_OK;
    }
  }
  return fail(h, RUQLP_ERR_INVALID, "unknown phase '%s'", phase);
}

}  // extern "C"
