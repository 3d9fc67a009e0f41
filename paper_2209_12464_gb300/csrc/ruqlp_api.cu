// C ABI of the RU-QLP library: handle, validation, workspace arena and the
// host-side orchestration of Algorithm 1 + Algorithm 2 (Section III) in the
// right-sketch orientation.  Every arithmetic step runs in the kernels of
// this library; the host only validates, carves the arena and launches.
#include <atomic>
#include <mutex>
#include <stdio.h>
#include <vector>
#include <stdarg.h>
#include <string.h>
#include <string>

#include "../../include/ruqlp.h"
#include "internal.h"

using namespace ruqlp;

struct ruqlp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int max_slots = 8;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  DevStatus* status = nullptr;       // device
  DevStatus* status_host = nullptr;  // pinned host
  std::string err;
  // policy knobs (ruqlp_set_option)
  int gram1_exact = 1;  // first CholeskyQR pass: FP64 products (1) or FP32 chunked (0)
  // phase timing with CUDA events on the handle's stream (option "profile")
  bool profile = false;
  struct Span { int cat; cudaEvent_t a, b; };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> pool;
  int64_t prof_count[4] = {0, 0, 0, 0};
  double prof_ms[4] = {0, 0, 0, 0};
};

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

// Profile categories: sketch products A X, transposed products A^T Y, orth(),
// and the whole decomposition.
enum { PROF_AX = 0, PROF_ATX = 1, PROF_ORTH = 2, PROF_STEP = 3 };
const char* kProfNames[4] = {"ax", "atx", "orth", "step"};

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
  ProfScope(ruqlp_ctx* h_, int c) : h(h_), cat(c) {
    if (h->profile) {
      a = ev_get(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~ProfScope() {
    if (h->profile && a) {
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
  size_t X, Y, Z, P, partial, G, R, Rw, total;
};

Layout layout_of(int64_t m, int64_t n, int d, Ty ct) {
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
  L.partial = take((size_t)kMaxSplits * d * d * sizeof(double));
  L.G = take((size_t)d * d * sizeof(double));
  L.R = take((size_t)d * d * sizeof(double));
  L.Rw = take((size_t)d * d * sizeof(double));
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
  return RUQLP_OK;
}

ruqlp_status validate(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                      const ruqlp_outputs* out, int64_t* m, int64_t* n, int* d) {
  if (!A || !prm || !out) return fail(h, RUQLP_ERR_INVALID, "NULL argument");
  if (A->is_csr) return fail(h, RUQLP_ERR_INVALID, "CSR input is not supported by this entry");
  const ruqlp_dense& D = A->dense;
  if (D.m < 1 || D.n < 1) return fail(h, RUQLP_ERR_INVALID, "A must be at least 1 x 1");
  if (D.ld < D.n) return fail(h, RUQLP_ERR_INVALID, "ld (%lld) < n (%lld)", (long long)D.ld,
                              (long long)D.n);
  if (!D.data) return fail(h, RUQLP_ERR_INVALID, "A.data is NULL");
  Ty at, ct;
  if (!ty_of(D.dtype, &at) || !ty_of(prm->compute, &ct))
    return fail(h, RUQLP_ERR_INVALID, "unknown dtype");
  if (at != ct) return fail(h, RUQLP_ERR_INVALID, "compute dtype must equal A's dtype");
  if (prm->k < 1) return fail(h, RUQLP_ERR_INVALID, "k must be >= 1 (got %d)", prm->k);
  if (prm->p < 0) return fail(h, RUQLP_ERR_INVALID, "p must be >= 0 (got %d)", prm->p);
  if (prm->q < 0) return fail(h, RUQLP_ERR_INVALID, "q must be >= 0 (got %d)", prm->q);
  const int64_t dd = (int64_t)prm->k + prm->p;
  if (dd > D.m || dd > D.n)
    return fail(h, RUQLP_ERR_INVALID, "d = k + p = %lld exceeds min(m, n) = %lld",
                (long long)dd, (long long)(D.m < D.n ? D.m : D.n));
  if (dd > 512) return fail(h, RUQLP_ERR_INVALID, "d = %lld exceeds the maximum of 512",
                            (long long)dd);
  if (!prm->omega) return fail(h, RUQLP_ERR_INVALID, "omega is NULL");
  if (!out->Q || !out->L || !out->P) return fail(h, RUQLP_ERR_INVALID, "NULL output buffer");
  if (out->out_dtype != RUQLP_F64 && out->out_dtype != RUQLP_F32)
    return fail(h, RUQLP_ERR_INVALID, "out_dtype must be F64 or F32");
  *m = D.m;
  *n = D.n;
  *d = (int)dd;
  return RUQLP_OK;
}

// Everything the orchestration needs for one decomposition.
struct Job {
  const void* A;
  int64_t lda, m, n;
  int d, dp, q;
  Ty ct, wt;
  const double* omega;  // device, n x d
  void* Qout;
  void* Lout;
  void* Pout;
  Ty ot;
  bool finish_paper;
};

// orth(): Q = Yin R^{-1} by CholeskyQR2, with a third (shifted-CholeskyQR3)
// pass that runs only when a Cholesky of this orth had to shift.
ruqlp_status orth(ruqlp_ctx* h, const Layout& Lo, const Job& J, const void* Yin, void* Qout,
                  int64_t M) {
  ProfScope ps(h, PROF_ORTH);
  char* base = (char*)h->arena;
  double* partial = (double*)(base + Lo.partial);
  double* G = (double*)(base + Lo.G);
  double* R = (double*)(base + Lo.R);
  void* Rw = base + Lo.Rw;
  const int d = J.d, dp = J.dp;
  const Ty wt = J.wt;
  const bool f64 = (wt == Ty::F64);
  const Mul g1 = (f64 || h->gram1_exact) ? Mul::F64 : Mul::F32_ACC64;
  const Mul g2 = f64 ? Mul::F64 : Mul::F32_ACC64;
  // shift = c * u * trace(G) (Fukaya et al. 2020 with ||Y||_2^2 <= trace(G));
  // u is the unit roundoff of the Gram's arithmetic.
  auto shift_rel = [&](Mul g) {
    if (g == Mul::F64) return 11.0 * ((double)M * d + (double)d * (d + 1)) * 1.1102230246251565e-16;
    return 4.0 * 17.0 * 5.960464477539063e-08;
  };
  const int S = tn_splits(d, M, d, kMaxSplits);
  const int32_t* gate = &h->status->shifted;
  CK(status_clear_shift(h->status, h->stream));
  // pass 1
  CK(simt_gemm_tn(wt, wt, Ty::F64, g1, Yin, dp, Yin, dp, G, d, d, M, d, S, partial, nullptr,
                  h->stream));
  CK(chol_upper(G, d, shift_rel(g1), R, Rw, wt, h->status, nullptr, h->stream));
  CK(trsm_right_upper(wt, Yin, dp, Rw, Qout, dp, M, d, nullptr, h->stream));
  // pass 2
  CK(simt_gemm_tn(wt, wt, Ty::F64, g2, Qout, dp, Qout, dp, G, d, d, M, d, S, partial, nullptr,
                  h->stream));
  CK(chol_upper(G, d, shift_rel(g2), R, Rw, wt, h->status, nullptr, h->stream));
  CK(trsm_right_upper(wt, Qout, dp, Rw, Qout, dp, M, d, nullptr, h->stream));
  // pass 3 (only after a shift)
  CK(simt_gemm_tn(wt, wt, Ty::F64, g2, Qout, dp, Qout, dp, G, d, d, M, d, S, partial, gate,
                  h->stream));
  CK(chol_upper(G, d, shift_rel(g2), R, Rw, wt, h->status, gate, h->stream));
  CK(trsm_right_upper(wt, Qout, dp, Rw, Qout, dp, M, d, gate, h->stream));
  return RUQLP_OK;
}

ruqlp_status run_dense(ruqlp_ctx* h, const Job& J) {
  const Layout Lo = layout_of(J.m, J.n, J.d, J.ct);
  ruqlp_status s = ensure_arena(h, Lo.total);
  if (s != RUQLP_OK) return s;
  char* base = (char*)h->arena;
  void* X = base + Lo.X;
  void* Y = base + Lo.Y;
  void* Z = base + Lo.Z;
  void* Pb = base + Lo.P;
  double* partial = (double*)(base + Lo.partial);
  double* G = (double*)(base + Lo.G);
  const int d = J.d, dp = J.dp;
  const Ty ct = J.ct, wt = J.wt;
  const Mul mul = (ct == Ty::F64) ? Mul::F64 : Mul::F32;
  const size_t wes = ty_size(wt);
  cudaStream_t st = h->stream;

  ProfScope pstep(h, PROF_STEP);
  CK(status_reset(h->status, st));
  // a1: Omega (FP64, n x d) -> X (work type, n x dp, zero padding)
  CK(cudaMemsetAsync(X, 0, (size_t)J.n * dp * wes, st));
  CK(copy_cast_2d(Ty::F64, J.omega, d, wt, X, dp, J.n, d, st));
  // a2: Y = A Omega
  {
    ProfScope p(h, PROF_AX);
    CK(simt_gemm_nn(ct, wt, wt, mul, J.A, J.lda, X, dp, Y, dp, J.m, J.n, d, st));
  }
  // a3: Q = orth(Y)
  s = orth(h, Lo, J, Y, Y, J.m);
  if (s != RUQLP_OK) return s;
  // a4: power iteration with orthonormalisation (Algorithm 2)
  for (int it = 0; it < J.q; ++it) {
    {
      ProfScope p(h, PROF_ATX);
      CK(simt_gemm_tn(ct, wt, wt, mul, J.A, J.lda, Y, dp, Z, dp, J.n, J.m, d, 1, nullptr,
                      nullptr, st));
    }
    s = orth(h, Lo, J, Z, Z, J.n);
    if (s != RUQLP_OK) return s;
    {
      ProfScope p(h, PROF_AX);
      CK(simt_gemm_nn(ct, wt, wt, mul, J.A, J.lda, Z, dp, Y, dp, J.m, J.n, d, st));
    }
    s = orth(h, Lo, J, Y, Y, J.m);
    if (s != RUQLP_OK) return s;
  }
  // a5: B^T = A^T Q
  {
    ProfScope p(h, PROF_ATX);
    CK(simt_gemm_tn(ct, wt, wt, mul, J.A, J.lda, Y, dp, Z, dp, J.n, J.m, d, 1, nullptr,
                    nullptr, st));
  }
  // a6: [P, R_B] = qr(B^T): P = orth(B^T), R_B = P^T B^T
  s = orth(h, Lo, J, Z, Pb, J.n);
  if (s != RUQLP_OK) return s;
  const Mul gr = (wt == Ty::F64) ? Mul::F64 : Mul::F32_ACC64;
  CK(simt_gemm_tn(wt, wt, Ty::F64, gr, Pb, dp, Z, dp, G, d, d, J.n, d,
                  tn_splits(d, J.n, d, kMaxSplits), partial, nullptr, st));
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
  if (h->status_host->breakdown)
    return fail(h, RUQLP_ERR_BREAKDOWN, "orth() broke down after its fallbacks");
  return RUQLP_OK;
}

}  // namespace

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
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
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
  if (strcmp(name, "gram1_exact") == 0) {
    h->gram1_exact = value ? 1 : 0;
    return RUQLP_OK;
  }
  if (strcmp(name, "profile") == 0) {
    h->profile = value != 0;
    for (int i = 0; i < 4; ++i) {
      h->prof_count[i] = 0;
      h->prof_ms[i] = 0.0;
    }
    return RUQLP_OK;
  }
  return fail(h, RUQLP_ERR_INVALID, "unknown option '%s'", name);
}

size_t ruqlp_workspace_bytes(int64_t m, int64_t n, int d, ruqlp_dtype compute, int is_csr) {
  Ty ct;
  if (m < 1 || n < 1 || d < 1 || d > 512 || !ty_of(compute, &ct) || is_csr) return 0;
  return layout_of(m, n, d, ct).total;
}

ruqlp_status ruqlp_reserve(ruqlp_handle h, int64_t m, int64_t n, int d, ruqlp_dtype compute,
                           int is_csr) {
  if (!h) return RUQLP_ERR_INVALID;
  const size_t b = ruqlp_workspace_bytes(m, n, d, compute, is_csr);
  if (b == 0) return fail(h, RUQLP_ERR_INVALID, "invalid sizes for ruqlp_reserve");
  return ensure_arena(h, b);
}

ruqlp_status ruqlp_decompose(ruqlp_handle h, const ruqlp_matrix* A, const ruqlp_params* prm,
                             ruqlp_outputs* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  int64_t m, n;
  int d;
  ruqlp_status s = validate(h, A, prm, out, &m, &n, &d);
  if (s != RUQLP_OK) return s;
  CK(cudaSetDevice(h->device));
  Job J{};
  J.A = A->dense.data;
  J.lda = A->dense.ld;
  J.m = m;
  J.n = n;
  J.d = d;
  J.dp = round16(d);
  J.q = prm->q;
  ty_of(prm->compute, &J.ct);
  J.wt = work_ty(J.ct);
  J.omega = prm->omega;
  J.Qout = out->Q;
  J.Lout = out->L;
  J.Pout = out->P;
  ty_of(out->out_dtype, &J.ot);
  J.finish_paper = prm->finish_paper != 0;
  if (J.finish_paper)
    return fail(h, RUQLP_ERR_INVALID, "finish_paper is not available in this build");
  s = run_dense(h, J);
  if (s != RUQLP_OK) return s;
  return finish(h, out);
}

ruqlp_status ruqlp_decompose_host(ruqlp_handle h, const ruqlp_matrix* A,
                                  const ruqlp_params* prm, ruqlp_outputs* out) {
  if (!h) return RUQLP_ERR_INVALID;
  h->err.clear();
  int64_t m, n;
  int d;
  ruqlp_status s = validate(h, A, prm, out, &m, &n, &d);
  if (s != RUQLP_OK) return s;
  CK(cudaSetDevice(h->device));
  Ty at, ot;
  ty_of(A->dense.dtype, &at);
  ty_of(out->out_dtype, &ot);
  const size_t aes = ty_size(at), oes = ty_size(ot);
  // host staging region: A (m x n, packed), Omega, Q, L, P after the workspace
  Layout Lo = layout_of(m, n, d, at);
  size_t off = align_up(Lo.total, 256);
  const size_t oA = off;
  off = align_up(off + (size_t)m * n * aes, 256);
  const size_t oOm = off;
  off = align_up(off + (size_t)n * d * sizeof(double), 256);
  const size_t oQ = off;
  off = align_up(off + (size_t)m * d * oes, 256);
  const size_t oL = off;
  off = align_up(off + (size_t)d * d * oes, 256);
  const size_t oP = off;
  off = align_up(off + (size_t)n * d * oes, 256);
  s = ensure_arena(h, off);
  if (s != RUQLP_OK) return s;
  char* base = (char*)h->arena;
  cudaStream_t st = h->stream;
  CK(cudaMemcpy2DAsync(base + oA, (size_t)n * aes, A->dense.data, (size_t)A->dense.ld * aes,
                       (size_t)n * aes, (size_t)m, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + oOm, prm->omega, (size_t)n * d * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  Job J{};
  J.A = base + oA;
  J.lda = n;
  J.m = m;
  J.n = n;
  J.d = d;
  J.dp = round16(d);
  J.q = prm->q;
  J.ct = at;
  J.wt = work_ty(at);
  J.omega = (const double*)(base + oOm);
  J.Qout = base + oQ;
  J.Lout = base + oL;
  J.Pout = base + oP;
  J.ot = ot;
  J.finish_paper = prm->finish_paper != 0;
  if (J.finish_paper)
    return fail(h, RUQLP_ERR_INVALID, "finish_paper is not available in this build");
  s = run_dense(h, J);
  if (s != RUQLP_OK) return s;
  CK(cudaMemcpyAsync(out->Q, base + oQ, (size_t)m * d * oes, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(out->L, base + oL, (size_t)d * d * oes, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(out->P, base + oP, (size_t)n * d * oes, cudaMemcpyDeviceToHost, st));
  return finish(h, out);
}

const char* ruqlp_last_error(ruqlp_handle h) { return h ? h->err.c_str() : "NULL handle"; }

int64_t ruqlp_launch_count(void) { return launch_count(); }

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
  for (int i = 0; i < 4; ++i) {
    if (strcmp(phase, kProfNames[i]) == 0) {
      *count = h->prof_count[i];
      *total_ms = h->prof_ms[i];
      return RUQLP_OK;
    }
  }
  return fail(h, RUQLP_ERR_INVALID, "unknown phase '%s'", phase);
}

}  // extern "C"
