// SIMT (CUDA-core) products for RU-QLP: the FP64 and FP32 paths of the
// sketch / power-iteration products (Section III-D: A X and A^T Y, O(mnd)),
// and the tall-skinny Gram and R products of orth() (O(md^2)).
//
// One CTA of 256 threads computes a 64 x 64 output tile; each thread owns a
// 4 x 4 sub-tile.  K is walked in 16-wide slabs staged in shared memory.
// Out-of-range rows/columns are zero-filled on load and skipped on store, so
// any M, K, N works (ragged tails included).
#include <type_traits>

#include "internal.h"

namespace ruqlp {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <Mul MODE> struct MulT;
template <> struct MulT<Mul::F64> { using mul = double; using acc = double; };
template <> struct MulT<Mul::F32> { using mul = float; using acc = float; };
template <> struct MulT<Mul::F32_ACC64> { using mul = float; using acc = double; };

template <typename T> __device__ __forceinline__ T zero() { return T(0); }

// TRANS_A = false: A is M x K (row-major, lda): C = A B.
// TRANS_A = true:  A is K x M (row-major, lda): C = A^T B.
// blockIdx.z selects a K slab [kz0, kz1); with PARTIAL the FP64 tile sums go to
// C + z*M*ldc (a [splits][M][ldc] FP64 buffer).
// ROUND_B: 1 = the B operand is rounded to BF16 as it is staged; 2 = to the
// sum of its two BF16 parts, h + bf16(b - h) (exact in FP32).
template <bool TRANS_A, typename TA, typename TB, typename TC, Mul MODE, bool PARTIAL,
          int ROUND_B = 0>
__device__ __forceinline__ void gemm_tile(const TA* __restrict__ A, int64_t lda,
                                          const TB* __restrict__ B, int64_t ldb,
                                          TC* __restrict__ C, int64_t ldc, int64_t M, int64_t K,
                                          int64_t N, int64_t kslab, int bx, int by, int bz) {
  using TM = typename MulT<MODE>::mul;
  using TAcc = typename MulT<MODE>::acc;
  __shared__ TM As[BK][BM + 4];
  __shared__ TM Bs[BK][BN + 4];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int64_t m0 = (int64_t)bx * BM;
  const int64_t n0 = (int64_t)by * BN;
  const int64_t kz0 = (int64_t)bz * kslab;
  const int64_t kz1 = min(K, kz0 + kslab);

  TAcc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<TAcc>();

  for (int64_t k0 = kz0; k0 < kz1; k0 += BK) {
    // stage A (BM x BK) as As[k][m]
#pragma unroll
    for (int e = t; e < BM * BK; e += NT) {
      int r, c;
      if (TRANS_A) { r = e % BM; c = e / BM; }   // consecutive threads walk m (contiguous)
      else         { r = e / BK; c = e % BK; }   // consecutive threads walk k (contiguous)
      const int64_t gm = m0 + r, gk = k0 + c;
      TM v = zero<TM>();
      if (gm < M && gk < kz1) {
        v = Cvt<TM>::from(TRANS_A ? A[gk * lda + gm] : A[gm * lda + gk]);
      }
      As[c][r] = v;
    }
    // stage B (BK x BN) as Bs[k][n]
#pragma unroll
    for (int e = t; e < BK * BN; e += NT) {
      const int r = e / BN, c = e % BN;
      const int64_t gk = k0 + r, gn = n0 + c;
      TM v = zero<TM>();
      if (gk < kz1 && gn < N) {
        v = Cvt<TM>::from(B[gk * ldb + gn]);
        if constexpr (ROUND_B == 1) v = __bfloat162float(__float2bfloat16_rn(v));
        if constexpr (ROUND_B == 2) {
          const float h = __bfloat162float(__float2bfloat16_rn(v));
          v = h + __bfloat162float(__float2bfloat16_rn(v - h));
        }
      }
      Bs[r][c] = v;
    }
    __syncthreads();
    TM part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = zero<TM>();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TM a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += (TAcc)part[i][j];
    __syncthreads();
  }

  TC* Cz = PARTIAL ? C + (int64_t)bz * M * ldc : C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx * 4 + j;
      if (gn < N) Cz[gm * ldc + gn] = Cvt<TC>::from(acc[i][j]);
    }
  }
}

template <bool TRANS_A, typename TA, typename TB, typename TC, Mul MODE, bool PARTIAL>
__global__ void __launch_bounds__(NT)
k_gemm(const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B, int64_t ldb,
       TC* __restrict__ C, int64_t ldc, int64_t M, int64_t K, int64_t N, int64_t kslab,
       const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  gemm_tile<TRANS_A, TA, TB, TC, MODE, PARTIAL>(A, lda, B, ldb, C, ldc, M, K, N, kslab,
                                                blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched products over a problem table: tile t of the whole launch maps to
// matrix i = (prefix[i] <= t < prefix[i+1]) and a 64 x 64 output tile of it.
//   TRANS_A = false: buf[dst] (m x d) = A buf[src] (n x d)
//   TRANS_A = true:  buf[dst] (n x d) = A^T buf[src] (m x d)
template <bool TRANS_A, typename TA, typename TB, int SPLIT2 = 0>
__global__ void __launch_bounds__(NT)
k_bgemm(const BMat* __restrict__ T, const int* __restrict__ prefix, int count, int src, int dst) {
  const int t = blockIdx.x;
  int lo = 0, hi = count;  // largest i with prefix[i] <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const BMat& b = T[prefix[count + 1 + lo]];  // the launch order's item lo
  const int local = t - prefix[lo];
  const int ntn = (b.d + BN - 1) / BN;
  const int64_t Mout = TRANS_A ? b.n : b.m, K = TRANS_A ? b.m : b.n;
  // with BF16 A the skinny operand is rounded to BF16 (or to its two-part
  // BF16 sum) as it is staged, the product the single-matrix BF16 path computes
  constexpr int RB = std::is_same<TA, __nv_bfloat16>::value ? (SPLIT2 ? 2 : 1) : 0;
  gemm_tile<TRANS_A, TA, TB, float, Mul::F32, false, RB>(
      (const TA*)b.A, b.lda, (const TB*)bbuf(b, src), b.dp, bbuf(b, dst), b.dp, Mout, K, b.d,
      ((K + BK - 1) / BK) * BK, local / ntn, local % ntn, 0);
}

// C[i][j] = sum_z P[z][i][j] in z order (deterministic), cast to TC.
template <typename TC>
__global__ void k_reduce_partials(const double* __restrict__ P, int splits, int64_t M, int64_t N,
                                  TC* __restrict__ C, int64_t ldc,
                                  const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx / N, j = idx % N;
  double s = 0.0;  // split order, eight independent loads in flight
  int z = 0;
  for (; z + 8 <= splits; z += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = P[(int64_t)(z + u) * M * N + idx];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; z < splits; ++z) s += P[(int64_t)z * M * N + idx];
  C[i * ldc + j] = Cvt<TC>::from(s);
}

template <bool TRANS_A, typename TA, typename TB, typename TC, Mul MODE>
cudaError_t launch(const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc,
                   int64_t M, int64_t K, int64_t N, int splits, double* partial,
                   const int32_t* gate, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits < 1) splits = 1;
  int64_t kslab = ((K + splits - 1) / splits + BK - 1) / BK * BK;
  if (kslab < BK) kslab = BK;
  splits = (int)((K + kslab - 1) / kslab);
  if (splits < 1) splits = 1;
  dim3 grid(ceil_div(M, BM), ceil_div(N, BN), splits);
  if (splits == 1) {
    k_gemm<TRANS_A, TA, TB, TC, MODE, false><<<grid, NT, 0, st>>>(
        (const TA*)A, lda, (const TB*)B, ldb, (TC*)C, ldc, M, K, N, kslab, gate);
    count_launch();
    return cudaGetLastError();
  }
  k_gemm<TRANS_A, TA, TB, double, MODE, true><<<grid, NT, 0, st>>>(
      (const TA*)A, lda, (const TB*)B, ldb, partial, N, M, K, N, kslab, gate);
    count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = M * N;
  k_reduce_partials<TC><<<ceil_div(tot, 256), 256, 0, st>>>(partial, splits, M, N, (TC*)C, ldc, gate);
    count_launch();
  return cudaGetLastError();
}

}  // namespace

int tn_splits(int64_t M, int64_t K, int64_t N, int max_splits) {
  const int64_t tiles = (int64_t)ceil_div(M, BM) * ceil_div(N, BN);
  int64_t s = (2 * 152 + tiles - 1) / tiles;        // about two CTAs per SM
  const int64_t kmax = (K + 4 * BK - 1) / (4 * BK);  // at least 64 rows per slab
  if (s > kmax) s = kmax;
  if (s > max_splits) s = max_splits;
  if (s < 1) s = 1;
  return (int)s;
}

#define RUQLP_DISPATCH(TRANS, TA_, TB_, TC_, MODE_, CTA, CTB, CTC)                         \
  if (ta == TA_ && tb == TB_ && tc == TC_ && mul == MODE_)                                 \
    return launch<TRANS, CTA, CTB, CTC, MODE_>(A, lda, B, ldb, C, ldc, M, K, N, splits,    \
                                               partial, gate, st);

cudaError_t simt_gemm_nn(Ty ta, Ty tb, Ty tc, Mul mul, const void* A, int64_t lda,
                         const void* B, int64_t ldb, void* C, int64_t ldc, int64_t M,
                         int64_t K, int64_t N, cudaStream_t st) {
  const int splits = 1;
  double* partial = nullptr;
  const int32_t* gate = nullptr;
  RUQLP_DISPATCH(false, Ty::F64, Ty::F64, Ty::F64, Mul::F64, double, double, double)
  RUQLP_DISPATCH(false, Ty::F32, Ty::F32, Ty::F32, Mul::F32, float, float, float)
  RUQLP_DISPATCH(false, Ty::BF16, Ty::F32, Ty::F32, Mul::F32, __nv_bfloat16, float, float)
  RUQLP_DISPATCH(false, Ty::BF16, Ty::BF16, Ty::F32, Mul::F32, __nv_bfloat16, __nv_bfloat16, float)
  RUQLP_DISPATCH(false, Ty::F32, Ty::F32, Ty::F32, Mul::F32_ACC64, float, float, float)
  return cudaErrorInvalidValue;
}

int bgemm_tiles(int64_t rows, int d) { return ceil_div(rows, BM) * ceil_div(d, BN); }

cudaError_t bgemm(bool trans, Ty ta, Ty tb, const BMat* T, const int* prefix, int total, int count,
                  int src, int dst, cudaStream_t st, bool split2) {
  if (total <= 0) return cudaSuccess;
  if (tb == Ty::F32) {
    if (ta == Ty::F32) {
      if (trans) k_bgemm<true, float, float><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
      else k_bgemm<false, float, float><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
    } else if (ta == Ty::BF16) {
      if (trans && split2)
        k_bgemm<true, __nv_bfloat16, float, 1><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
      else if (trans) k_bgemm<true, __nv_bfloat16, float><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
      else if (split2)
        k_bgemm<false, __nv_bfloat16, float, 1><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
      else k_bgemm<false, __nv_bfloat16, float><<<total, NT, 0, st>>>(T, prefix, count, src, dst);
    } else {
      return cudaErrorInvalidValue;
    }
  } else {
    return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t simt_gemm_tn(Ty ta, Ty tb, Ty tc, Mul mul, const void* A, int64_t lda,
                         const void* B, int64_t ldb, void* C, int64_t ldc, int64_t M,
                         int64_t K, int64_t N, int splits, double* partial,
                         const int32_t* gate, cudaStream_t st) {
  if (splits > 1 && partial == nullptr) return cudaErrorInvalidValue;
  RUQLP_DISPATCH(true, Ty::F64, Ty::F64, Ty::F64, Mul::F64, double, double, double)
  RUQLP_DISPATCH(true, Ty::F32, Ty::F32, Ty::F32, Mul::F32, float, float, float)
  RUQLP_DISPATCH(true, Ty::BF16, Ty::F32, Ty::F32, Mul::F32, __nv_bfloat16, float, float)
  RUQLP_DISPATCH(true, Ty::BF16, Ty::BF16, Ty::F32, Mul::F32, __nv_bfloat16, __nv_bfloat16, float)
  RUQLP_DISPATCH(true, Ty::F32, Ty::F32, Ty::F64, Mul::F32_ACC64, float, float, double)
  RUQLP_DISPATCH(true, Ty::F32, Ty::F32, Ty::F64, Mul::F64, float, float, double)
  return cudaErrorInvalidValue;
}

}  // namespace ruqlp
