// Kernels of orth() / qr() for tall-skinny matrices (Section II-A: orth() and
// unpivoted qr(); used by Algorithm 1 steps 3-4 and Algorithm 2): the d x d
// FP64 Cholesky of CholeskyQR2 with a shifted-Cholesky fallback (Fukaya,
// Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020), the
// triangular solve Q = Y R^{-1}, and small layout helpers.
#include <math.h>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace ruqlp {
namespace {

constexpr int CHOL_THREADS = 1024;
constexpr size_t CHOL_SMEM_MAX = 200 * 1024;

// Index of (i, j), i <= j, in the working upper triangle: packed rows in
// shared memory, or a full row-major d x d array in global memory.
template <bool PACKED>
__device__ __forceinline__ int64_t uidx(int i, int j, int d) {
  return PACKED ? (int64_t)i * d - ((int64_t)i * (i - 1)) / 2 + (j - i) : (int64_t)i * d + j;
}

template <typename TW> __device__ __forceinline__ TW from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return (float)v; }

// Right-looking Cholesky G = R^T R (upper R), one CTA, arithmetic in TF.
// Attempt 0 factors G (skipped with force_shift); if a pivot is not positive
// it restarts on G + shift I (attempt 1), where a pivot that is still not
// positive is replaced by `shift` (rank deficiency, flagged).  check = 1 (or
// 2 while status->shifted is still 0, i.e. no later pass will run): the last
// pass of a CholeskyQR, whose Gram should be close to I -- a pivot outside
// [1/2, 2] flags RUQLP_FLAG_RANKDEF.
template <bool PACKED, typename TF, typename TW>
__global__ void __launch_bounds__(CHOL_THREADS)
k_chol(const double* __restrict__ G, int d, double shift_rel, int force_shift,
       double* __restrict__ R, TW* __restrict__ Rw, DevStatus* __restrict__ status,
       const int32_t* __restrict__ gate, int check) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ double smem_d[];
  __shared__ int s_bad;
  __shared__ int s_rankdef;
  __shared__ int s_far;
  __shared__ double s_shift;
  const bool check_on = check == 1 || (check == 2 && status->shifted == 0);
  TF* W = PACKED ? reinterpret_cast<TF*>(smem_d) : reinterpret_cast<TF*>(R);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;

  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < d; ++i) tr += G[(int64_t)i * d + i];
    double sh = shift_rel * tr;
    if (!(sh > 0.0)) sh = 1e-300;
    s_shift = sh;
    s_rankdef = 0;
    s_far = 0;
  }
  int attempt = force_shift ? 1 : 0;
  for (; attempt < 2; ++attempt) {
    __syncthreads();
    const double add = attempt ? s_shift : 0.0;
    for (int i = warp; i < d; i += nwarps)
      for (int j = i + lane; j < d; j += 32)
        W[uidx<PACKED>(i, j, d)] = (TF)(G[(int64_t)i * d + j] + (i == j ? add : 0.0));
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < d; ++k) {
      if (tid == 0) {
        TF piv = W[uidx<PACKED>(k, k, d)];
        if (check_on && attempt == 0 && !(piv >= TF(0.5) && piv <= TF(2))) s_far = 1;
        if (!(piv > TF(0)) || !isfinite((double)piv)) {
          if (attempt == 0) {
            s_bad = 1;
          } else {
            piv = (TF)s_shift;
            s_rankdef = 1;
          }
        }
        W[uidx<PACKED>(k, k, d)] = sqrt(piv);
      }
      __syncthreads();
      if (s_bad) break;
      const TF rkk = W[uidx<PACKED>(k, k, d)];
      for (int j = k + 1 + tid; j < d; j += blockDim.x) W[uidx<PACKED>(k, j, d)] /= rkk;
      __syncthreads();
      for (int i = k + 1 + warp; i < d; i += nwarps) {
        const TF rki = W[uidx<PACKED>(k, i, d)];
        for (int j = i + lane; j < d; j += 32)
          W[uidx<PACKED>(i, j, d)] -= rki * W[uidx<PACKED>(k, j, d)];
      }
      __syncthreads();
    }
    if (!s_bad) break;
  }
  __syncthreads();
  // R (full FP64, zero lower part) and its working-type copy; in global mode
  // with TF = double the upper part of R already holds the factor
  if (!PACKED && sizeof(TF) != sizeof(double)) {
    // float factor stored in R's memory: widen in place from the end
    if (tid == 0) {
      for (int64_t e = (int64_t)d * d - 1; e >= 0; --e) {
        const int i = (int)(e / d), j = (int)(e % d);
        const double v = (j >= i) ? (double)W[e] : 0.0;
        R[e] = v;
      }
    }
    __syncthreads();
    for (int i = warp; i < d; i += nwarps)
      for (int j = lane; j < d; j += 32) Rw[(int64_t)i * d + j] = (TW)R[(int64_t)i * d + j];
  } else {
    for (int i = warp; i < d; i += nwarps) {
      for (int j = lane; j < d; j += 32) {
        const double v = (j >= i) ? (double)W[uidx<PACKED>(i, j, d)] : 0.0;
        if (PACKED || j < i) R[(int64_t)i * d + j] = v;
        Rw[(int64_t)i * d + j] = (TW)v;
      }
    }
  }
  if (tid == 0) {
    if (attempt > 0) {
      status->shifted = 1;
      if (!force_shift) status->flags |= RUQLP_FLAG_SHIFTED;
    }
    if (s_rankdef || s_far) status->flags |= RUQLP_FLAG_RANKDEF;
  }
}

// Rows of X = Y R^{-1}: each warp owns whole rows, kept in shared memory; for
// every column j, x_j = y_j / R_jj and y_l -= x_j R_jl (l > j).
template <typename T>
__global__ void __launch_bounds__(256)
k_trsm(const T* __restrict__ Y, int64_t ldy, const T* __restrict__ R, T* __restrict__ X,
       int64_t ldx, int64_t M, int d, int rows, const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int nr = (int)min((int64_t)rows, M - r0);
  for (int e = tid; e < nr * d; e += blockDim.x) {
    const int r = e / d, c = e % d;
    S[(int64_t)r * d + c] = Y[(r0 + r) * ldy + c];
  }
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    const T inv = T(1) / R[(int64_t)j * d + j];
    for (int r = warp; r < nr; r += 8) {
      T* srow = S + (int64_t)r * d;
      const T xj = srow[j] * inv;
      __syncwarp();  // every lane has read y_j before lane 0 overwrites it
      for (int l = j + 1 + lane; l < d; l += 32) srow[l] -= xj * R[(int64_t)j * d + l];
      if (lane == 0) srow[j] = xj;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < nr * d; e += blockDim.x) {
    const int r = e / d, c = e % d;
    X[(r0 + r) * ldx + c] = S[(int64_t)r * d + c];
  }
}

template <typename TS, typename TD>
__global__ void k_copy_cast(const TS* __restrict__ src, int64_t lds, TD* __restrict__ dst,
                            int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx / cols, j = idx % cols;
  dst[i * ldd + j] = Cvt<TD>::from(src[i * lds + j]);
}

// dst = h + bf16(v - h), h = bf16(v): v rounded to the sum of its two BF16
// parts (exact in FP32), the skinny operand of a two-part BF16 product.
template <typename TS>
__global__ void k_round2_bf16(const TS* __restrict__ src, int64_t lds, float* __restrict__ dst,
                              int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx / cols, j = idx % cols;
  const float v = (float)src[i * lds + j];
  const float h = __bfloat162float(__float2bfloat16_rn(v));
  dst[i * ldd + j] = h + __bfloat162float(__float2bfloat16_rn(v - h));
}

template <typename TL>
__global__ void k_write_L(const double* __restrict__ R, int d, TL* __restrict__ L, bool upper,
                          int ldl) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d * d) return;
  const int i = idx / d, j = idx % d;
  double v;
  if (upper) v = (j >= i) ? R[(int64_t)i * d + j] : 0.0;
  else       v = (j <= i) ? R[(int64_t)j * d + i] : 0.0;
  L[(int64_t)i * ldl + j] = Cvt<TL>::from(v);
}

__global__ void k_status(DevStatus* s, int full) {
  if (full) { s->flags = 0; s->breakdown = 0; s->timeout = 0; s->invalid = 0; }
  s->shifted = 0;
}

}  // namespace

cudaError_t chol_upper(const double* G, int d, double shift_rel, double* R, void* Rw, Ty tw,
                       DevStatus* status, const int32_t* gate, cudaStream_t st, Ty tf,
                       bool force_shift, int check) {
  const size_t esz = (tf == Ty::F64) ? sizeof(double) : sizeof(float);
  const size_t packed = (size_t)d * (d + 1) / 2 * esz;
  const bool use_smem = packed <= CHOL_SMEM_MAX;
  const size_t sm = use_smem ? packed : 0;
  const int fs = force_shift ? 1 : 0;
  cudaError_t e = cudaSuccess;
#define RUQLP_CHOL(PK, TF, TW)                                                              \
  {                                                                                         \
    if (PK) e = cudaFuncSetAttribute(k_chol<PK, TF, TW>,                                    \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                     (int)CHOL_SMEM_MAX);                                   \
    if (e != cudaSuccess) return e;                                                         \
    k_chol<PK, TF, TW><<<1, CHOL_THREADS, sm, st>>>(G, d, shift_rel, fs, R, (TW*)Rw, status, \
                                                    gate, check);                           \
    count_launch();                                                                         \
    return cudaGetLastError();                                                              \
  }
  if (tf == Ty::F64 && tw == Ty::F64) {
    if (use_smem) RUQLP_CHOL(true, double, double) else RUQLP_CHOL(false, double, double)
  }
  if (tf == Ty::F64 && tw == Ty::F32) {
    if (use_smem) RUQLP_CHOL(true, double, float) else RUQLP_CHOL(false, double, float)
  }
  if (tf == Ty::F32 && tw == Ty::F32) {
    if (use_smem) RUQLP_CHOL(true, float, float) else RUQLP_CHOL(false, float, float)
  }
#undef RUQLP_CHOL
  return cudaErrorInvalidValue;
}

cudaError_t trsm_right_upper(Ty ty, const void* Y, int64_t ldy, const void* R, void* X,
                             int64_t ldx, int64_t M, int d, const int32_t* gate,
                             cudaStream_t st) {
  if (M <= 0 || d <= 0) return cudaSuccess;
  const size_t es = ty_size(ty);
  int rows = (int)((200 * 1024) / ((size_t)d * es));
  if (rows > 64) rows = 64;
  rows = rows / 8 * 8;
  if (rows < 8) return cudaErrorInvalidValue;
  const size_t sm = (size_t)rows * d * es;
  const int grid = ceil_div(M, rows);
  cudaError_t e;
  if (ty == Ty::F64) {
    e = cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_trsm<double><<<grid, 256, sm, st>>>((const double*)Y, ldy, (const double*)R, (double*)X,
                                           ldx, M, d, rows, gate);
    count_launch();
    return cudaGetLastError();
  }
  if (ty == Ty::F32) {
    e = cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_trsm<float><<<grid, 256, sm, st>>>((const float*)Y, ldy, (const float*)R, (float*)X, ldx,
                                         M, d, rows, gate);
    count_launch();
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

cudaError_t round2_bf16_2d(Ty ts, const void* src, int64_t lds, float* dst, int64_t ldd,
                          int64_t rows, int64_t cols, cudaStream_t st) {
  const int64_t tot = rows * cols;
  if (tot <= 0) return cudaSuccess;
  const int grid = ceil_div(tot, 256);
  if (ts == Ty::F32)
    k_round2_bf16<float><<<grid, 256, 0, st>>>((const float*)src, lds, dst, ldd, rows, cols);
  else if (ts == Ty::F64)
    k_round2_bf16<double><<<grid, 256, 0, st>>>((const double*)src, lds, dst, ldd, rows, cols);
  else
    return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

cudaError_t copy_cast_2d(Ty ts, const void* src, int64_t lds, Ty td, void* dst, int64_t ldd,
                         int64_t rows, int64_t cols, cudaStream_t st) {
  const int64_t tot = rows * cols;
  if (tot <= 0) return cudaSuccess;
  const int grid = ceil_div(tot, 256);
#define RUQLP_CC(TS_, TD_, CS, CD)                                                           \
  if (ts == TS_ && td == TD_) {                                                              \
    k_copy_cast<CS, CD><<<grid, 256, 0, st>>>((const CS*)src, lds, (CD*)dst, ldd, rows, cols); \
    count_launch();                                                                          \
    return cudaGetLastError();                                                               \
  }
  RUQLP_CC(Ty::F64, Ty::F64, double, double)
  RUQLP_CC(Ty::F64, Ty::F32, double, float)
  RUQLP_CC(Ty::F64, Ty::BF16, double, __nv_bfloat16)
  RUQLP_CC(Ty::F32, Ty::F32, float, float)
  RUQLP_CC(Ty::F32, Ty::F64, float, double)
  RUQLP_CC(Ty::F32, Ty::BF16, float, __nv_bfloat16)
#undef RUQLP_CC
  return cudaErrorInvalidValue;
}

cudaError_t write_L(const double* R, int d, Ty tl, void* L, bool upper, cudaStream_t st,
                    int ldl) {
  const int grid = ceil_div((int64_t)d * d, 256);
  if (ldl <= 0) ldl = d;
  if (tl == Ty::F64) {
    k_write_L<double><<<grid, 256, 0, st>>>(R, d, (double*)L, upper, ldl);
    count_launch();
    return cudaGetLastError();
  }
  if (tl == Ty::F32) {
    k_write_L<float><<<grid, 256, 0, st>>>(R, d, (float*)L, upper, ldl);
    count_launch();
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

cudaError_t status_reset(DevStatus* s, cudaStream_t st) {
  k_status<<<1, 1, 0, st>>>(s, 1);
    count_launch();
  return cudaGetLastError();
}

cudaError_t status_clear_shift(DevStatus* s, cudaStream_t st) {
  k_status<<<1, 1, 0, st>>>(s, 0);
    count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
