// Sparse (CSR) products of RU-QLP (Section III-D: with s nonzeros the method
// costs O(sd); the same passes over A as the dense path).
//
//   Y[rows x d] = A X    with A in CSR (rowptr, colidx, values)
//   Z[cols x d] = A^T Y  with the CSR of A^T (the CSC of A), built once per
//                        decomposition and kept in the workspace.
//
// SpMM: one warp per output row; lane l owns columns 4l..4l+3 (then +128, ...)
// of the d columns; for each nonzero the warp gathers the matching row of the
// skinny operand (L2-resident) with 128-bit loads.  Every output entry is a
// sum over the row's nonzeros in storage order, so the result is
// deterministic.  The transpose is made deterministic too: nonzeros are
// scattered to their column (atomic cursors), then each column's entries are
// sorted by row index, the unique order of the CSC.
#include <algorithm>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace ruqlp {
namespace {

template <typename TV> __device__ __forceinline__ float val_f32(TV v);
template <> __device__ __forceinline__ float val_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float val_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

// flag bit 1: rowptr not a valid prefix (rowptr[0] != 0, decreasing, or
// rowptr[m] != nnz); bit 2: column index out of range or not strictly
// increasing inside a row.
__global__ void k_csr_validate(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                               int64_t m, int64_t n, int64_t nnz, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > m) return;
  if (i == 0 && rowptr[0] != 0) atomicOr(flag, 1);
  if (i == m) {
    if ((int64_t)rowptr[m] != nnz) atomicOr(flag, 1);
    return;
  }
  const int32_t a = rowptr[i], b = rowptr[i + 1];
  if (b < a || a < 0 || (int64_t)b > nnz) { atomicOr(flag, 1); return; }
  int32_t prev = -1;
  for (int32_t e = a; e < b; ++e) {
    const int32_t c = colidx[e];
    if (c <= prev || (int64_t)c >= n) { atomicOr(flag, 2); return; }
    prev = c;
  }
}

__global__ void k_col_count(const int32_t* __restrict__ colidx, int64_t nnz, int32_t* counts) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[colidx[e]], 1);
}

// exclusive scan of counts[0..n) into ptr[0..n], one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ counts, int64_t n,
                                               int32_t* __restrict__ ptr, int32_t* __restrict__ cursor) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + 1023) / 1024;
  const int64_t a = t * per, b = min(n, a + per);
  int32_t s = 0;
  for (int64_t i = a; i < b; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan of the parts
    const int32_t v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = (t == 0) ? 0 : part[t - 1];
  for (int64_t i = a; i < b; ++i) {
    ptr[i] = run;
    cursor[i] = run;
    run += counts[i];
  }
  if (t == 1023) ptr[n] = part[1023];
}

template <typename TV>
__global__ void k_csc_scatter(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                              const TV* __restrict__ vals, int64_t m, int32_t* cursor,
                              int32_t* __restrict__ rowidx, TV* __restrict__ cvals) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const int32_t a = rowptr[warp], b = rowptr[warp + 1];
  for (int32_t e = a + lane; e < b; e += 32) {
    const int32_t pos = atomicAdd(&cursor[colidx[e]], 1);
    rowidx[pos] = (int32_t)warp;
    cvals[pos] = vals[e];
  }
}

// Sort each column's (row, value) entries by row: one warp per column,
// bitonic sort of up to 1024 entries in shared memory.  flag bit 4: a
// column holds more than 1024 nonzeros.
constexpr int SORT_MAX = 1024;
template <typename TV>
__global__ void __launch_bounds__(128)
k_csc_sort(const int32_t* __restrict__ colptr, int64_t n, int32_t* __restrict__ rowidx,
           TV* __restrict__ cvals, int* flag) {
  __shared__ int32_t keys[4][SORT_MAX];
  __shared__ TV sv[4][SORT_MAX];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * 4 + w;
  if (c >= n) return;
  const int32_t a = colptr[c], b = colptr[c + 1];
  const int len = b - a;
  if (len <= 1) return;
  if (len > SORT_MAX) {
    if (lane == 0) atomicOr(flag, 4);
    return;
  }
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  int32_t* K = keys[w];
  TV* V = sv[w];
  for (int i = lane; i < p2; i += 32) {
    K[i] = (i < len) ? rowidx[a + i] : 0x7fffffff;
    V[i] = cvals[a + ((i < len) ? i : 0)];  // padding keys sort last, values unused
  }
  __syncwarp();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < p2; i += 32) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const int32_t ki = K[i], kj = K[j];
          if ((ki > kj) == up) {
            K[i] = kj;
            K[j] = ki;
            const TV t = V[i];
            V[i] = V[j];
            V[j] = t;
          }
        }
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < len; i += 32) {
    rowidx[a + i] = K[i];
    cvals[a + i] = V[i];
  }
}

// Y[r][0..d) = sum_e val[e] X[col[e]][0..d) for r in [0, rows); X, Y FP32.
template <typename TV>
__global__ void __launch_bounds__(256)
k_spmm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const TV* __restrict__ vals,
       int64_t rows, const float* __restrict__ X, int64_t ldx, int d, float* __restrict__ Y,
       int64_t ldy) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const int32_t a = ptr[r], b = ptr[r + 1];
  const int nchunk = (d + 127) / 128;  // 128 columns per warp sweep (4 per lane)
  for (int ch = 0; ch < nchunk; ++ch) {
    const int c = ch * 128 + lane * 4;
    const bool on = c < d;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int32_t e = a;
    for (; e + 4 <= b; e += 4) {  // four independent gathers in flight
      int32_t col[4];
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[u] = idx[e + u];
        v[u] = val_f32(vals[e + u]);
      }
      if (on) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const float4*>(X + (int64_t)col[u] * ldx + c);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc.x = fmaf(v[u], x[u].x, acc.x);
          acc.y = fmaf(v[u], x[u].y, acc.y);
          acc.z = fmaf(v[u], x[u].z, acc.z);
          acc.w = fmaf(v[u], x[u].w, acc.w);
        }
      }
    }
    for (; e < b; ++e) {
      const int32_t col = idx[e];
      const float v = val_f32(vals[e]);
      if (on) {
        const float4 x = *reinterpret_cast<const float4*>(X + (int64_t)col * ldx + c);
        acc.x = fmaf(v, x.x, acc.x);
        acc.y = fmaf(v, x.y, acc.y);
        acc.z = fmaf(v, x.z, acc.z);
        acc.w = fmaf(v, x.w, acc.w);
      }
    }
    if (on) *reinterpret_cast<float4*>(Y + r * ldy + c) = acc;
  }
}

// out[r][c] += t[r][c], r < rows, c < d (FP32).
__global__ void k_add_rows(float* __restrict__ out, int64_t ldo, const float* __restrict__ t,
                           int64_t ldt, int64_t rows, int d) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int c = threadIdx.x; c < d; c += blockDim.x) out[r * ldo + c] += t[r * ldt + c];
}

}  // namespace

cudaError_t add_rows_f32(float* out, int64_t ldo, const float* t, int64_t ldt, int64_t rows, int d,
                         cudaStream_t st) {
  if (rows <= 0 || d <= 0) return cudaSuccess;
  k_add_rows<<<(int)std::min<int64_t>(rows, 152 * 16), 128, 0, st>>>(out, ldo, t, ldt, rows, d);
  count_launch();
  return cudaGetLastError();
}

cudaError_t csr_validate(const int32_t* rowptr, const int32_t* colidx, int64_t m, int64_t n,
                         int64_t nnz, int* flag, cudaStream_t st) {
  k_csr_validate<<<ceil_div(m + 1, 256), 256, 0, st>>>(rowptr, colidx, m, n, nnz, flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t csr_transpose(Ty tv, const int32_t* rowptr, const int32_t* colidx, const void* vals,
                          int64_t m, int64_t n, int64_t nnz, int32_t* colptr, int32_t* rowidx,
                          void* cvals, int32_t* scratch, int* flag, cudaStream_t st) {
  int32_t* counts = scratch;        // n
  int32_t* cursor = scratch + n;    // n
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)n * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (nnz > 0) {
    k_col_count<<<1216, 256, 0, st>>>(colidx, nnz, counts);
    count_launch();
  }
  k_scan<<<1, 1024, 0, st>>>(counts, n, colptr, cursor);
  count_launch();
  const int gw = ceil_div(m * 32, 256);
  const int gs = ceil_div(n, 4);
  if (tv == Ty::F32) {
    k_csc_scatter<float><<<gw, 256, 0, st>>>(rowptr, colidx, (const float*)vals, m, cursor, rowidx,
                                             (float*)cvals);
    count_launch();
    k_csc_sort<float><<<gs, 128, 0, st>>>(colptr, n, rowidx, (float*)cvals, flag);
    count_launch();
  } else if (tv == Ty::BF16) {
    k_csc_scatter<__nv_bfloat16><<<gw, 256, 0, st>>>(rowptr, colidx, (const __nv_bfloat16*)vals, m,
                                                     cursor, rowidx, (__nv_bfloat16*)cvals);
    count_launch();
    k_csc_sort<__nv_bfloat16><<<gs, 128, 0, st>>>(colptr, n, rowidx, (__nv_bfloat16*)cvals, flag);
    count_launch();
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t spmm_csr(Ty tv, const int32_t* ptr, const int32_t* idx, const void* vals, int64_t rows,
                     const float* X, int64_t ldx, int d, float* Y, int64_t ldy, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if ((ldx % 4) || (ldy % 4) || ((uintptr_t)X & 15) || ((uintptr_t)Y & 15))
    return cudaErrorInvalidValue;
  const int grid = ceil_div(rows * 32, 256);
  if (tv == Ty::F32)
    k_spmm<float><<<grid, 256, 0, st>>>(ptr, idx, (const float*)vals, rows, X, ldx, d, Y, ldy);
  else if (tv == Ty::BF16)
    k_spmm<__nv_bfloat16><<<grid, 256, 0, st>>>(ptr, idx, (const __nv_bfloat16*)vals, rows, X, ldx,
                                                d, Y, ldy);
  else
    return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
