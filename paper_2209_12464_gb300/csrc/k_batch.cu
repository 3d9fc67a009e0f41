// Element-wise steps of the batched path (ruqlp_decompose_batch): the
// Omega intake (Section III-A step 1) and the output writes (Q, L = R_B^T, P),
// one launch over every matrix of the problem table (blockIdx.y = matrix).
#include "internal.h"
#include "philox.cuh"

namespace ruqlp {
namespace {

// X_i (n x dp, FP32) <- Omega_i (n x d, FP64), zero padding columns; for
// tensor-core items also Bt_i = bf16(X_i)^T (dp x ldbt, K-major), the first
// product's B operand.  64-row blocks through a shared tile, so both the
// row-major and the transposed writes are coalesced; a thread issues its
// eight loads of a 64 x 32 chunk before any store.
constexpr int OB = 64;  // rows per block of the Omega intake
__global__ void __launch_bounds__(256) k_bcast_omega(const BMat* __restrict__ T) {
  __shared__ float t[OB][33];
  const BMat& b = T[blockIdx.y];
  __nv_bfloat16* Bt = b.use_tc ? (__nv_bfloat16*)b.Bt : nullptr;
  const double* __restrict__ om = b.omega;
  float* __restrict__ X = b.X;
  const int64_t n = b.n;
  const int d = b.d, dp = b.dp;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int64_t r0 = (int64_t)blockIdx.x * OB; r0 < n; r0 += (int64_t)gridDim.x * OB) {
    for (int c0 = 0; c0 < dp; c0 += 32) {
      const int c = c0 + tx;
      float v[OB / 8];
#pragma unroll
      for (int q = 0; q < OB / 8; ++q) {
        const int64_t r = r0 + ty + 8 * q;
        v[q] = 0.f;
        if (r < n && c < d) v[q] = (float)(om != nullptr ? om[r * d + c] : omega_entry(b.seed, r, c));
      }
      __syncthreads();  // the previous chunk's transposed reads are done
#pragma unroll
      for (int q = 0; q < OB / 8; ++q) {
        const int64_t r = r0 + ty + 8 * q;
        t[ty + 8 * q][tx] = v[q];
        if (r < n && c < dp) X[r * dp + c] = v[q];
      }
      if (Bt == nullptr) continue;
      __syncthreads();
      // column c0 + i of the chunk: lane tx writes rows r0 + 2 tx, r0 + 2 tx + 1
      for (int i = ty; i < 32; i += 8) {
        const int cc = c0 + i;
        const int64_t r = r0 + 2 * tx;
        if (cc >= dp || r >= n) continue;
        __nv_bfloat16* p = Bt + (int64_t)cc * b.ldbt + r;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(t[2 * tx][i]);
        if (r + 1 < n && (((uintptr_t)p & 3) == 0)) {
          __nv_bfloat162 h2;
          h2.x = h0;
          h2.y = __float2bfloat16_rn(t[2 * tx + 1][i]);
          *reinterpret_cast<__nv_bfloat162*>(p) = h2;
        } else {
          p[0] = h0;
          if (r + 1 < n) p[1] = __float2bfloat16_rn(t[2 * tx + 1][i]);
        }
      }
    }
  }
}

// dst (rows x d, leading dimension d) <- src (rows x dp): one warp per group
// of 8 rows, a 32-column chunk at a time, the group's loads issued before its
// stores.
template <typename TO>
__device__ __forceinline__ void copy_rows(const float* __restrict__ src, int64_t rows, int d,
                                          int dp, TO* __restrict__ dst) {
  constexpr int RW = 8;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = w * RW; r0 < rows; r0 += nw * RW) {
    for (int c = lane; c < d; c += 32) {
      float v[RW];
#pragma unroll
      for (int u = 0; u < RW; ++u) v[u] = (r0 + u < rows) ? src[(r0 + u) * dp + c] : 0.f;
#pragma unroll
      for (int u = 0; u < RW; ++u)
        if (r0 + u < rows) dst[(r0 + u) * d + c] = (TO)v[u];
    }
  }
}

// Q_i = Y_i (m x d), P_i = P buffer (n x d), L_i = R_B^T (d x d, R_B in G_i),
// all row-major with leading dimension d in the output type.
template <typename TO>
__device__ __forceinline__ void outputs_body(const BMat& b) {
  copy_rows<TO>(b.Y, b.m, b.d, b.dp, (TO*)b.Qout);
  copy_rows<TO>(b.P, b.n, b.d, b.dp, (TO*)b.Pout);
  TO* L = (TO*)b.Lout;
  for (int64_t i = blockIdx.x; i < b.d; i += gridDim.x)
    for (int j = threadIdx.x; j < b.d; j += blockDim.x)
      L[i * b.d + j] = (j <= i) ? (TO)b.G[(int64_t)j * b.d + i] : (TO)0;
}

__global__ void __launch_bounds__(256) k_boutputs(const BMat* __restrict__ T) {
  const BMat& b = T[blockIdx.y];
  if (b.ot == (int)Ty::F64) outputs_body<double>(b);
  else outputs_body<float>(b);
}

}  // namespace

cudaError_t bcast_omega(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  (void)max_elems;
  k_bcast_omega<<<dim3(16, count), dim3(32, 8), 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

cudaError_t boutputs(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  (void)max_elems;
  k_boutputs<<<dim3(16, count), 256, 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
