// Element-wise steps of the batched path (ruqlp_decompose_batch): the
// Omega intake (Section III-A step 1) and the output writes (Q, L = R_B^T, P),
// one launch over every matrix of the problem table (blockIdx.y = matrix).
#include "internal.h"
#include "philox.cuh"

namespace ruqlp {
namespace {

// X_i (n x dp, FP32) <- Omega_i (n x d, FP64), zero padding columns; for
// tensor-core items also Bt_i = bf16(X_i)^T (dp x ldbt, K-major), the first
// product's B operand.  32-row blocks through a shared tile, so both the
// row-major and the transposed writes are coalesced.
__global__ void __launch_bounds__(256) k_bcast_omega(const BMat* __restrict__ T) {
  __shared__ float t[32][33];
  const BMat& b = T[blockIdx.y];
  __nv_bfloat16* Bt = b.use_tc ? (__nv_bfloat16*)b.Bt : nullptr;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < b.n; r0 += (int64_t)gridDim.x * 32) {
    for (int c0 = 0; c0 < b.dp; c0 += 32) {
      __syncthreads();
      for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int c = c0 + tx;
        float v = 0.f;
        if (r < b.n && c < b.d)
          v = (float)(b.omega != nullptr ? b.omega[r * b.d + c] : omega_entry(b.seed, r, c));
        t[i][tx] = v;
        if (r < b.n && c < b.dp) b.X[r * b.dp + c] = v;
      }
      if (Bt == nullptr) continue;
      __syncthreads();
      for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i;
        const int64_t r = r0 + tx;
        if (c < b.dp && r < b.n) Bt[(int64_t)c * b.ldbt + r] = __float2bfloat16_rn(t[tx][i]);
      }
    }
  }
}

template <typename TO>
__device__ __forceinline__ void copy_rows(const float* __restrict__ src, int64_t rows, int d,
                                          int dp, TO* __restrict__ dst) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int c = threadIdx.x; c < d; c += blockDim.x) dst[r * d + c] = (TO)src[r * dp + c];
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

__global__ void __launch_bounds__(64) k_boutputs(const BMat* __restrict__ T) {
  const BMat& b = T[blockIdx.y];
  if (b.ot == (int)Ty::F64) outputs_body<double>(b);
  else outputs_body<float>(b);
}

}  // namespace

cudaError_t bcast_omega(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  (void)max_elems;
  k_bcast_omega<<<dim3(32, count), dim3(32, 8), 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

cudaError_t boutputs(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  (void)max_elems;
  k_boutputs<<<dim3(128, count), 64, 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
