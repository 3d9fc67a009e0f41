// Element-wise steps of the batched path (ruqlp_decompose_batch): the
// Omega intake (Section III-A step 1) and the output writes (Q, L = R_B^T, P),
// one launch over every matrix of the problem table (blockIdx.y = matrix).
#include "internal.h"

namespace ruqlp {
namespace {

// X_i (n x dp, FP32) <- Omega_i (n x d, FP64), zero padding columns.
__global__ void k_bcast_omega(const BMat* __restrict__ T) {
  const BMat& b = T[blockIdx.y];
  const int64_t tot = b.n * b.dp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / b.dp;
    const int c = (int)(e % b.dp);
    b.X[e] = (c < b.d) ? (float)b.omega[r * b.d + c] : 0.f;
  }
}

template <typename TO>
__device__ __forceinline__ void put(void* base, int64_t idx, double v) {
  reinterpret_cast<TO*>(base)[idx] = (TO)v;
}

// Q_i = Y_i (m x d), P_i = P buffer (n x d), L_i = R_B^T (d x d, R_B in G_i),
// all row-major with leading dimension d in the output type.
__global__ void k_boutputs(const BMat* __restrict__ T) {
  const BMat& b = T[blockIdx.y];
  const int d = b.d;
  const int64_t nq = b.m * d, np = b.n * d, nl = (int64_t)d * d;
  const int64_t tot = nq + np + nl;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v;
    void* dst;
    int64_t idx;
    if (e < nq) {
      v = b.Y[(e / d) * b.dp + e % d];
      dst = b.Qout;
      idx = e;
    } else if (e < nq + np) {
      idx = e - nq;
      v = b.P[(idx / d) * b.dp + idx % d];
      dst = b.Pout;
    } else {
      idx = e - nq - np;
      const int i = (int)(idx / d), j = (int)(idx % d);
      v = (j <= i) ? b.G[(int64_t)j * d + i] : 0.0;
      dst = b.Lout;
    }
    if (b.ot == (int)Ty::F64) put<double>(dst, idx, v);
    else put<float>(dst, idx, v);
  }
}

}  // namespace

cudaError_t bcast_omega(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int gx = ceil_div(max_elems, 256);
  if (gx > 4096) gx = 4096;
  k_bcast_omega<<<dim3(gx, count), 256, 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

cudaError_t boutputs(const BMat* T, int count, int64_t max_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int gx = ceil_div(max_elems, 256);
  if (gx > 4096) gx = 4096;
  k_boutputs<<<dim3(gx, count), 256, 0, st>>>(T);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
