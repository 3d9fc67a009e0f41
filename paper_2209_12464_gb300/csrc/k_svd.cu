// SVD-like finish of RU-QLP (Section III-C, Remark 1): with L = U S V^T the
// d x d middle factor, A ~= Q L P^T = (Q U) S (P V)^T.
//
// One CTA factors L by one-sided Jacobi (Hestenes): the columns of W = L are
// rotated in pairs until every pair is orthogonal to tol relative to the
// product of their norms, V accumulating the rotations; then S = column
// norms, U = W S^{-1}, sorted by decreasing S.  A sweep visits every pair
// once in d' - 1 rounds of d'/2 disjoint pairs (d' = d rounded up to even,
// a round-robin tournament), each pair handled by one warp (column dot
// products reduced with a fixed shuffle tree, so the result is
// deterministic).  W and V are kept column-major in global memory (L2).
#include "internal.h"

namespace ruqlp {
namespace {

constexpr int SVD_THREADS = 512;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// W (column-major, ldw = d): on entry L, on exit U; V (column-major): on exit
// V; s: singular values, descending.  scratch: 2 d ints + d T.
template <typename T>
__global__ void __launch_bounds__(SVD_THREADS)
k_svd_jacobi(T* __restrict__ W, T* __restrict__ V, T* __restrict__ s, int d, T tol, int max_sweeps,
             int* __restrict__ order, T* __restrict__ tmpcol, int* __restrict__ sweeps_out) {
  __shared__ int s_rot;
  __shared__ int perm[520], perm2[520];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = SVD_THREADS / 32;
  const int dd = (d + 1) & ~1;  // players (d' = d + 1 with a dummy when d is odd)
  for (int e = tid; e < d * d; e += SVD_THREADS) V[e] = ((e / d) == (e % d)) ? T(1) : T(0);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int k = tid; k < dd; k += SVD_THREADS) perm[k] = k;
    __syncthreads();
    for (int round = 0; round < dd - 1; ++round) {
      for (int pr = warp; pr < dd / 2; pr += nw) {
        int p = perm[pr], q = perm[dd - 1 - pr];
        if (p >= d || q >= d) continue;  // the dummy player sits out
        if (p > q) { const int t = p; p = q; q = t; }
        T* wp = W + (int64_t)p * d;
        T* wq = W + (int64_t)q * d;
        T a = 0, b = 0, g = 0;
        for (int i = lane; i < d; i += 32) {
          const T x = wp[i], y = wq[i];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (g == T(0) || fabs(g) <= tol * sqrt(a * b)) continue;
        const T zeta = (b - a) / (T(2) * g);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
        for (int i = lane; i < d; i += 32) {
          const T x = wp[i], y = wq[i];
          wp[i] = c * x - sn * y;
          wq[i] = sn * x + c * y;
        }
        T* vp = V + (int64_t)p * d;
        T* vq = V + (int64_t)q * d;
        for (int i = lane; i < d; i += 32) {
          const T x = vp[i], y = vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
      // next pairing: keep perm[0], rotate perm[1..dd-1] by one place
      for (int k = tid; k < dd; k += SVD_THREADS) perm2[k] = perm[k];
      __syncthreads();
      for (int k = 1 + tid; k < dd; k += SVD_THREADS) perm[k] = perm2[k == 1 ? dd - 1 : k - 1];
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  // singular values, descending (rank by comparison; ties by index)
  for (int j = warp; j < d; j += nw) {
    T a = 0;
    for (int i = lane; i < d; i += 32) a += W[(int64_t)j * d + i] * W[(int64_t)j * d + i];
    a = warp_sum(a);
    if (lane == 0) tmpcol[j] = sqrt(a);
  }
  __syncthreads();
  for (int j = tid; j < d; j += SVD_THREADS) {
    const T sj = tmpcol[j];
    int r = 0;
    for (int k = 0; k < d; ++k) {
      const T sk = tmpcol[k];
      r += (sk > sj || (sk == sj && k < j)) ? 1 : 0;
    }
    order[r] = j;
    s[r] = sj;
  }
  __syncthreads();
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// Uo (d x d row-major, ld ldo) = W[:, order] / s, Vo likewise from V.
template <typename T>
__global__ void k_svd_gather(const T* __restrict__ W, const T* __restrict__ V,
                             const T* __restrict__ s, const int* __restrict__ order, int d,
                             T* __restrict__ Uo, T* __restrict__ Vo, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), r = (int)(e % d);  // row i, sorted column r
  const int j = order[r];
  const T sj = s[r];
  Uo[(int64_t)i * ldo + r] = sj > T(0) ? W[(int64_t)j * d + i] / sj : T(0);
  Vo[(int64_t)i * ldo + r] = V[(int64_t)j * d + i];
}

template <typename TS, typename TO>
__global__ void k_write_diag(const TS* __restrict__ s, int d, TO* __restrict__ L) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), j = (int)(e % d);
  L[e] = (i == j) ? (TO)s[i] : (TO)0;
}

}  // namespace

cudaError_t write_diag(Ty t, const void* s, int d, Ty to, void* L, cudaStream_t st) {
  const int g = ceil_div((int64_t)d * d, 256);
  if (t == Ty::F64 && to == Ty::F64) k_write_diag<double, double><<<g, 256, 0, st>>>((const double*)s, d, (double*)L);
  else if (t == Ty::F64 && to == Ty::F32) k_write_diag<double, float><<<g, 256, 0, st>>>((const double*)s, d, (float*)L);
  else if (t == Ty::F32 && to == Ty::F64) k_write_diag<float, double><<<g, 256, 0, st>>>((const float*)s, d, (double*)L);
  else if (t == Ty::F32 && to == Ty::F32) k_write_diag<float, float><<<g, 256, 0, st>>>((const float*)s, d, (float*)L);
  else return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

cudaError_t svd_jacobi(Ty t, void* W, void* V, void* s, int d, int max_sweeps, int* order,
                       void* tmpcol, int* sweeps, void* Uo, void* Vo, int64_t ldo,
                       cudaStream_t st) {
  if (d < 1 || d > 512) return cudaErrorInvalidValue;
  const int gb = ceil_div((int64_t)d * d, 256);
  if (t == Ty::F64) {
    k_svd_jacobi<double><<<1, SVD_THREADS, 0, st>>>((double*)W, (double*)V, (double*)s, d,
                                                    (double)d * 2.220446049250313e-16, max_sweeps,
                                                    order, (double*)tmpcol, sweeps);
    count_launch();
    k_svd_gather<double><<<gb, 256, 0, st>>>((const double*)W, (const double*)V,
                                             (const double*)s, order, d, (double*)Uo,
                                             (double*)Vo, ldo);
  } else if (t == Ty::F32) {
    k_svd_jacobi<float><<<1, SVD_THREADS, 0, st>>>((float*)W, (float*)V, (float*)s, d,
                                                   (float)d * 1.1920929e-07f, max_sweeps, order,
                                                   (float*)tmpcol, sweeps);
    count_launch();
    k_svd_gather<float><<<gb, 256, 0, st>>>((const float*)W, (const float*)V, (const float*)s,
                                            order, d, (float*)Uo, (float*)Vo, ldo);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
