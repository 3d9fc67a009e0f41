// FP32 pieces of the shifted CholeskyQR3 orth() (Section II-A orth();
// Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020) for d <= 288:
//
//  * k_chol_inv: one CTA factors the d x d Gram G (+ shift I) = R^T R and
//    inverts R, both blocked in 32 x 32 tiles held in shared memory (upper
//    block triangle, padded to a multiple of 32 with the identity).  Each
//    32 x 32 diagonal factorisation / inversion is done by one warp with
//    __syncwarp only; the panel solves and trailing updates spread over all
//    warps, so the whole factorisation takes about 6 block barriers per tile
//    row instead of 3 per column.
//  * k_mul_upper: Q = Y R^{-1} as a product with the explicit upper-triangular
//    inverse (rows of Y staged in shared memory, so Q may overwrite Y).
#include <math.h>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace ruqlp {
namespace {

constexpr int TB = 32;        // tile edge
constexpr int TP = TB + 1;    // padded row pitch (bank-conflict free column walks)
constexpr int MAXNB = 9;      // d <= 288
constexpr int NTH = 256;   // 8 warps: up to 255 registers for the per-lane tile columns

__device__ __forceinline__ int bidx(int I, int J, int nb) { return I * nb - (I * (I - 1)) / 2 + (J - I); }

__global__ void __launch_bounds__(NTH)
k_chol_inv(const double* __restrict__ G, int d, double shift_rel, int force_shift,
           float* __restrict__ Rinv, DevStatus* __restrict__ status,
           const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float sm[];
  __shared__ double s_shift;
  __shared__ int s_bad, s_rankdef;
  __shared__ float S[TB][TP];  // inverse of the current diagonal tile
  const int nb = (d + TB - 1) / TB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NTH / 32;
  auto tile = [&](int I, int J) { return sm + (size_t)bidx(I, J, nb) * TB * TP; };

  // shift = shift_rel * trace(G), reduced by warp 0
  if (warp == 0) {
    double t = 0.0;
    for (int i = lane; i < d; i += 32) t += G[(size_t)i * d + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      double sh = shift_rel * t;
      if (!(sh > 0.0)) sh = 1e-30;
      s_shift = sh;
      s_rankdef = 0;
    }
  }
  int attempt = force_shift ? 1 : 0;
  for (; attempt < 2; ++attempt) {
    __syncthreads();
    const double add = attempt ? s_shift : 0.0;
    // load the upper block triangle (padding: identity)
    const int ntiles = nb * (nb + 1) / 2;
    for (int e = tid; e < ntiles * TB * TB; e += NTH) {
      const int t = e / (TB * TB), rc = e % (TB * TB), r = rc / TB, c = rc % TB;
      int I = 0, tt = t;
      while (tt >= nb - I) { tt -= nb - I; ++I; }
      const int J = I + tt;
      const int i = I * TB + r, j = J * TB + c;
      double v;
      if (i < d && j < d) v = G[(size_t)i * d + j] + (i == j ? add : 0.0);
      else v = (i == j) ? 1.0 : 0.0;
      tile(I, J)[r * TP + c] = (float)v;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int K = 0; K < nb; ++K) {
      // (a) factor the diagonal tile: warp 0, lane c owns column c
      if (warp == 0) {
        float* B = tile(K, K);
        for (int k = 0; k < TB; ++k) {
          __syncwarp();
          float piv = B[k * TP + k];
          if (!(piv > 0.f) || !isfinite(piv)) {
            if (attempt == 0) {
              if (lane == 0) s_bad = 1;
              break;  // uniform: every lane read the same pivot
            }
            piv = (float)s_shift;
            if (lane == 0) s_rankdef = 1;
          }
          const float rkk = sqrtf(piv);
          float bk = B[k * TP + lane];
          __syncwarp();
          if (lane == k) B[k * TP + k] = rkk;
          else if (lane > k) B[k * TP + lane] = bk / rkk;
          __syncwarp();
          if (lane > k) {
            const float rkl = B[k * TP + lane];
            for (int i = k + 1; i <= lane; ++i) B[i * TP + lane] -= B[k * TP + i] * rkl;
          }
        }
      }
      __syncthreads();
      if (s_bad) break;
      // (b) panel: B_KJ <- R_KK^{-T} B_KJ for J > K (forward substitution)
      for (int J = K + 1 + warp; J < nb; J += nw) {
        const float* R = tile(K, K);
        float* B = tile(K, J);
        float x[TB];
#pragma unroll
        for (int r = 0; r < TB; ++r) {
          float acc = B[r * TP + lane];
#pragma unroll
          for (int k = 0; k < r; ++k) acc -= R[k * TP + r] * x[k];
          x[r] = acc / R[r * TP + r];
        }
#pragma unroll
        for (int r = 0; r < TB; ++r) B[r * TP + lane] = x[r];
      }
      __syncthreads();
      // (c) trailing update: B_IJ -= B_KI^T B_KJ for K < I <= J
      const int rem = nb - K - 1;
      const int nupd = rem * (rem + 1) / 2;
      for (int u = warp; u < nupd; u += nw) {
        int I = 0, tt = u;
        while (tt >= rem - I) { tt -= rem - I; ++I; }
        I += K + 1;
        const int J = I + tt;
        const float* BI = tile(K, I);
        const float* BJ = tile(K, J);
        float* C = tile(I, J);
        float bj[TB];
#pragma unroll
        for (int k = 0; k < TB; ++k) bj[k] = BJ[k * TP + lane];
#pragma unroll 4
        for (int r = 0; r < TB; ++r) {
          float acc = C[r * TP + lane];
#pragma unroll
          for (int k = 0; k < TB; ++k) acc -= BI[k * TP + r] * bj[k];
          C[r * TP + lane] = acc;
        }
      }
      __syncthreads();
    }
    if (!s_bad) break;
  }
  __syncthreads();

  // inverse X = R^{-1}, tile rows from the bottom, in place of R
  for (int I = nb - 1; I >= 0; --I) {
    if (warp == 0) {  // S = R_II^{-1} by back substitution, lane c owns column c
      const float* R = tile(I, I);
      float x[TB];
#pragma unroll
      for (int r = TB - 1; r >= 0; --r) {
        float acc = (r == lane) ? 1.f : 0.f;
#pragma unroll
        for (int k = r + 1; k < TB; ++k) acc -= R[r * TP + k] * x[k];
        x[r] = acc / R[r * TP + r];
      }
#pragma unroll
      for (int r = 0; r < TB; ++r) S[r][lane] = x[r];
    }
    __syncthreads();
    // X_IJ = -S (sum_{K=I+1..J} R_IK X_KJ) for J > I (rows K > I already hold X)
    float out[TB];
    const int J = I + 1 + warp;
    const bool mine = J < nb;  // nb - 1 - I <= 8 = warps: one tile per warp
    if (mine) {
      float t[TB];
#pragma unroll
      for (int r = 0; r < TB; ++r) t[r] = 0.f;
      for (int K = I + 1; K <= J; ++K) {
        const float* RK = tile(I, K);
        const float* XK = tile(K, J);
        float xk[TB];
#pragma unroll
        for (int k = 0; k < TB; ++k) xk[k] = XK[k * TP + lane];
#pragma unroll
        for (int r = 0; r < TB; ++r) {
          float acc = t[r];
#pragma unroll
          for (int k = 0; k < TB; ++k) acc += RK[r * TP + k] * xk[k];
          t[r] = acc;
        }
      }
#pragma unroll
      for (int r = 0; r < TB; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < TB; ++k) acc -= S[r][k] * t[k];
        out[r] = acc;
      }
    }
    __syncthreads();
    if (mine) {
      float* X = tile(I, J);
#pragma unroll
      for (int r = 0; r < TB; ++r) X[r * TP + lane] = out[r];
    }
    if (warp == nw - 1) {
      float* X = tile(I, I);
#pragma unroll
      for (int r = 0; r < TB; ++r) X[r * TP + lane] = S[r][lane];
    }
    __syncthreads();
  }
  // write R^{-1} (row-major, ld d, zero lower triangle)
  for (int e = tid; e < d * d; e += NTH) {
    const int i = e / d, j = e % d;
    float v = 0.f;
    if (j >= i) v = tile(i / TB, j / TB)[(i % TB) * TP + (j % TB)];
    Rinv[e] = v;
  }
  if (tid == 0) {
    if (attempt > 0) {
      status->shifted = 1;
      if (!force_shift) status->flags |= RUQLP_FLAG_SHIFTED;
    }
    if (s_rankdef) status->flags |= RUQLP_FLAG_RANKDEF;
  }
}

// X = Y U for upper-triangular U (d x d, ld d): 64-row blocks of Y are staged
// in shared memory first, so X may alias Y.
constexpr int MR = 64;
__global__ void __launch_bounds__(256)
k_mul_upper(const float* __restrict__ Y, int64_t ldy, const float* __restrict__ U, float* X,
            int64_t ldx, int64_t M, int d) {
  extern __shared__ float ys[];  // MR x (d + 1)
  __shared__ float us[32][64];
  const int pitch = d + 1;
  const int64_t r0 = (int64_t)blockIdx.x * MR;
  const int nr = (int)min((int64_t)MR, M - r0);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  for (int e = t; e < MR * d; e += 256) {
    const int r = e / d, c = e % d;
    ys[r * pitch + c] = (r < nr) ? Y[(r0 + r) * ldy + c] : 0.f;
  }
  __syncthreads();
  for (int c0 = 0; c0 < d; c0 += 64) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int kmax = min(d, c0 + 64);  // U[k][c] = 0 for k > c
    for (int k0 = 0; k0 < kmax; k0 += 32) {
      for (int e = t; e < 32 * 64; e += 256) {
        const int kk = e / 64, cc = e % 64;
        const int k = k0 + kk, c = c0 + cc;
        us[kk][cc] = (k < d && c < d) ? U[(size_t)k * d + c] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const int k = k0 + kk;
        if (k >= d) break;
        float a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = ys[(ty * 4 + i) * pitch + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = us[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty * 4 + i;
      if (r >= nr) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + tx * 4 + j;
        if (c < d) X[(r0 + r) * ldx + c] = acc[i][j];
      }
    }
  }
}

}  // namespace

size_t chol_inv_f32_smem(int d) {
  const int nb = (d + TB - 1) / TB;
  return (size_t)nb * (nb + 1) / 2 * TB * TP * sizeof(float);
}

bool chol_inv_f32_supported(int d) {
  return d >= 1 && (d + TB - 1) / TB <= MAXNB && chol_inv_f32_smem(d) <= 200 * 1024;
}

cudaError_t chol_inv_f32(const double* G, int d, double shift_rel, bool force_shift, float* Rinv,
                         DevStatus* status, const int32_t* gate, cudaStream_t st) {
  if (!chol_inv_f32_supported(d)) return cudaErrorInvalidValue;
  const size_t sm = chol_inv_f32_smem(d);
  cudaError_t e =
      cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_chol_inv<<<1, NTH, sm, st>>>(G, d, shift_rel, force_shift ? 1 : 0, Rinv, status, gate);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mul_upper_f32(const float* Y, int64_t ldy, const float* U, float* X, int64_t ldx,
                          int64_t M, int d, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const size_t sm = (size_t)MR * (d + 1) * sizeof(float);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e =
      cudaFuncSetAttribute(k_mul_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_mul_upper<<<ceil_div(M, MR), 256, sm, st>>>(Y, ldy, U, X, ldx, M, d);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
