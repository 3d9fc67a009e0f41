// FP32 pieces of the shifted CholeskyQR3 orth() (Section II-A orth();
// Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020) for d <= 256:
//
//  * k_chol_tiles: one CTA factors the d x d Gram G (+ shift I) = R^T R,
//    blocked in 32 x 32 tiles held in shared memory (upper block triangle,
//    padded to a multiple of 32 with the identity).  Each diagonal tile is
//    factored and inverted by one warp in registers (shuffles); the panel
//    solves (products with the tile inverse) and trailing updates are 32 x 32
//    tile products spread over all warps with 128-bit broadcast loads, so the
//    factorisation needs three block barriers per tile row, not per column.
//  * k_trsm_tiles: Q = Y R^{-1} by blocked forward substitution with those
//    tiles (rows of Y staged in shared memory, so Q may overwrite Y).
#include <math.h>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace ruqlp {
size_t chol_tiles_smem(int d);
namespace {

constexpr int TB = 32;        // tile edge
constexpr int TP = 36;        // row pitch: 16-byte aligned rows for 128-bit loads
constexpr int MAXNB = 8;      // d <= 256
constexpr int NTH = 512;      // 16 warps; up to 128 registers for per-lane tile columns
constexpr size_t TILE_FLOATS = (size_t)TB * TP;

__device__ __forceinline__ int bidx(int I, int J, int nb) { return I * nb - (I * (I - 1)) / 2 + (J - I); }

// acc[r] (r = r0..r0+7) += sum_k A[k][r] * bcol[k] for one lane's column
// bcol (in registers).  A is a 32 x 32 tile in shared memory (pitch TP); each
// 128-bit load of A serves 4 rows, and the 8 rows are independent chains.
__device__ __forceinline__ void tile_tn8(const float* __restrict__ A, int r0, const float (&bcol)[TB],
                                         float (&acc)[8]) {
#pragma unroll
  for (int k = 0; k < TB; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * TP + r0);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * TP + r0 + 4);
    acc[0] = fmaf(a0.x, bcol[k], acc[0]);
    acc[1] = fmaf(a0.y, bcol[k], acc[1]);
    acc[2] = fmaf(a0.z, bcol[k], acc[2]);
    acc[3] = fmaf(a0.w, bcol[k], acc[3]);
    acc[4] = fmaf(a1.x, bcol[k], acc[4]);
    acc[5] = fmaf(a1.y, bcol[k], acc[5]);
    acc[6] = fmaf(a1.z, bcol[k], acc[6]);
    acc[7] = fmaf(a1.w, bcol[k], acc[7]);
  }
}

__device__ __forceinline__ void load_col(const float* __restrict__ T, int lane, float (&c)[TB]) {
#pragma unroll
  for (int k = 0; k < TB; ++k) c[k] = T[k * TP + lane];
}

// One warp factors the 32 x 32 tile B = R^T R in registers (lane c owns
// column c) and writes R (upper) back and S = R^{-1} (upper) to Sout.
// Step k broadcasts row k of the partially reduced tile through the shared
// row buffer rb (one store per lane, 128-bit broadcast loads of the whole
// row issued together), so every lane forms r_ki itself; there are no
// shuffles and no branches in the loop.  Reciprocal square roots and
// reciprocals replace IEEE sqrt/divide (the factor only has to be consistent
// with the solve that uses it).  A non-positive pivot is replaced by
// bad_fill; the return value (same in every lane) reports whether that
// happened.
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&r)[TB]) {
#pragma unroll
  for (int q = 0; q < TB / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(p)[q];
    r[4 * q] = v.x;
    r[4 * q + 1] = v.y;
    r[4 * q + 2] = v.z;
    r[4 * q + 3] = v.w;
  }
}

__device__ bool factor_tile(float* __restrict__ B, float* __restrict__ Sout, float* __restrict__ dinv,
                            float* __restrict__ rb, int lane, float bad_fill) {
  float col[TB];
  load_col(B, lane, col);
  float myinv = 0.f;  // 1 / R[lane][lane]
  bool bad = false;
#pragma unroll
  for (int k = 0; k < TB; ++k) {
    __syncwarp();
    rb[lane] = col[k];  // row k of the current tile, lane c holds B[k][c]
    __syncwarp();
    float row[TB];
    load_row(rb, row);
    float piv = row[k];
    const bool nonpos = !(piv > 0.f) || !(piv < 3.0e38f);
    bad = bad || nonpos;
    piv = nonpos ? bad_fill : piv;
    const float rinv = rsqrtf(piv);
    const float rkc = (lane == k) ? piv * rinv : col[k] * rinv;  // r_kc for c >= k
    myinv = (lane == k) ? rinv : myinv;
    col[k] = (lane >= k) ? rkc : col[k];
#pragma unroll
    for (int i = k + 1; i < TB; ++i) {
      const float rki = row[i] * rinv;
      const float upd = fmaf(-rki, rkc, col[i]);
      col[i] = (lane >= i) ? upd : col[i];
    }
  }
  // R row-major into B; R transposed (column c of R as row c) into Sout,
  // which the inverse below reads before overwriting it
#pragma unroll
  for (int r = 0; r < TB; ++r) {
    const float v = (r <= lane) ? col[r] : 0.f;
    B[r * TP + lane] = v;
    Sout[lane * TP + r] = v;
  }
  dinv[lane] = myinv;
  __syncwarp();
  // S = R^{-1}, right-looking: lane c solves R x = e_c from the bottom;
  // acc[j] -= R[j][r] x[r] for j < r are independent multiply-adds
  float dv[TB];
  load_row(dinv, dv);
  float acc[TB];
#pragma unroll
  for (int r = 0; r < TB; ++r) acc[r] = (r == lane) ? 1.f : 0.f;
#pragma unroll
  for (int r = TB - 1; r >= 0; --r) {
    const float xr = acc[r] * dv[r];
    acc[r] = xr;
    float rc[TB];  // column r of R (rows j < r are used)
    load_row(Sout + r * TP, rc);
#pragma unroll
    for (int j = 0; j < r; ++j) acc[j] = fmaf(-rc[j], xr, acc[j]);
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < TB; ++r) Sout[r * TP + lane] = acc[r];
  return !bad;
}

// Blocked Cholesky G (+ shift I) = R^T R, d <= 256, one CTA.  Writes the
// upper tiles R_IJ (I <= J) and the diagonal-tile inverses R_KK^{-1}, FP32,
// 32 x 32 row-major each, to `tiles`: first the nb (nb+1)/2 R tiles in
// row-of-tiles order, then the nb inverse tiles.
__device__ __forceinline__ void chol_body(const double* __restrict__ G, int d, double shift_rel,
                                          int force_shift, float* __restrict__ tiles,
                                          DevStatus* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double s_shift;
  __shared__ int s_bad, s_rankdef;
  __shared__ __align__(16) float s_dinv[TB];
  __shared__ __align__(16) float s_row[TB];
  const int nb = (d + TB - 1) / TB;
  const int ntiles = nb * (nb + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NTH / 32;
  auto tile = [&](int I, int J) { return sm + (size_t)bidx(I, J, nb) * TILE_FLOATS; };
  auto dinv_s = [&](int K) { return sm + (size_t)(ntiles + K) * TILE_FLOATS; };  // shared

  if (warp == 0) {  // shift = shift_rel * trace(G)
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
    // upper block triangle of G + shift I (identity padding), eight
    // independent loads in flight per thread
    for (int e0 = tid; e0 < ntiles * TB * TB; e0 += 8 * NTH) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * NTH;
        x[u] = 0.0;
        if (e < ntiles * TB * TB) {
          const int t = e >> 10, r = (e >> 5) & 31, c = e & 31;
          int I = 0, tt = t;
          while (tt >= nb - I) { tt -= nb - I; ++I; }
          const int i = I * TB + r, j = (I + tt) * TB + c;
          if (i < d && j < d) x[u] = G[(size_t)i * d + j];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * NTH;
        if (e < ntiles * TB * TB) {
          const int t = e >> 10, r = (e >> 5) & 31, c = e & 31;
          int I = 0, tt = t;
          while (tt >= nb - I) { tt -= nb - I; ++I; }
          const int i = I * TB + r, j = (I + tt) * TB + c;
          double v = x[u];
          if (i == j) v = (i < d) ? v + add : 1.0;
          sm[(size_t)t * TILE_FLOATS + r * TP + c] = (float)v;
        }
      }
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int K = 0; K < nb; ++K) {
      if (warp == 0) {  // (a) diagonal tile, its inverse (kept in shared memory)
        const bool ok = factor_tile(tile(K, K), dinv_s(K), s_dinv, s_row, lane,
                                    attempt == 0 ? 1.f : (float)s_shift);
        if (lane == 0 && !ok) {
          if (attempt == 0) s_bad = 1;  // retry on G + shift I
          else s_rankdef = 1;           // pivots replaced by the shift
        }
      }
      __syncthreads();
      if (s_bad) break;
      // (b) panel B_KJ <- R_KK^{-T} B_KJ: one warp per tile; each lane reads
      // and writes only its own column
      for (int J = K + 1 + warp; J < nb; J += nw) {
        float* B = tile(K, J);
        float bc[TB];
        load_col(B, lane, bc);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          tile_tn8(dinv_s(K), q * 8, bc, acc);
#pragma unroll
          for (int i = 0; i < 8; ++i) B[(q * 8 + i) * TP + lane] = acc[i];
        }
      }
      __syncthreads();
      // (c) trailing update B_IJ -= B_KI^T B_KJ, items (I, J, 8-row slice)
      const int rem = nb - K - 1;
      const int nupd = rem * (rem + 1) / 2 * 4;
      for (int u = warp; u < nupd; u += nw) {
        int I = 0, tt = u / 4;
        while (tt >= rem - I) { tt -= rem - I; ++I; }
        I += K + 1;
        const int J = I + tt, r0 = (u % 4) * 8;
        float bc[TB];
        load_col(tile(K, J), lane, bc);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        tile_tn8(tile(K, I), r0, bc, acc);
        float* C = tile(I, J);
#pragma unroll
        for (int i = 0; i < 8; ++i) C[(r0 + i) * TP + lane] -= acc[i];
      }
      __syncthreads();
    }
    if (!s_bad) break;
  }
  __syncthreads();
  // write R tiles and the diagonal-tile inverses (32 x 32 row-major each)
  for (int t = warp; t < ntiles + nb; t += nw) {
    const float* src = sm + (size_t)t * TILE_FLOATS;
    float* dst = tiles + (size_t)t * TB * TB;
#pragma unroll 8
    for (int r = 0; r < TB; ++r) dst[r * TB + lane] = src[r * TP + lane];
  }
  if (tid == 0) {
    if (attempt > 0) {
      status->shifted = 1;
      if (!force_shift) status->flags |= RUQLP_FLAG_SHIFTED;
    }
    if (s_rankdef) status->flags |= RUQLP_FLAG_RANKDEF;
  }
}

__global__ void __launch_bounds__(NTH)
k_chol_tiles(const double* __restrict__ G, int d, double shift_rel, int force_shift,
             float* __restrict__ tiles, DevStatus* __restrict__ status,
             const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  chol_body(G, d, shift_rel, force_shift, tiles, status);
}

// One CTA per matrix of the problem table.
__global__ void __launch_bounds__(NTH)
k_bchol(const BMat* __restrict__ T, double shift_rel, int force_shift) {
  const BMat& b = T[blockIdx.x];
  chol_body(b.G, b.d, shift_rel, force_shift, b.tiles, b.status);
}

// X = Y R^{-1} by blocked forward substitution over 32-column tiles:
//   X_J = (Y_J - sum_{K<J} X_K R_KJ) R_JJ^{-1}.
// A CTA owns 32 rows, staged in shared memory (so X may alias Y).  R tiles
// and diagonal-tile inverses come from k_chol_tiles' packed layout; they are
// fetched with cp.async NPF tiles ahead of their use (L2 latency is long).
constexpr int SR = 32;
constexpr int NPF = 4;  // tile buffers (prefetch distance NPF - 1)
__device__ __forceinline__ void trsm_body(const float* __restrict__ Y, int64_t ldy,
                                          const float* __restrict__ tiles, float* X, int64_t ldx,
                                          int64_t M, int d, int rb) {
  extern __shared__ __align__(16) float ys[];  // SR x pitch
  __shared__ __align__(16) float Rt[NPF][TB][TB];
  const int nb = (d + TB - 1) / TB;
  const int ntiles = nb * (nb + 1) / 2;
  const int pitch = nb * TB + 4;
  const int64_t r0 = (int64_t)rb * SR;
  const int nr = (int)min((int64_t)SR, M - r0);
  const int t = threadIdx.x;
  // stage the rows (float4 when the row pitch allows it)
  const int nv = nb * TB / 4;  // float4s per padded row
  const bool vec = (ldy % 4 == 0) && (((uintptr_t)Y & 15) == 0);
  // loads are issued in batches of 8 before their stores, so 8 are in flight
  for (int e0 = t; e0 < SR * nv; e0 += 8 * 128) {
    float4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 128;
      v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < SR * nv) {
        const int r = e / nv, c = (e % nv) * 4;
        if (r < nr) {
          const float* p = Y + (r0 + r) * ldy + c;
          if (vec && c + 3 < d) v[q] = *reinterpret_cast<const float4*>(p);
          else {
            if (c < d) v[q].x = p[0];
            if (c + 1 < d) v[q].y = p[1];
            if (c + 2 < d) v[q].z = p[2];
            if (c + 3 < d) v[q].w = p[3];
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 128;
      if (e < SR * nv) {
        const int r = e / nv, c = (e % nv) * 4;
        *reinterpret_cast<float4*>(ys + r * pitch + c) = v[q];
      }
    }
  }
  // sequence of tiles used: for J: R_0J .. R_{J-1}J, then inv(R_JJ)
  auto tile_ptr = [&](int J, int K) {
    return (K < J) ? tiles + (size_t)bidx(K, J, nb) * TB * TB
                   : tiles + (size_t)(ntiles + J) * TB * TB;
  };
  // asynchronous copy of one 4 KB tile (2 x 16 bytes per thread)
  auto fetch = [&](int b, const float* src) {
    for (int e = t; e < TB * TB / 4; e += 128) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&Rt[b][0][0] + 4 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 4 * e)
                   : "memory");
    }
  };
  const int row = t >> 2, c0 = (t & 3) * 8;
  float* yr = ys + row * pitch;
  // the tile sequence is (J=0: inv00), (J=1: R01, inv11), (J=2: R02, R12, inv22) ...
  // step s -> (J, K) with K <= J; total nb (nb + 1) / 2 steps
  const int nsteps = nb * (nb + 1) / 2;
  auto step_tile = [&](int sidx) {
    int J = 0;
    while (sidx > J) { sidx -= J + 1; ++J; }
    return tile_ptr(J, sidx);
  };
  for (int q = 0; q < NPF - 1; ++q) {
    if (q < nsteps) fetch(q % NPF, step_tile(q));
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int sidx = 0;
  for (int J = 0; J < nb; ++J) {
    float acc[8];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = yr[J * TB + c0 + i];
    for (int K = 0; K <= J; ++K, ++sidx) {
      __syncthreads();  // everyone is done with the buffer about to be refilled
      if (sidx + NPF - 1 < nsteps) fetch((sidx + NPF - 1) % NPF, step_tile(sidx + NPF - 1));
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (K == J) {
        // stage the updated tile of this row, then multiply by R_JJ^{-1}
#pragma unroll
        for (int i = 0; i < 8; ++i) yr[J * TB + c0 + i] = acc[i];
      }
      asm volatile("cp.async.wait_group %0;" ::"n"(NPF - 1) : "memory");  // step's tile landed
      __syncthreads();
      const float* R = &Rt[sidx % NPF][0][0];
      if (K < J) {
#pragma unroll 8
        for (int k = 0; k < TB; ++k) {
          const float x = yr[K * TB + k];
          const float4 a0 = *reinterpret_cast<const float4*>(R + k * TB + c0);
          const float4 a1 = *reinterpret_cast<const float4*>(R + k * TB + c0 + 4);
          acc[0] = fmaf(-x, a0.x, acc[0]);
          acc[1] = fmaf(-x, a0.y, acc[1]);
          acc[2] = fmaf(-x, a0.z, acc[2]);
          acc[3] = fmaf(-x, a0.w, acc[3]);
          acc[4] = fmaf(-x, a1.x, acc[4]);
          acc[5] = fmaf(-x, a1.y, acc[5]);
          acc[6] = fmaf(-x, a1.z, acc[6]);
          acc[7] = fmaf(-x, a1.w, acc[7]);
        }
      } else {
        float out[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int k = 0; k < TB; ++k) {
          const float x = yr[J * TB + k];
          const float4 a0 = *reinterpret_cast<const float4*>(R + k * TB + c0);
          const float4 a1 = *reinterpret_cast<const float4*>(R + k * TB + c0 + 4);
          out[0] = fmaf(x, a0.x, out[0]);
          out[1] = fmaf(x, a0.y, out[1]);
          out[2] = fmaf(x, a0.z, out[2]);
          out[3] = fmaf(x, a0.w, out[3]);
          out[4] = fmaf(x, a1.x, out[4]);
          out[5] = fmaf(x, a1.y, out[5]);
          out[6] = fmaf(x, a1.z, out[6]);
          out[7] = fmaf(x, a1.w, out[7]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) yr[J * TB + c0 + i] = out[i];
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const bool vecx = (ldx % 4 == 0) && (((uintptr_t)X & 15) == 0);
  for (int e = t; e < SR * nv; e += 128) {
    const int r = e / nv, c = (e % nv) * 4;
    if (r >= nr || c >= d) continue;
    const float4 v = *reinterpret_cast<const float4*>(ys + r * pitch + c);
    float* p = X + (r0 + r) * ldx + c;
    if (vecx && c + 3 < d) *reinterpret_cast<float4*>(p) = v;
    else {
      p[0] = v.x;
      if (c + 1 < d) p[1] = v.y;
      if (c + 2 < d) p[2] = v.z;
      if (c + 3 < d) p[3] = v.w;
    }
  }
}

__global__ void __launch_bounds__(128)
k_trsm_tiles(const float* __restrict__ Y, int64_t ldy, const float* __restrict__ tiles, float* X,
             int64_t ldx, int64_t M, int d) {
  trsm_body(Y, ldy, tiles, X, ldx, M, d, blockIdx.x);
}

// Batched: block t -> (matrix, 32-row block); M = rows of buf[src].
__global__ void __launch_bounds__(128)
k_btrsm(const BMat* __restrict__ T, const int* __restrict__ prefix, int count, int src, int dst) {
  const int t = blockIdx.x;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const BMat& b = T[lo];
  const int64_t M = (src == B_Y) ? b.m : b.n;
  trsm_body(bbuf(b, src), b.dp, b.tiles, bbuf(b, dst), b.dp, M, b.d, t - prefix[lo]);
}

}  // namespace

int btrsm_blocks(int64_t M) { return ceil_div(M, SR); }

cudaError_t bchol(const BMat* T, int count, double shift_rel, bool force_shift, int dmax,
                  cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (!chol_tiles_supported(dmax)) return cudaErrorInvalidValue;
  const size_t sm = chol_tiles_smem(dmax);
  cudaError_t e =
      cudaFuncSetAttribute(k_bchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_bchol<<<count, NTH, sm, st>>>(T, shift_rel, force_shift ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t btrsm(const BMat* T, const int* prefix, int total, int count, int src, int dst,
                  int dmax, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  const int nb = (dmax + TB - 1) / TB;
  const size_t sm = (size_t)SR * (nb * TB + 4) * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_btrsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_btrsm<<<total, 128, sm, st>>>(T, prefix, count, src, dst);
  count_launch();
  return cudaGetLastError();
}

size_t chol_tiles_smem(int d) {
  const int nb = (d + TB - 1) / TB;
  return ((size_t)nb * (nb + 1) / 2 + nb) * TILE_FLOATS * sizeof(float);
}

bool chol_tiles_supported(int d) {
  return d >= 1 && (d + TB - 1) / TB <= MAXNB && chol_tiles_smem(d) <= 220 * 1024;
}

size_t chol_tiles_bytes(int d) {
  const int nb = (d + TB - 1) / TB;
  return ((size_t)nb * (nb + 1) / 2 + nb) * TB * TB * sizeof(float);
}

cudaError_t chol_tiles_f32(const double* G, int d, double shift_rel, bool force_shift,
                           float* tiles, DevStatus* status, const int32_t* gate, cudaStream_t st) {
  if (!chol_tiles_supported(d)) return cudaErrorInvalidValue;
  const size_t sm = chol_tiles_smem(d);
  cudaError_t e =
      cudaFuncSetAttribute(k_chol_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_chol_tiles<<<1, NTH, sm, st>>>(G, d, shift_rel, force_shift ? 1 : 0, tiles, status, gate);
  count_launch();
  return cudaGetLastError();
}

cudaError_t trsm_tiles_f32(const float* Y, int64_t ldy, const float* tiles, float* X, int64_t ldx,
                           int64_t M, int d, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const int nb = (d + TB - 1) / TB;
  const size_t sm = (size_t)SR * (nb * TB + 4) * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_trsm_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_trsm_tiles<<<ceil_div(M, SR), 128, sm, st>>>(Y, ldy, tiles, X, ldx, M, d);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
