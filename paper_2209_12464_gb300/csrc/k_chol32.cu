// FP32 pieces of the shifted CholeskyQR3 orth() (Section II-A orth();
// Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020) for d <= 288:
//
//  * k_chol_tiles: one CTA factors the d x d Gram G (+ shift I) = R^T R,
//    blocked in 32 x 32 tiles held in shared memory (upper block triangle,
//    padded to a multiple of 32 with the identity; loaded with cp.async).
//    Each diagonal tile is factored and inverted by one warp in registers
//    (row broadcasts through shared memory); the panel solves (products with
//    the tile inverse) and trailing updates are 32 x 16 half-tile products,
//    one per warp, 4 x 4 outputs per lane, so the factorisation needs three
//    block barriers per tile row, not per column.  The Gram arrives in FP32
//    (rounded by the slab reduction), so the kernel does no FP64 arithmetic.
//    The last pass of a CholeskyQR (its own instantiation) checks the pivots
//    for numerical rank deficiency and, for a Gram within sqrt(2^-25 / d) of
//    I, writes the factor to first order in G - I instead.
//  * k_trsm_tiles: Q = Y R^{-1} by blocked forward substitution with those
//    tiles (rows of Y staged transposed in shared memory, so Q may overwrite
//    Y).
#include <math.h>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace ruqlp {
size_t chol_tiles_smem(int d);
namespace {

constexpr int TB = 32;        // tile edge
constexpr int TP = 36;        // row pitch: 16-byte aligned rows for 128-bit loads
constexpr int MAXNB = 9;      // d <= 288
constexpr int NTH = 512;      // 16 warps; up to 128 registers for per-lane tile columns
constexpr size_t TILE_FLOATS = (size_t)TB * TP;

__device__ __forceinline__ int bidx(int I, int J, int nb) { return I * nb - (I * (I - 1)) / 2 + (J - I); }

// acc[i][j] = sum_k A[k][r0 + i] B[k][c0 + j] for a lane's 4 x 4 block of a
// 32 x 32 tile product A^T B (tiles in shared memory, pitch TP), k ascending
// from zero; two 128-bit loads feed 16 multiply-adds.
__device__ __forceinline__ void tile_tn44(const float* __restrict__ A, const float* __restrict__ B,
                                          int r0, int c0, float (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 8
  for (int k = 0; k < TB; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(A + k * TP + r0);
    const float4 b = *reinterpret_cast<const float4*>(B + k * TP + c0);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

__device__ __forceinline__ void load_col(const float* __restrict__ T, int lane, float (&c)[TB]) {
#pragma unroll
  for (int k = 0; k < TB; ++k) c[k] = T[k * TP + lane];
}

// One warp factors the 32 x 32 tile B = R^T R in registers (lane c owns
// column c) and writes R (upper) back and S = R^{-1} (upper, row-major) to
// Sout.  Step k broadcasts row k of the partially reduced tile through the
// shared row buffer rb (one store per lane, 128-bit broadcast loads of the
// whole row issued together) and the pivot by a shuffle, so every lane forms
// r_ki itself; there are no branches or masks in the loop.  The inverse comes
// out of the same elimination: the row operations that reduce B (row i -=
// (b_ki / b_kk) row k) are applied to the identity too, which leaves the
// inverse of the unit lower factor; lane c's copy of column c, scaled by
// 1 / r_jj as pivot j is formed, is row c of S.  Reciprocal square roots
// replace IEEE sqrt/divide (the factor only has to be consistent with the
// solve that uses it).  A non-positive pivot is replaced by bad_fill; the
// return value (same in every lane) reports whether that happened.
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

__device__ __noinline__ bool factor_tile(float* __restrict__ B, float* __restrict__ Sout,
                                         float* __restrict__ rb, int lane, float bad_fill) {
  float col[TB], ecol[TB];
  load_col(B, lane, col);
#pragma unroll
  for (int i = 0; i < TB; ++i) ecol[i] = (i == lane) ? 1.f : 0.f;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < TB; ++k) {
    __syncwarp();
    rb[lane] = col[k];  // row k of the current tile, lane c holds B[k][c]
    float piv = __shfl_sync(0xffffffffu, col[k], k);
    __syncwarp();
    float row[TB];
    load_row(rb, row);
    const bool nonpos = !(piv > 0.f) || !(piv < 3.0e38f);
    bad = bad || nonpos;
    piv = nonpos ? bad_fill : piv;
    const float rinv = rsqrtf(piv);
    const float rkc = ((lane == k) ? piv : col[k]) * rinv;  // r_kc for c >= k
    col[k] = rkc;
    const float skc = ecol[k] * rinv;  // S[c][k]
    ecol[k] = skc;
    // b_ic -= r_ki r_kc with r_ki = b_ki / sqrt(piv), and the same row
    // operation on the identity: one multiply-add per entry each.  The
    // entries of B below the diagonal (i > c) are updated too, without a
    // mask: they are never read as row values (step k reads only lanes >= k)
    // and are zeroed on the way out.
    const float tkc = rkc * rinv, tec = skc * rinv;
#pragma unroll
    for (int i = k + 1; i < TB; ++i) {
      col[i] = fmaf(-row[i], tkc, col[i]);
      ecol[i] = fmaf(-row[i], tec, ecol[i]);
    }
  }
#pragma unroll
  for (int r = 0; r < TB; ++r) {
    B[r * TP + lane] = (r <= lane) ? col[r] : 0.f;
    Sout[lane * TP + r] = (r >= lane) ? ecol[r] : 0.f;
  }
  __syncwarp();
  return !bad;
}

// Blocked Cholesky G (+ shift I) = R^T R, d <= 288, one CTA of NT threads
// (NT >= 128; each tile operation is done by one warp, so the result does not
// depend on NT).  Writes the upper tiles R_IJ (I <= J) and the diagonal-tile
// inverses R_KK^{-1}, FP32, 32 x 32 row-major each, to `tiles`: first the
// nb (nb+1)/2 R tiles in row-of-tiles order, then the nb inverse tiles.
// CHECK: this is the last pass of a CholeskyQR whose input should already be
// orthonormal to working accuracy, so every pivot must lie in [1/2, 2]; if
// one does not, the sketch is numerically rank deficient for CholeskyQR at
// this precision and RUQLP_FLAG_RANKDEF is raised (the host then redoes the
// decomposition with Householder TSQR).  When such a Gram is within
// sqrt(2^-25 / d) of I entry by entry, the factor is formed to first order
// in G - I instead of by elimination (the same factor to working precision;
// no chain of pivots).
template <int NT, bool CHECK>
__device__ __forceinline__ void chol_body(const float* __restrict__ G, int d, double shift_rel,
                                          int force_shift, float* __restrict__ tiles,
                                          DevStatus* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float s_shift;
  __shared__ int s_bad, s_rankdef, s_far, s_near;
  __shared__ float s_red[NT / 32];
  __shared__ __align__(16) float s_row[TB];
  __shared__ unsigned char s_tI[MAXNB * (MAXNB + 1) / 2], s_tJ[MAXNB * (MAXNB + 1) / 2];
  const int nb = (d + TB - 1) / TB;
  const int ntiles = nb * (nb + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
  auto tile = [&](int I, int J) { return sm + (size_t)bidx(I, J, nb) * TILE_FLOATS; };
  // the current diagonal tile's inverse (shared; copied out once used)
  float* const dinv_sm = sm + (size_t)ntiles * TILE_FLOATS;
  // a lane's 4 x 4 block within a 32 x 16 half tile: rows 4 rg.., columns 4 cg..
  const int rg = lane >> 2, cg = lane & 3;

  if (tid == 0) {
    s_rankdef = 0;
    s_far = 0;
    s_near = 0;
  }
  if (tid < ntiles) {  // packed tile index -> (I, J)
    int I = 0, tt = tid;
    while (tt >= nb - I) { tt -= nb - I; ++I; }
    s_tI[tid] = (unsigned char)I;
    s_tJ[tid] = (unsigned char)(I + tt);
  }
  // rows of G start on 16 bytes when d % 4 == 0: then whole 4-column chunks
  // are either inside G or past its edge
  const bool vec = (d % 4 == 0) && (((uintptr_t)G & 15) == 0);
  // item u of a step's trailing update (rem tile rows left): tile (I, J),
  // K < I <= J, column half u & 1
  auto update = [&](int K, int rem, int u) {
    int I = 0, tt = u >> 1;
    while (tt >= rem - I) { tt -= rem - I; ++I; }
    I += K + 1;
    const int J = I + tt, c0 = (u & 1) * 16 + cg * 4;
    float acc[4][4];
    tile_tn44(tile(K, I), tile(K, J), rg * 4, c0, acc);
    float* C = tile(I, J);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4* pc = reinterpret_cast<float4*>(C + (rg * 4 + i) * TP + c0);
      float4 v = *pc;
      v.x -= acc[i][0];
      v.y -= acc[i][1];
      v.z -= acc[i][2];
      v.w -= acc[i][3];
      *pc = v;
    }
  };
  int attempt = force_shift ? 1 : 0;
  for (; attempt < 2; ++attempt) {
    __syncthreads();
    // upper block triangle of G
    if (vec) {
      // 16-byte cp.async chunks (zero-filled past the edge), all in flight at once
      for (int e = tid; e < ntiles * TB * 8; e += NT) {
        const int t = e >> 8, r = (e >> 3) & 31, c4 = (e & 7) * 4;
        const int I = s_tI[t], J = s_tJ[t];
        const int i = I * TB + r, j = J * TB + c4;
        const bool in = i < d && j < d;
        const float* src = in ? G + (size_t)i * d + j : G;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tile(I, J) + r * TP + c4);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                     "r"(in ? 16 : 0)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else {
      // one warp per tile, lane = column, 16 row loads in flight per lane
      for (int t = warp; t < ntiles; t += nw) {
        const int I = s_tI[t], J = s_tJ[t];
        const int j = J * TB + lane;
        float* T = tile(I, J);
#pragma unroll
        for (int h = 0; h < TB; h += 16) {
          float v[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int i = I * TB + h + r;
            v[r] = (i < d && j < d) ? G[(size_t)i * d + j] : 0.f;
          }
#pragma unroll
          for (int r = 0; r < 16; ++r) T[(h + r) * TP + lane] = v[r];
        }
      }
    }
    __syncthreads();
    if (warp == 0) {  // shift = shift_rel * trace(G), from the loaded tiles
      float t = 0.f;
      for (int i = lane; i < d; i += 32) t += tile(i / TB, i / TB)[(i % TB) * (TP + 1)];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        float sh = (float)shift_rel * t;
        if (!(sh > 0.f)) sh = 1e-30f;
        s_shift = sh;
        s_bad = 0;
      }
    }
    __syncthreads();
    const float add = attempt ? s_shift : 0.f;
    for (int i = tid; i < nb * TB; i += NT) {  // + shift I; identity padding
      float* p = tile(i / TB, i / TB) + (i % TB) * (TP + 1);
      *p = (i < d) ? *p + add : 1.f;
    }
    __syncthreads();
    if (CHECK && attempt == 0) {
      // The last pass of a CholeskyQR: G = I + E with E at the level of the
      // previous pass's loss of orthogonality.  R = I + X with X upper
      // triangular solves X + X^T = E - X^T X, so X = Phi(E) (the strict
      // upper triangle of E and half its diagonal) up to |X^T X| <= d e^2,
      // e = max |E_ij|; when d e^2 <= 2^-25 that is below FP32 rounding and
      // R = I + Phi(E) is the Cholesky factor to working precision, its
      // diagonal tiles' inverses I - (R_KK - I) likewise (the dropped
      // (R_KK - I)^2 is at most 32 e^2).  NaN entries fail the test.
      float e = 0.f;
      for (int x = tid; x < ntiles * TB * TB; x += NT) {
        const int tt = x >> 10, r = (x >> 5) & (TB - 1), c = x & (TB - 1);
        const int I = s_tI[tt], J = s_tJ[tt];
        if (I == J && c < r) continue;
        const float g = tile(I, J)[r * TP + c];
        const float v = fabsf((I == J && r == c) ? g - 1.f : g);
        e = (v > e || v != v) ? v : e;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, e, o);
        e = (w > e || w != w) ? w : e;
      }
      if (lane == 0) s_red[warp] = e;
      __syncthreads();
      if (tid == 0) {
        float m = 0.f;
        for (int w = 0; w < nw; ++w) m = (s_red[w] > m || s_red[w] != s_red[w]) ? s_red[w] : m;
        s_near = (float)d * m * m <= 2.98023223876953125e-08f;  // 2^-25
      }
      __syncthreads();
      if (s_near) {
        for (int x = tid; x < ntiles * TB * TB; x += NT) {
          const int tt = x >> 10, r = (x >> 5) & (TB - 1), c = x & (TB - 1);
          const int I = s_tI[tt], J = s_tJ[tt];
          if (I != J) continue;
          float* p = tile(I, J) + r * TP + c;
          *p = c < r ? 0.f : (c == r ? 0.5f * (1.f + *p) : *p);
        }
        __syncthreads();
        for (int x = tid; x < nb * TB * TB; x += NT) {
          const int K = x >> 10, r = (x >> 5) & (TB - 1), c = x & (TB - 1);
          const float rv = tile(K, K)[r * TP + c];
          tiles[(size_t)(ntiles + K) * TB * TB + r * TB + c] =
              c < r ? 0.f : (c == r ? 1.f / rv : -rv);
        }
        break;
      }
    }
    const float fill = attempt == 0 ? 1.f : add;
    // Step K = -1 only factors the first diagonal tile; step K >= 0 does the
    // panel of tile row K, updates tile (K+1, K+1), then factors it on warp 0
    // while the warps of the other three schedulers (warp % 4 != 0) do the
    // rest of the trailing update, so that the one-warp chain keeps its issue
    // slots.  The factorisation has one call site (its unrolled code is
    // large).
    for (int K = -1; K < nb; ++K) {
      if (K >= 0) {
        if (s_bad) break;
        // (b) panel B_KJ <- R_KK^{-T} B_KJ, items (J, column half): each item
        // reads and writes only its own 32 x 16 block, so a warp barrier
        // separates its reads from its writes.  The last warp also copies
        // the diagonal inverse out.
        const int npan = 2 * (nb - K - 1);
        for (int u = warp; u < npan; u += nw) {
          float* B = tile(K, K + 1 + (u >> 1));
          const int c0 = (u & 1) * 16 + cg * 4;
          float acc[4][4];
          tile_tn44(dinv_sm, B, rg * 4, c0, acc);
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 4; ++i)
            *reinterpret_cast<float4*>(B + (rg * 4 + i) * TP + c0) =
                make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
          __syncwarp();
        }
        if (warp == nw - 1) {
          float* gi = tiles + (size_t)(ntiles + K) * TB * TB;
#pragma unroll 8
          for (int r = 0; r < TB; ++r) gi[r * TB + lane] = dinv_sm[r * TP + lane];
        }
        __syncthreads();
      }
      // (c) trailing update B_IJ -= B_KI^T B_KJ (items 0 and 1 are the two
      // halves of tile (K+1, K+1)) and the next diagonal tile
      const int rem = nb - K - 1;
      if (rem > 0) {
        if (K >= 0) {
          if (warp < 2) update(K, rem, warp);
          __syncthreads();
        }
        if (warp == 0) {
          const bool ok = factor_tile(tile(K + 1, K + 1), dinv_sm, s_row, lane, fill);
          if (lane == 0 && !ok) {
            if (attempt == 0) s_bad = 1;  // retry on G + shift I
            else s_rankdef = 1;           // pivots replaced by the shift
          }
        } else if (K >= 0 && (warp & 3) != 0) {
          const int nw3 = nw - nw / 4, w3 = warp - warp / 4 - 1;  // 0 .. nw3 - 1
          for (int u = 2 + w3; u < rem * (rem + 1); u += nw3) update(K, rem, u);
        }
      }
      __syncthreads();
    }
    if (!s_bad) break;
  }
  __syncthreads();
  if (CHECK && !s_near && warp == 0) {
    // the last pass of a CholeskyQR: its Gram should be close to I, so every
    // pivot r_ii^2 lies in [1/2, 2] and no retry with the shift was needed
    bool far = attempt > 0 && !force_shift;
    for (int i = lane; i < d; i += 32) {
      const float r = tile(i / TB, i / TB)[(i % TB) * (TP + 1)];
      far = far || !(r * r >= 0.5f && r * r <= 2.0f);
    }
    if (__any_sync(0xffffffffu, far) && lane == 0) s_far = 1;
  }
  __syncthreads();
  // write the R tiles (32 x 32 row-major each; the inverses are out already)
  for (int t = warp; t < ntiles; t += nw) {
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
    if (s_rankdef || s_far) status->flags |= RUQLP_FLAG_RANKDEF;
  }
}

// CHECK (the last pass of a CholeskyQR: the near-identity route and the
// rank-deficiency check) is a separate instantiation: the code it adds
// around the factorisation made the other passes' factorisation measurably
// slower (instruction-cache residency of its unrolled body).
template <bool CHECK>
__global__ void __launch_bounds__(NTH)
k_chol_tiles(const float* __restrict__ G, int d, double shift_rel, int force_shift,
             float* __restrict__ tiles, DevStatus* __restrict__ status,
             const int32_t* __restrict__ gate) {
  pdl_launch();
  pdl_wait();
  if (gate != nullptr && *gate == 0) return;
  chol_body<NTH, CHECK>(G, d, shift_rel, force_shift, tiles, status);
}

// One CTA per matrix of the problem table; small batches of small d take
// 128-thread CTAs, four per SM.
template <int NT, bool CHECK>
__global__ void __launch_bounds__(NT, NT == 128 ? 4 : 1)
k_bchol(const BMat* __restrict__ T, double shift_rel, int force_shift) {
  const BMat& b = T[blockIdx.x];
  chol_body<NT, CHECK>(b.Gf, b.d, shift_rel, force_shift, b.tiles, b.status);
}

template <int NT, bool CHECK>
cudaError_t bchol_launch(const BMat* T, int count, double shift_rel, bool force_shift, size_t sm,
                         cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_bchol<NT, CHECK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_bchol<NT, CHECK><<<count, NT, sm, st>>>(T, shift_rel, force_shift ? 1 : 0);
  return cudaSuccess;
}

// X = Y R^{-1} by blocked forward substitution over 32-column tiles:
//   X_J = (Y_J - sum_{K<J} X_K R_KJ) R_JJ^{-1}.
// A CTA of 64 threads owns 32 rows, staged TRANSPOSED in shared memory
// (ys[c][r], so X may alias Y); thread (rg, cg) keeps a 4 x 4 block (rows
// 4rg.., columns 4cg.. of the current tile) in registers, and every step of a
// tile product is two 128-bit loads (4 rows of X, 4 columns of R) for 16
// multiply-adds.  R tiles and diagonal-tile inverses come from k_chol_tiles'
// packed layout and are fetched with cp.async NPF - 1 tiles ahead.
// SR rows per CTA (32 for single matrices, 128 for batches of small ones;
// the arithmetic of every element is the same either way), TT = 2 SR threads,
// YP = pitch of a transposed column (16-byte aligned).
constexpr int SR1 = 32, SRB = 128;
constexpr int NPF = 3;        // tile buffers (prefetch distance NPF - 1)
// Bt (optional): also write X^T in BF16 (dp x ldbt, K-major: the next
// tensor-core product's B operand), zero in the padding rows d..dp; Btl
// (optional) the low parts bf16(x - bf16(x)) in the same layout.
template <int SR>
__device__ __forceinline__ void trsm_body(const float* __restrict__ Y, int64_t ldy,
                                          const float* __restrict__ tiles, float* X, int64_t ldx,
                                          int64_t M, int d, int rb,
                                          __nv_bfloat16* __restrict__ Bt = nullptr,
                                          int64_t ldbt = 0,
                                          __nv_bfloat16* __restrict__ Btl = nullptr) {
  constexpr int TT = 2 * SR, YP = SR + 4, RG = SR / 4;
  extern __shared__ __align__(16) float ys[];  // round4(d) x YP, ys[c * YP + r]
  __shared__ __align__(16) float Rt[NPF][TB][TB];
  const int nb = (d + TB - 1) / TB;
  const int ntiles = nb * (nb + 1) / 2;
  const int64_t r0 = (int64_t)rb * SR;
  const int nr = (int)min((int64_t)SR, M - r0);
  const int t = threadIdx.x;
  // 4-column groups holding columns below d: the padding columns of the
  // last block column are never read as inputs (the diagonal step sums
  // k < vJ only and no block column K < J reaches past d), so they are not
  // staged
  const int nv = (d + 3) / 4;
  const bool vec = (ldy % 4 == 0) && (((uintptr_t)Y & 15) == 0);
  // stage: item e -> row e % SR, column group e / SR (a warp takes one group
  // of 32 rows, so the transposed stores hit 32 banks); 8 loads in flight
  for (int e0 = t; e0 < SR * nv; e0 += 8 * TT) {
    float4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * TT;
      v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < SR * nv) {
        const int r = e % SR, c = (e / SR) * 4;
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
      const int e = e0 + q * TT;
      if (e < SR * nv) {
        const int r = e % SR, c = (e / SR) * 4;
        ys[(c + 0) * YP + r] = v[q].x;
        ys[(c + 1) * YP + r] = v[q].y;
        ys[(c + 2) * YP + r] = v[q].z;
        ys[(c + 3) * YP + r] = v[q].w;
      }
    }
  }
  // sequence of tiles used: for J: R_0J .. R_{J-1}J, then inv(R_JJ)
  auto tile_ptr = [&](int J, int K) {
    return (K < J) ? tiles + (size_t)bidx(K, J, nb) * TB * TB
                   : tiles + (size_t)(ntiles + J) * TB * TB;
  };
  // asynchronous copy of one 4 KB tile (4 x 16 bytes per thread)
  auto fetch = [&](int b, const float* src) {
    for (int e = t; e < TB * TB / 4; e += TT) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&Rt[b][0][0] + 4 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 4 * e)
                   : "memory");
    }
  };
  const int rg = t % RG, cg = t / RG;  // rows 4rg..4rg+3, tile columns 4cg..4cg+3
  // the tile sequence is (J=0: inv00), (J=1: R01, inv11), (J=2: R02, R12, inv22) ...
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
  auto col4 = [&](int c) { return reinterpret_cast<float4*>(ys + c * YP + rg * 4); };
  int sidx = 0;
  __syncthreads();  // the staged rows
  for (int J = 0; J < nb; ++J) {
    // block column J holds vJ = min(32, d - 32 J) columns: a thread whose
    // four columns lie past them (not live) neither reads nor writes the
    // staged block in this block column, so the staging holds only the
    // columns below d rounded up to 4.  A thread's own columns of block J
    // are read and written only by itself until the diagonal step.
    const int vJ = min(TB, d - J * TB);
    const bool live = cg * 4 < vJ;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = live ? *col4(J * TB + cg * 4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[0][j] = v.x;
      acc[1][j] = v.y;
      acc[2][j] = v.z;
      acc[3][j] = v.w;
    }
    for (int K = 0; K <= J; ++K, ++sidx) {
      if (K == J && live) {
        // stage the updated tile of this row block, then multiply by R_JJ^{-1}
#pragma unroll
        for (int j = 0; j < 4; ++j)
          *col4(J * TB + cg * 4 + j) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
      }
      asm volatile("cp.async.wait_group %0;" ::"n"(NPF - 2) : "memory");  // own copies of this step's tile
      // one barrier per step: every thread's copies of this step's tile have
      // landed, the staged tile above is visible, and every thread is done
      // with step sidx - 1, whose buffer the next copy refills
      __syncthreads();
      if (sidx + NPF - 1 < nsteps) fetch((sidx + NPF - 1) % NPF, step_tile(sidx + NPF - 1));
      asm volatile("cp.async.commit_group;" ::: "memory");
      const float* R = &Rt[sidx % NPF][0][0];
      // a thread that is not live skips the tile products; the diagonal
      // step sums k < min(vJ, 4 cg + 4) only (the inverse of R_JJ is upper
      // triangular: S[k][j] = 0 for k > j, so the terms dropped for the
      // thread's columns j <= 4 cg + 3 are exact zeros)
      if (K < J) {
        if (live)
#pragma unroll 8
        for (int k = 0; k < TB; ++k) {
          const float4 y = *col4(K * TB + k);
          const float4 r = *reinterpret_cast<const float4*>(R + k * TB + cg * 4);
          const float yv[4] = {y.x, y.y, y.z, y.w}, rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(-yv[i], rv[j], acc[i][j]);
        }
      } else {
        float out[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) out[i][j] = 0.f;
        const int kend = live ? min(vJ, cg * 4 + 4) : 0;
#pragma unroll 4
        for (int k = 0; k < kend; ++k) {
          const float4 y = *col4(J * TB + k);
          const float4 r = *reinterpret_cast<const float4*>(R + k * TB + cg * 4);
          const float yv[4] = {y.x, y.y, y.z, y.w}, rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) out[i][j] = fmaf(yv[i], rv[j], out[i][j]);
        }
        __syncthreads();
        if (live)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *col4(J * TB + cg * 4 + j) = make_float4(out[0][j], out[1][j], out[2][j], out[3][j]);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const bool vecx = (ldx % 4 == 0) && (((uintptr_t)X & 15) == 0);
  for (int e = t; e < SR * nv; e += TT) {
    const int r = e % SR, c = (e / SR) * 4;
    if (r >= nr || c >= d) continue;
    const float4 v = make_float4(ys[c * YP + r], ys[(c + 1) * YP + r], ys[(c + 2) * YP + r],
                                 ys[(c + 3) * YP + r]);
    float* p = X + (r0 + r) * ldx + c;
    if (vecx && c + 3 < d) *reinterpret_cast<float4*>(p) = v;
    else {
      p[0] = v.x;
      if (c + 1 < d) p[1] = v.y;
      if (c + 2 < d) p[2] = v.z;
      if (c + 3 < d) p[3] = v.w;
    }
  }
  if (Bt != nullptr) {  // rows of X^T are columns of the staged block: contiguous in r
    const int dp = (d + 15) / 16 * 16;
    // eight consecutive rows of one column per item: two 128-bit shared
    // loads and one 128-bit store per part
    const bool vb = ((((uintptr_t)Bt | (uintptr_t)(Btl != nullptr ? Btl : Bt)) & 15) == 0) &&
                    (ldbt % 8 == 0) && (r0 % 8 == 0);
    constexpr int G8 = SR / 8;
    for (int e = t; e < G8 * dp; e += TT) {
      const int r = (e % G8) * 8, c = e / G8;
      if (r >= nr) continue;
      float v[8];
      if (c < d) {
        const float4 a = *reinterpret_cast<const float4*>(ys + c * YP + r);
        const float4 b = *reinterpret_cast<const float4*>(ys + c * YP + r + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
      }
      __nv_bfloat16 h[8], l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = __float2bfloat16_rn(v[u]);
        l[u] = __float2bfloat16_rn(v[u] - __bfloat162float(h[u]));
      }
      const int64_t o = (int64_t)c * ldbt + r0 + r;
      if (vb && r + 8 <= nr) {
        auto pack = [](const __nv_bfloat16 (&x)[8]) {
          uint32_t w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            w[u] = (uint32_t)__bfloat16_as_ushort(x[2 * u]) |
                   ((uint32_t)__bfloat16_as_ushort(x[2 * u + 1]) << 16);
          return make_uint4(w[0], w[1], w[2], w[3]);
        };
        *reinterpret_cast<uint4*>(Bt + o) = pack(h);
        if (Btl != nullptr) *reinterpret_cast<uint4*>(Btl + o) = pack(l);
      } else {
        for (int u = 0; u < 8 && r + u < nr; ++u) {
          Bt[o + u] = h[u];
          if (Btl != nullptr) Btl[o + u] = l[u];
        }
      }
    }
  }
}

__global__ void __launch_bounds__(2 * SR1)
k_trsm_tiles(const float* __restrict__ Y, int64_t ldy, const float* __restrict__ tiles, float* X,
             int64_t ldx, int64_t M, int d, __nv_bfloat16* __restrict__ Bt, int64_t ldbt,
             __nv_bfloat16* __restrict__ Btl) {
  pdl_launch();
  pdl_wait();
  trsm_body<SR1>(Y, ldy, tiles, X, ldx, M, d, blockIdx.x, Bt, ldbt, Btl);
}

// Batched: block t -> (matrix, 128-row block); M = rows of buf[src].
__global__ void __launch_bounds__(2 * SRB, 4)
k_btrsm(const BMat* __restrict__ T, const int* __restrict__ prefix, int count, int src, int dst,
        int make_bt) {
  const int t = blockIdx.x;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const BMat& b = T[prefix[count + 1 + lo]];  // the launch order's item lo
  const int64_t M = (src == B_Y) ? b.m : b.n;
  // make_bt == 2 marks the last solve of the final orth of Y
  const bool direct = make_bt == 2 && b.q_direct;
  trsm_body<SRB>(bbuf(b, src), b.dp, b.tiles, direct ? (float*)b.Qout : bbuf(b, dst),
            direct ? (int64_t)b.d : (int64_t)b.dp, M, b.d, t - prefix[lo],
            (make_bt && b.use_tc) ? (__nv_bfloat16*)b.Bt : nullptr, b.ldbt,
            (make_bt == 2 && b.use_tc) ? (__nv_bfloat16*)b.Btl : nullptr);
}

}  // namespace

int btrsm_blocks(int64_t M) { return ceil_div(M, SRB); }

cudaError_t bchol(const BMat* T, int count, double shift_rel, bool force_shift, int dmax,
                  cudaStream_t st, bool check) {
  if (count <= 0) return cudaSuccess;
  if (!chol_tiles_supported(dmax)) return cudaErrorInvalidValue;
  const size_t sm = chol_tiles_smem(dmax);
  cudaError_t e;
  if (dmax <= 96)
    e = check ? bchol_launch<128, true>(T, count, shift_rel, force_shift, sm, st)
              : bchol_launch<128, false>(T, count, shift_rel, force_shift, sm, st);
  else
    e = check ? bchol_launch<NTH, true>(T, count, shift_rel, force_shift, sm, st)
              : bchol_launch<NTH, false>(T, count, shift_rel, force_shift, sm, st);
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

cudaError_t btrsm(const BMat* T, const int* prefix, int total, int count, int src, int dst,
                  int dmax, cudaStream_t st, int make_bt) {
  if (total <= 0) return cudaSuccess;
  const size_t sm = (size_t)((dmax + 3) / 4 * 4) * (SRB + 4) * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_btrsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // the whole unified L1 as shared memory, so four CTAs fit per SM
  e = cudaFuncSetAttribute(k_btrsm, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  k_btrsm<<<total, 2 * SRB, sm, st>>>(T, prefix, count, src, dst, make_bt);
  count_launch();
  return cudaGetLastError();
}

size_t chol_tiles_smem(int d) {
  const int nb = (d + TB - 1) / TB;
  return ((size_t)nb * (nb + 1) / 2 + 1) * TILE_FLOATS * sizeof(float);
}

bool chol_tiles_supported(int d) {
  return d >= 1 && (d + TB - 1) / TB <= MAXNB && chol_tiles_smem(d) <= 220 * 1024;
}

size_t chol_tiles_bytes(int d) {
  const int nb = (d + TB - 1) / TB;
  return ((size_t)nb * (nb + 1) / 2 + nb) * TB * TB * sizeof(float);
}

cudaError_t chol_tiles_f32(const float* G, int d, double shift_rel, bool force_shift,
                           float* tiles, DevStatus* status, const int32_t* gate, cudaStream_t st,
                           bool check) {
  if (!chol_tiles_supported(d)) return cudaErrorInvalidValue;
  const size_t sm = chol_tiles_smem(d);
  auto kern = check ? k_chol_tiles<true> : k_chol_tiles<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3(1), dim3(NTH), sm, st, G, d, shift_rel, force_shift ? 1 : 0, tiles,
                 status, gate);
  count_launch();
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t trsm_tiles_f32(const float* Y, int64_t ldy, const float* tiles, float* X, int64_t ldx,
                           int64_t M, int d, cudaStream_t st, void* Bt, int64_t ldbt, void* Btl) {
  if (M <= 0) return cudaSuccess;
  const size_t sm = (size_t)((d + 3) / 4 * 4) * (SR1 + 4) * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_trsm_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_trsm_tiles, dim3(ceil_div(M, SR1)), dim3(2 * SR1), sm, st, Y, ldy, tiles, X,
                 ldx, M, d, (__nv_bfloat16*)Bt, ldbt,
                 Bt != nullptr ? (__nv_bfloat16*)Btl : nullptr);
  count_launch();
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace ruqlp
