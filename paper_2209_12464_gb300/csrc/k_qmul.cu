// Q = Y R^{-1} of orth() (Section II-A, CholeskyQR) on the tensor cores, for
// tall FP32 Y (M >= 8192 rows, d <= 256):
//
//  * k_trinv: S = R^{-1} (upper triangular, d x d) from the blocked Cholesky's
//    R tiles and diagonal-tile inverses, one CTA per 32-column block J (all
//    its tiles loaded at once):
//    S_JJ is given, and for K = J down to 1
//        acc_I += R_IK S_KJ          (all I < K, one tile product each)
//        S_{K-1,J} = -S_{K-1,K-1} acc_{K-1},
//    which is back substitution on R S_{:,J} = E_J.  S^T is written as three
//    BF16 parts s = h + m + l (h = bf16(s), m = bf16(s - h), l = bf16(s - h - m)),
//    K-major ([part][n][k], k padded to 256 with zeros): the B operand below.
//  * k_qmul_tc: Q = Y S with tcgen05.mma (BF16 x BF16 -> FP32 in TMEM).  Y is
//    split the same way on the fly; of the nine part products the six above
//    2^-24 are kept (hh, hm, mh, mm, hl, lh), so Q matches an FP32 product.
//    One CTA per SM owns an equal range of rows, taken as 128-row sub-tiles;
//    a sub-tile is accumulated over 64-wide K chunks, chunk c only into the
//    columns n >= 64 c (S is upper triangular).  Converter warps write the Y
//    chunk's parts into 128B-swizzled stages while a producer warp loads the
//    S parts with TMA and an MMA warp issues 6 x 4 MMAs per chunk and
//    sub-tile; the epilogue drains TMEM (two accumulators) and stores Q (and
//    optionally Q^T in BF16, the next product's operand).  A sub-tile's rows
//    are read in full before they are written, so Q may overwrite Y.
// Every mbarrier wait is bounded; on timeout the CTA sets the error word,
// waits for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace ruqlp {
namespace {

constexpr int TB = 32;   // tile edge of the Cholesky's blocking
constexpr int TP = 36;   // shared-memory row pitch (16-byte aligned rows)
constexpr int KP = 256;  // padded K of the S^T parts
constexpr int KPB = BO_KP;  // the same for batched items (d <= 128)
constexpr size_t TILE_F = (size_t)TB * TP;

__device__ __forceinline__ int bidx(int I, int J, int nb) { return I * nb - (I * (I - 1)) / 2 + (J - I); }

// acc[i][j] += sum_{k0 <= k < k1} A[rg + (128 / W) i][k] B[k][c0 + j] for a
// lane's (W / 4) x 4 block of a 32-row x W-column strip of A B (lanes:
// rg = lane / (W / 4), c0 = strip + 4 (lane % (W / 4))); k in order.
template <int W>
__device__ __forceinline__ void tile_strip(const float* __restrict__ A, const float* __restrict__ B,
                                           int rg, int c0, int k0, int k1,
                                           float (&acc)[W / 4][4]) {
  constexpr int RI = W / 4, RS = 128 / W;
#pragma unroll 2
  for (int k = k0; k < k1; k += 4) {
    float4 a[RI], b[4];
#pragma unroll
    for (int i = 0; i < RI; ++i) a[i] = *reinterpret_cast<const float4*>(A + (rg + RS * i) * TP + k);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = *reinterpret_cast<const float4*>(B + (k + q) * TP + c0);
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[i][0] = fmaf(av[q], b[q].x, acc[i][0]);
        acc[i][1] = fmaf(av[q], b[q].y, acc[i][1]);
        acc[i][2] = fmaf(av[q], b[q].z, acc[i][2]);
        acc[i][3] = fmaf(av[q], b[q].w, acc[i][3]);
      }
    }
  }
}

// 32 x 32 tile (pitch 32, global) -> shared (pitch TP) with cp.async
__device__ __forceinline__ void fetch_tile(float* dst, const float* src, int t, int nt) {
  for (int e = t; e < TB * 8; e += nt) {
    const int r = e >> 3, c4 = (e & 7) * 4;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst + r * TP + c4);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src + r * TB + c4)
                 : "memory");
  }
}

constexpr int TI_THREADS = 512;
constexpr int TI_W = 4;                 // columns of S per CTA (a strip)
constexpr int TI_STRIPS = TB / TI_W;    // strips per 32-column block

// Columns 32 J + W h .. + W - 1 of S = R^{-1} (block column J, strip h of
// 32 / W: the strips are independent right-hand sides of the back
// substitution, so each has its own CTA, the chain's tile products shrink to
// 32 x W strips and every element is formed exactly as with whole tiles).
// tiles: the Cholesky's R tiles (packed upper block triangle, 32 x 32
// row-major each) followed by the nb diagonal-tile inverses.  Writes rows
// n = 32 J + W h .. of St[3][dp][KPX] (K padded to KPX).  Every tile the
// column needs (R_IK for I < K <= J, S_KK for K <= J) is loaded at once;
// acc_I is accumulated in the slot of S_IJ and turned into S_IJ in place.
template <int KPX>
__device__ __forceinline__ void trinv_body(const float* __restrict__ tiles, int d, int dp, int J,
                                           int h, __nv_bfloat16* __restrict__ St, float* sm) {
  constexpr int W = TI_W, RI = W / 4, RS = 128 / W;
  const int nb = (d + TB - 1) / TB, ntiles = nb * (nb + 1) / 2;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = TI_THREADS / 32;
  const int rg = lane / RI, c0 = h * W + (lane % RI) * 4;
  pdl_launch();
  pdl_wait();
  // shared: Scol[K] (K <= J), R_IK at Rs[K (K - 1) / 2 + I] (I < K <= J),
  // diagonal inverses Ds[K] (K < J)
  float* Scol = sm;
  float* Rs = Scol + (size_t)nb * TILE_F;
  float* Ds = Rs + (size_t)nb * (nb - 1) / 2 * TILE_F;
  float* Ps = Ds + (size_t)nb * TILE_F;  // 4 partial products (k quarters)
  auto rtile = [&](int I, int K) { return tiles + (size_t)bidx(I, K, nb) * TB * TB; };
  auto dtile = [&](int K) { return tiles + (size_t)(ntiles + K) * TB * TB; };
  fetch_tile(Scol + (size_t)J * TILE_F, dtile(J), t, TI_THREADS);
  for (int K = 1; K <= J; ++K)
    for (int I = 0; I < K; ++I)
      fetch_tile(Rs + ((size_t)K * (K - 1) / 2 + I) * TILE_F, rtile(I, K), t, TI_THREADS);
  for (int K = 0; K < J; ++K) fetch_tile(Ds + (size_t)K * TILE_F, dtile(K), t, TI_THREADS);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int e = t; e < J * TB * TB; e += TI_THREADS) {  // acc_I = 0, I < J
    const int I = e >> 10, r = (e >> 5) & 31, c = e & 31;
    Scol[I * TILE_F + r * TP + c] = 0.f;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  for (int K = J; K >= 1; --K) {
    const float* SKJ = Scol + (size_t)K * TILE_F;
    // acc_I += R_IK S_KJ, one item per I (this CTA's strip)
    for (int u = warp; u < K; u += nw) {
      const int I = u;
      float* C = Scol + (size_t)I * TILE_F;
      float a4[RI][4];
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(C + (rg + RS * i) * TP + c0);
        a4[i][0] = v.x;
        a4[i][1] = v.y;
        a4[i][2] = v.z;
        a4[i][3] = v.w;
      }
      tile_strip<W>(Rs + ((size_t)K * (K - 1) / 2 + I) * TILE_F, SKJ, rg, c0, 0, TB, a4);
#pragma unroll
      for (int i = 0; i < RI; ++i)
        *reinterpret_cast<float4*>(C + (rg + RS * i) * TP + c0) =
            make_float4(a4[i][0], a4[i][1], a4[i][2], a4[i][3]);
    }
    __syncthreads();
    // S_{K-1,J} = -S_{K-1,K-1} acc_{K-1}, in place: warps (k quarter) form
    // partial products of this strip, then every thread adds the four
    // partials of two entries in quarter order
    float* D = Scol + (size_t)(K - 1) * TILE_F;
    if (warp < 4) {
      const int kq = warp;
      float o[RI][4] = {};
      tile_strip<W>(Ds + (size_t)(K - 1) * TILE_F, D, rg, c0, 8 * kq, 8 * kq + 8, o);
      float* Pq = Ps + (size_t)kq * TILE_F;
#pragma unroll
      for (int i = 0; i < RI; ++i)
        *reinterpret_cast<float4*>(Pq + (rg + RS * i) * TP + c0) =
            make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
    }
    __syncthreads();
    for (int e = t; e < TB * (W / 2); e += TI_THREADS) {
      const int r = e / (W / 2), c = h * W + (e % (W / 2)) * 2;
      float2 v = *reinterpret_cast<const float2*>(Ps + r * TP + c);
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        const float2 w = *reinterpret_cast<const float2*>(Ps + (size_t)q * TILE_F + r * TP + c);
        v.x += w.x;
        v.y += w.y;
      }
      *reinterpret_cast<float2*>(D + r * TP + c) = make_float2(-v.x, -v.y);
    }
    __syncthreads();
  }
  // St[p][n][k] = part p of S[k][n], n = 32 J + c: lane = k within a
  // 32-row block, so a warp writes 64 contiguous bytes per row n
  for (int e = warp; e < W * (KPX / TB); e += nw) {
    const int c = h * W + e / (KPX / TB), kb = e % (KPX / TB);
    const int n = J * TB + c, k = kb * TB + lane;
    if (n >= dp) continue;
    float v = 0.f;
    if (kb <= J && k < d && n < d) v = Scol[(size_t)kb * TILE_F + lane * TP + c];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
    const size_t o = (size_t)n * KPX + k;
    St[o] = h;
    St[(size_t)dp * KPX + o] = m;
    St[2 * (size_t)dp * KPX + o] = l;
  }
}

// grid = TI_STRIPS nb CTAs (block column J = blockIdx.x / TI_STRIPS, strip
// blockIdx.x % TI_STRIPS), S^T parts K-padded to 256.
__global__ void __launch_bounds__(TI_THREADS)
k_trinv(const float* __restrict__ tiles, int d, int dp, __nv_bfloat16* __restrict__ St) {
  extern __shared__ __align__(16) float sm[];
  trinv_body<KP>(tiles, d, dp, blockIdx.x / TI_STRIPS, blockIdx.x % TI_STRIPS, St, sm);
}

// Batched: grid (TI_STRIPS x block columns, items); item list[blockIdx.y] of the table,
// S^T parts K-padded to 128 in its St buffer.
__global__ void __launch_bounds__(TI_THREADS)
k_btrinv(const BMat* __restrict__ T, const int* __restrict__ list) {
  extern __shared__ __align__(16) float sm[];
  const BMat& b = T[list[blockIdx.y]];
  if ((int)(blockIdx.x / TI_STRIPS) >= (b.d + TB - 1) / TB) return;  // block-uniform
  trinv_body<KPB>(b.tiles, b.d, b.dp, blockIdx.x / TI_STRIPS, blockIdx.x % TI_STRIPS,
                  (__nv_bfloat16*)b.St, sm);
}

constexpr int QM_CONV = 8;                      // converter / epilogue warps
constexpr int QM_PROD = QM_CONV;                // TMA producer warp
constexpr int QM_MMA = QM_CONV + 1;             // MMA warp
constexpr int QM_THREADS = 32 * (QM_CONV + 2);
constexpr int QM_PER = 128 * 16 / (QM_CONV * 32);  // float4 of a chunk per thread
constexpr int QM_BM = 128;
constexpr uint32_t QM_APART = QM_BM * 128;       // A part: [128 rows][64 BF16], 16 KB
constexpr uint32_t QM_ASTAGE = 3 * QM_APART;     // 48 KB
constexpr uint32_t QM_BPART = 256 * 128;         // B part: [256 rows][64 BF16], 32 KB
constexpr uint32_t QM_BBOX = 64 * 128;           // one TMA box of a part: 64 rows, 8 KB
constexpr uint32_t QM_B = 3 * QM_BPART;          // 96 KB
constexpr int QM_SP = 20;                        // epilogue staging pitch (floats)
constexpr uint32_t QM_STG = QM_CONV * 32 * QM_SP * 4;  // 20 KB
constexpr uint32_t QM_BAR = 2 * QM_ASTAGE + QM_B + QM_STG;
constexpr size_t QM_SMEM = 1024 + (size_t)QM_BAR + 128;

struct QmParams {
  const float* Y;
  int64_t ldy;
  float* Q;
  int64_t ldq;
  __nv_bfloat16* Bt;   // optional Q^T (dp x ldbt)
  __nv_bfloat16* Btl;  // optional low part of Q^T (two-part products)
  int64_t ldbt;
  int64_t M;
  int64_t R;  // rows per CTA
  int gs;     // sub-tiles per group (1 or 2)
  int d, dp;
  int* err;
};

// Every CTA owns an equal range of ceil(M / CTAs) rows (so no CTA takes a
// second tile while the others idle), handled as groups of two 128-row
// sub-tiles that share each chunk's S load.  K chunk c (k in [64 c, 64 c +
// 64)) contributes to the output columns n >= 64 c only: per sub-tile one MMA
// chain of width N = dp - 64 c, whose S rows 64 c .. dp - 1 come in 64-row TMA
// boxes.  Warps 0..7 convert Y chunks into the two A stages (one per
// sub-tile) and drain the accumulators (the epilogue of group g - 1 runs
// after chunk 0 of group g is converted); warp 8 loads the S parts; warp 9
// issues the MMAs.  One TMEM accumulator per sub-tile (2 x 256 columns).
__global__ void __launch_bounds__(QM_THREADS, 1)
k_qmul_tc(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ QmParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t sB = base + 2 * QM_ASTAGE;
  float* stg_all = (float*)(base_ptr + 2 * QM_ASTAGE + QM_B);
  // barriers: a_full[2] (8 arrivals), a_empty[2] (MMA commit), b_full (TMA),
  // b_empty (MMA commit), acc_full[2] (MMA commit), acc_empty[2] (8
  // arrivals), drain
  const uint32_t bar = base + QM_BAR;
  auto a_full = [&](int s) { return bar + 8u * s; };
  auto a_empty = [&](int s) { return bar + 16u + 8u * s; };
  const uint32_t b_full = bar + 32, b_empty = bar + 40;
  auto acc_full = [&](int s) { return bar + 48u + 8u * s; };
  auto acc_empty = [&](int s) { return bar + 64u + 8u * s; };
  const uint32_t drain = bar + 80;
  uint32_t* tmem_slot = (uint32_t*)(base_ptr + QM_BAR + 96);
  __shared__ int s_abort;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    mbar_init(a_full(0), QM_CONV);
    mbar_init(a_full(1), QM_CONV);
    mbar_init(a_empty(0), 1);
    mbar_init(a_empty(1), 1);
    mbar_init(b_full, 1);
    mbar_init(b_empty, 1);
    mbar_init(acc_full(0), 1);
    mbar_init(acc_full(1), 1);
    mbar_init(acc_empty(0), QM_CONV);
    mbar_init(acc_empty(1), QM_CONV);
    mbar_init(drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmS) : "memory");
  }
  if (warp == QM_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  pdl_launch();
  pdl_wait();

  const int dp = p.dp, d = p.d;
  const int nsteps = (dp + 63) / 64;  // K chunks
  // this CTA's rows [r_begin, r_end), in groups of gs (1 or 2) 128-row
  // sub-tiles.  gs = 2: sub-tile s uses A stage s and accumulator s.  gs = 1:
  // the steps alternate between the A stages and the groups between the
  // accumulators, so the epilogue of a group overlaps the next one's MMAs.
  const int gs = p.gs;
  const int64_t r_begin = (int64_t)blockIdx.x * p.R;
  const int64_t r_end = min(p.M, r_begin + p.R);
  const int ngroups =
      r_end > r_begin ? (int)((r_end - r_begin + gs * QM_BM - 1) / (gs * QM_BM)) : 0;
  auto sub_row0 = [&](int g, int s) { return r_begin + (int64_t)(gs * g + s) * QM_BM; };
  auto nsub = [&](int g) { return gs == 2 && sub_row0(g, 1) < r_end ? 2 : 1; };
  // A stage of sub-tile s at step j and its use count before step j
  auto astage = [&](int j, int s) { return gs == 2 ? s : (j & 1); };
  auto ause = [&](int j) { return gs == 2 ? j : (j >> 1); };
  // accumulator of sub-tile s of group g and its use count before group g
  auto aset = [&](int g, int s) { return gs == 2 ? s : (g & 1); };
  auto acc_use = [&](int g) { return gs == 2 ? g : (g >> 1); };
  const int total = ngroups * nsteps;

  if (warp == QM_PROD) {
    // ---------------- TMA producer: S^T parts, rows 64 c .. dp - 1 ----------------
    if (lane == 0) {
      const uint64_t pol = policy_evict_last();
      bool pending = false;
      uint32_t pend_par = 0;
      for (int j = 0; j < total; ++j) {
        const int c = j % nsteps;
        const int nbox = (dp - 64 * c + 63) / 64;  // 64-row boxes per part
        if (j >= 1 && !mbar_wait(b_empty, (uint32_t)((j - 1) & 1), abort_flag)) {
          s_abort = 1;
          break;
        }
        mbar_expect_tx(b_full, 3u * (uint32_t)nbox * QM_BBOX);
        for (int q = 0; q < 3; ++q)
          for (int b = 0; b < nbox; ++b)
            tma_load_2d(sB + q * QM_BPART + b * QM_BBOX, &tmS, b_full, 64 * c,
                        q * dp + 64 * c + 64 * b, pol);
        pending = true;
        pend_par = (uint32_t)(j & 1);
      }
      volatile int never = 0;
      // the last copy must land before the CTA exits (the MMA warp waited for
      // the others)
      if (pending) mbar_wait(b_full, pend_par, &never);
    }
  } else if (warp == QM_MMA) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      bool ok = true;
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
      const uint64_t bd0 = sdesc(sB, 16, 1024);
      for (int g = 0; g < ngroups && ok; ++g) {
        const int ns = nsub(g), v = acc_use(g);
        // the accumulators were drained by the epilogue of their last group
        for (int s = 0; s < ns && v >= 1 && ok; ++s)
          ok = mbar_wait(acc_empty(aset(g, s)), (uint32_t)((v - 1) & 1), abort_flag);
        if (!ok) break;
        tc_fence_after();
        for (int c = 0; c < nsteps; ++c) {
          const int j = g * nsteps + c;
          if (!mbar_wait(b_full, (uint32_t)(j & 1), abort_flag)) {
            ok = false;
            break;
          }
          const int n = dp - 64 * c;
          const uint32_t id = idesc_bf16(n, false);
          for (int s = 0; s < ns; ++s) {
            const int st = astage(j, s), set = aset(g, s);
            if (!mbar_wait(a_full(st), (uint32_t)(ause(j) & 1), abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dcol = tmem_base + (uint32_t)(256 * set + 64 * c);
            const uint64_t ad0 = sdesc(base + st * QM_ASTAGE, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                const uint64_t ad = ad0 + (uint64_t)((pa[q] * QM_APART + kk * 32) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((pb[q] * QM_BPART + kk * 32) >> 4);
                mma_bf16(dcol, ad, bd, id, (c > 0 || kk > 0 || q > 0) ? 1u : 0u);
              }
            }
            mma_commit(a_empty(st));
            if (c == nsteps - 1) mma_commit(acc_full(set));
          }
          if (!ok) break;
          mma_commit(b_empty);
        }
      }
      if (!ok) s_abort = 1;
    }
  } else {
    // ---------------- converters + epilogue (warps 0..7) ----------------
    const int ct = t;  // 0..255
    // unit (g, c, s): sub-tile s of group g, columns 64 c .. 64 c + 63 of Y
    auto load_a = [&](int g, int c, int s, float4 (&x)[QM_PER]) {
      const int64_t r0 = sub_row0(g, s);
#pragma unroll
      for (int q = 0; q < QM_PER; ++q) {
        const int e = ct + q * QM_CONV * 32;
        const int row = e >> 4, k = c * 64 + (e & 15) * 4;
        x[q] = (r0 + row < r_end && k < d)
                   ? *reinterpret_cast<const float4*>(p.Y + (r0 + row) * p.ldy + k)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
        if (k + 3 >= d && k < d) {  // zero the columns past d
          if (k + 1 >= d) x[q].y = 0.f;
          if (k + 2 >= d) x[q].z = 0.f;
          if (k + 3 >= d) x[q].w = 0.f;
        }
      }
    };
    // the unit after (g, c, s) in issue order; false after the last
    auto next_unit = [&](int& g, int& c, int& s) {
      if (s == 0 && nsub(g) == 2) {
        s = 1;
        return true;
      }
      s = 0;
      if (++c == nsteps) {
        c = 0;
        if (++g == ngroups) return false;
      }
      return true;
    };
    bool ok = true;
    // one unit: wait for its A stage, start the next unit's loads into nxt,
    // convert cur into the stage, signal the MMA warp
    auto unit = [&](int g, int c, int s, float4 (&cur)[QM_PER], float4 (&nxt)[QM_PER]) {
      const int j = g * nsteps + c, st = astage(j, s), u = ause(j);
      const uint32_t stA = base + st * QM_ASTAGE;
      if (u >= 1 &&
          !__all_sync(0xffffffffu, mbar_wait(a_empty(st), (uint32_t)((u - 1) & 1), abort_flag))) {
        ok = false;
        return false;
      }
      int ng = g, nc = c, nsb = s;
      const bool more = next_unit(ng, nc, nsb);
      if (more) load_a(ng, nc, nsb, nxt);
      asm volatile("" ::: "memory");  // the loads are issued before the conversion
      // rows past the CTA's range are not converted: a row of the MMA's
      // output depends on the same row of A only, and those output rows are
      // never stored (a range of 132 rows leaves a 4-row second sub-tile)
      const int64_t r0s = sub_row0(g, s);
#pragma unroll
      for (int q = 0; q < QM_PER; ++q) {
        const int e = ct + q * QM_CONV * 32;
        const int row = e >> 4, kc = (e & 15) * 4;
        if (r0s + row >= r_end) continue;
        const float v[4] = {cur[q].x, cur[q].y, cur[q].z, cur[q].w};
        uint32_t hp[2], mp[2], lp[2];
        split3_bf16x4(v, hp, mp, lp);
        const uint32_t off = (uint32_t)row * 128 + ((uint32_t)((kc >> 3) ^ (row & 7)) << 4) +
                             (uint32_t)((kc & 7) * 2);
        const uint32_t a = stA + off;
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(hp[0]), "r"(hp[1])
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + QM_APART), "r"(mp[0]),
                     "r"(mp[1])
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + 2 * QM_APART), "r"(lp[0]),
                     "r"(lp[1])
                     : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(a_full(st));
      return more;
    };
    // drain the accumulators of group g: warp w reads TMEM lanes
    // 32 (w % 4) + lane (sub-tile rows) and columns 128 (w / 4) .. + 127,
    // stages 16 columns at a time and stores 64-byte row segments
    float* stg = stg_all + warp * 32 * QM_SP;
    auto epilogue = [&](int g) {
      const int h = warp >> 2, q4 = warp & 3;
      const int c1 = min(dp, 128 * h + 128);
      for (int s = 0; s < nsub(g); ++s) {
        const int set = aset(g, s);
        if (!__all_sync(0xffffffffu,
                        mbar_wait(acc_full(set), (uint32_t)(acc_use(g) & 1), abort_flag))) {
          ok = false;
          return;
        }
        tc_fence_after();
        const int64_t rbase = sub_row0(g, s) + q4 * 32;
        // (a warp whose 32 rows all lie past the range has nothing to store)
        for (int col = 128 * h; col < c1 && rbase < r_end; col += 16) {
          float v[16];
          tmem_ld16(tmem_base + (uint32_t)(256 * set + col) + ((uint32_t)(q4 * 32) << 16), v);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(stg + lane * QM_SP + 4 * u) =
                make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
          if (p.Bt != nullptr && rbase + lane < r_end) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const __nv_bfloat16 hv = __float2bfloat16_rn(v[u]);
              p.Bt[(int64_t)(col + u) * p.ldbt + rbase + lane] = hv;
              if (p.Btl != nullptr)
                p.Btl[(int64_t)(col + u) * p.ldbt + rbase + lane] =
                    __float2bfloat16_rn(v[u] - __bfloat162float(hv));
            }
          }
          __syncwarp();
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const int row = rr * 8 + (lane >> 2), c4 = lane & 3;
            if (rbase + row < r_end)
              *reinterpret_cast<float4*>(p.Q + (rbase + row) * p.ldq + col + 4 * c4) =
                  *reinterpret_cast<const float4*>(stg + row * QM_SP + 4 * c4);
          }
          __syncwarp();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty(set));
      }
    };
    if (ngroups > 0) {
      float4 x0[QM_PER], x1[QM_PER];
      load_a(0, 0, 0, x0);
      int g = 0, c = 0, s = 0;
      bool more = true;
      for (int u = 0; more && ok; ++u) {
        const int pg = g, pc = c, ps = s;
        more = (u & 1) ? unit(g, c, s, x1, x0) : unit(g, c, s, x0, x1);
        if (!ok) break;
        if (more) next_unit(g, c, s);
        // group pg - 1 is drained once chunk 0 of group pg is converted
        if (pc == 0 && pg > 0 && ps == nsub(pg) - 1) epilogue(pg - 1);
      }
      if (ok) epilogue(ngroups - 1);
    }
    if (!ok) s_abort = 1;
  }
  __syncthreads();
  if (warp == QM_MMA) {
    if (lane == 0) {
      volatile int never = 0;
      tc_fence_after();
      mma_commit(drain);  // every MMA this CTA issued has completed before TMEM is freed
      mbar_wait(drain, 0, &never);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base)
                 : "memory");
  }
  if (t == 0 && *abort_flag) atomicExch(p.err, 1);
}

}  // namespace

size_t qmul_st_bytes(int d) {
  const int dp = (d + 15) / 16 * 16;
  return (size_t)3 * dp * KP * sizeof(__nv_bfloat16);
}

bool qmul_supported(int64_t M, int d, int64_t ldy, const void* Y, int64_t ldq, const void* Q) {
  const int dp = (d + 15) / 16 * 16;
  return M >= 8192 && d >= 1 && dp <= 256 && ldy % 4 == 0 && ldq % 4 == 0 && ldy >= dp &&
         ldq >= dp && ((uintptr_t)Y & 15) == 0 && ((uintptr_t)Q & 15) == 0;
}

cudaError_t qmul_tc(const float* Y, int64_t ldy, const float* tiles, int64_t M, int d, void* St,
                    float* Q, int64_t ldq, void* Bt, int64_t ldbt, int* err, cudaStream_t st,
                    void* Btl) {
  if (!qmul_supported(M, d, ldy, Y, ldq, Q) || ((uintptr_t)St & 15) != 0)
    return cudaErrorInvalidValue;
  const int dp = (d + 15) / 16 * 16;
  const int nb = (d + TB - 1) / TB;
  const size_t ti_smem = (size_t)(nb + nb * (nb - 1) / 2 + nb + 4) * TILE_F * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ti_smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_trinv, dim3(TI_STRIPS * nb), dim3(TI_THREADS), ti_smem, st, tiles, d, dp,
                 (__nv_bfloat16*)St);
  count_launch();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  if (!make_map(&map, St, KP, (uint64_t)3 * dp, KP, 64, 64)) return cudaErrorInvalidValue;
  QmParams p;
  p.Y = Y;
  p.ldy = ldy;
  p.Q = Q;
  p.ldq = ldq;
  p.Bt = (__nv_bfloat16*)Bt;
  p.Btl = Bt != nullptr ? (__nv_bfloat16*)Btl : nullptr;
  p.ldbt = ldbt;
  p.M = M;
  p.d = d;
  p.dp = dp;
  p.err = err;
  e = cudaFuncSetAttribute(k_qmul_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QM_SMEM);
  if (e != cudaSuccess) return e;
  // equal row ranges, one per CTA (at most one per SM); up to 256 rows a
  // CTA's two sub-tiles share each S load, beyond that its 128-row sub-tiles
  // pipeline one after another
  p.R = (M + sm_count() - 1) / sm_count();
  p.gs = p.R <= 2 * QM_BM ? 2 : 1;
  const int P = (int)((M + p.R - 1) / p.R);
  e = launch_pdl(k_qmul_tc, dim3(P), dim3(QM_THREADS), QM_SMEM, st, map, p);
  count_launch();
  return e == cudaSuccess ? cudaGetLastError() : e;
}

size_t bo_st_bytes(int d) {
  const int dp = (d + 15) / 16 * 16;
  return (size_t)3 * dp * KPB * sizeof(__nv_bfloat16);
}

cudaError_t btrinv(const BMat* T, const int* list, int n, int dmax, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (dmax > KPB) return cudaErrorInvalidValue;
  const int nb = (dmax + TB - 1) / TB;
  const size_t smem = (size_t)(nb + nb * (nb - 1) / 2 + nb + 4) * TILE_F * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_btrinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_btrinv<<<dim3(TI_STRIPS * nb, n), TI_THREADS, smem, st>>>(T, list);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
