// Batched CholeskyQR passes on the tensor cores: orth() of Section II-A for
// the many small matrices of a batch at once.  Items whose padded width dp
// is at most BO_DPMAX (80) take these kernels; the slab reduction
// (k_bgram_reduce), the Cholesky factorisation (k_bchol) and the inverse
// S = R^{-1} (k_btrinv) are separate launches.
//
// Both kernels are persistent (one CTA per SM) over units: a row range of
// one item.  CTA c takes units uoff[c] .. uoff[c + 1] - 1, whose rows the
// host balanced over the CTAs.  Eight converter warps load 64- or 128-row
// chunks of the FP32 operand straight into registers, three (Gram) or one
// (Q) chunks ahead of the one they convert, split each value three ways into
// BF16 (h + m + l) and store the parts in 128B-swizzled stages; one MMA lane
// issues the six part products above 2^-24 (hh, hm, mh, mm, hl, lh) per
// 16-wide K step.
//
//  * k_bgram_tc: one unit = one row slab of gram_slabs() (the CUDA-core
//    Gram's slabs).  Per 64-row chunk, Y_c^T Y_c with M = 128 Gram rows and
//    N = dp (both operands MN-major), accumulated over the slab in one of two
//    TMEM accumulators; the converters drain a slab's sum at the start of the
//    next unit and store it as FP64 into the item's partial[slab], lower
//    triangle (row j >= column i, a lane per column i: coalesced).
//  * k_bqmul_tc: Q = Y S, 128-row sub-tiles, 64-wide K chunks (N = dp).  The
//    three BF16 parts of S^T are loaded into shared memory at each unit
//    start; the converters drain each finished sub-tile into Q (and
//    optionally Q^T in BF16, the next tensor-core product's operand).  A
//    sub-tile's rows are read in full before they are written, so Q may
//    overwrite Y.
// Every mbarrier wait is bounded; on timeout the CTA sets the error word,
// waits for its own MMAs, frees TMEM and returns.  An item's results depend
// on its shape only (slabs from gram_slabs; each row of Q independent of the
// unit split), so it gets the same bits alone and inside any batch.
#include <cuda.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace ruqlp {
namespace {

__device__ __forceinline__ int64_t item_rows(const BMat& b, int src) {
  return src == B_Y ? b.m : b.n;
}

// The three BF16 parts of four consecutive values into a 128B-swizzled
// stage: part 0 at shared address a, parts 1 and 2 part_stride further.
__device__ __forceinline__ void st_parts(uint32_t a, uint32_t part_stride, const float4& x) {
  const float v[4] = {x.x, x.y, x.z, x.w};
  uint32_t hp[2], mp[2], lp[2];
  split3_bf16x4(v, hp, mp, lp);
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(hp[0]), "r"(hp[1]) : "memory");
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + part_stride), "r"(mp[0]), "r"(mp[1])
               : "memory");
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + 2 * part_stride), "r"(lp[0]),
               "r"(lp[1])
               : "memory");
}

// Bounded wait on an mbarrier phase, as mbar_wait but inlined: the
// converters call it with their next chunks' loads in flight, and a call
// boundary there would make those loads complete first.  False on timeout
// or when another role of the CTA has already given up.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > WAIT_NS) return false;
    }
  }
}

// Position of a CTA in its unit range: unit index u (local), chunk k.
struct Cursor {
  int u, k;
};

// A 16-byte streaming load that does not allocate in L1 (the operand is read
// once; L1 keeps the CTA's other data).
__device__ __forceinline__ float4 ldg_stream(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Per-unit parameters, gathered into shared memory once per launch so the
// chunk loop reads no global metadata.
struct GDesc {      // Gram unit
  const float* Y;   // the unit's first row
  double* P;        // its slab's partial (d x d)
  int rows, d, dp, nch;
};
struct QDesc {      // Q = Y R^{-1} unit
  const float* Y;   // the unit's first row of the operand
  float* Q;         // ... and of the result
  __nv_bfloat16* Bt;   // Q^T (BF16) from the unit's first row, or null
  __nv_bfloat16* Btl;  // its low part, or null
  const __nv_bfloat16* St;
  int64_t ldbt;
  int rows, d, dp, nsub;
};

constexpr int BO_CONV = 8;                      // converter / drain warps
constexpr int BO_THREADS = 32 * (BO_CONV + 1);  // + the MMA warp
static_assert(BO_MAXU <= BO_THREADS, "one thread fills each unit descriptor");

// ============================ Gram =======================================
constexpr int BG_ROWS = 64;                     // rows per chunk (the MMAs' K)
constexpr uint32_t BG_BOX = BG_ROWS * 128;      // [64 rows][64 BF16], 8 KB
constexpr uint32_t BG_PART = 2 * BG_BOX;        // columns 0..127 of one part
constexpr uint32_t BG_STAGE = 3 * BG_PART;      // h, m, l: 48 KB
constexpr int BG_NST = 3;                       // ring depth
constexpr int BG_PER = (BG_ROWS * (BO_DPMAX / 4) + BO_CONV * 32 - 1) / (BO_CONV * 32);
constexpr uint32_t BG_BAR = BG_NST * BG_STAGE;
constexpr int BG_NBAR = 2 * BG_NST + 3;  // full, empty, acc_full[2], drain
constexpr size_t BG_SMEM = 1024 + BG_BAR + 8 * BG_NBAR + 16;
constexpr uint32_t BG_TMEM_COLS = 256;  // two accumulators of 128 columns

__global__ void __launch_bounds__(BO_THREADS, 1)
k_bgram_tc(const BMat* __restrict__ T, const BoUnit* __restrict__ units,
           const int* __restrict__ uoff, int src, int max_slabs, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t bar = base + BG_BAR;
  auto full = [&](uint32_t s) { return bar + 8u * s; };
  auto empty = [&](uint32_t s) { return bar + 8u * (BG_NST + s); };
  auto accf = [&](uint32_t s) { return bar + 8u * (2 * BG_NST + s); };
  const uint32_t drain = bar + 8u * (2 * BG_NST + 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + BG_BAR + 8 * BG_NBAR);
  __shared__ int s_abort;
  __shared__ GDesc ud[BO_MAXU];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ub = uoff[blockIdx.x];
  const int nu = min(uoff[blockIdx.x + 1] - ub, BO_MAXU);  // (the host keeps it <= BO_MAXU)
  if (t < nu) {
    const BoUnit un = units[ub + t];
    const BMat& b = T[un.item];
    int64_t slab;
    gram_slabs(item_rows(b, src), max_slabs, &slab);
    GDesc g;
    g.Y = bbuf(b, src) + un.row0 * b.dp;
    g.P = b.partial + (un.row0 / slab) * (int64_t)b.d * b.d;
    g.rows = un.rows;
    g.d = b.d;
    g.dp = b.dp;
    g.nch = (un.rows + BG_ROWS - 1) / BG_ROWS;
    ud[t] = g;
  }
  if (t == 0) {
    for (int s = 0; s < BG_NST; ++s) {
      mbar_init(full(s), BO_CONV);
      mbar_init(empty(s), 1);
    }
    mbar_init(accf(0), 1);
    mbar_init(accf(1), 1);
    mbar_init(drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // The stages start at zero: the A operand spans columns 0..127 and a
  // narrow item leaves the columns past its dp unwritten (they only reach
  // Gram rows that are never read, but stay finite).
  for (uint32_t o = (uint32_t)t * 16; o < BG_NST * BG_STAGE; o += BO_THREADS * 16)
    *reinterpret_cast<uint4*>(base_ptr + o) = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == BO_CONV) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "n"(BG_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  bool ok = true;

  if (warp == BO_CONV) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
      uint32_t gi = 0;  // chunks issued by this CTA
      for (int u = 0; u < nu && ok; ++u) {
        const int dp = ud[u].dp;
        // kind::f16, BF16 x BF16 -> FP32, A and B MN-major, M = 128, N = dp
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(dp >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const uint32_t set = (uint32_t)u & 1u;
        const int nch = ud[u].nch;
        for (int k = 0; k < nch; ++k) {
          const uint32_t st = gi % BG_NST;
          if (!wait_bar(full(st), (gi / BG_NST) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t stage = base + st * BG_STAGE;
#pragma unroll
          for (int kk = 0; kk < BG_ROWS / 16; ++kk) {
            const uint64_t d0 = sdesc(stage + kk * 2048, BG_BOX, 1024);
#pragma unroll
            for (int q = 0; q < 6; ++q)
              mma_bf16(tmem_base + set * 128u, d0 + (uint64_t)((pa[q] * BG_PART) >> 4),
                       d0 + (uint64_t)((pb[q] * BG_PART) >> 4), idesc,
                       (k > 0 || kk > 0 || q > 0) ? 1u : 0u);
          }
          mma_commit(empty(st));
          ++gi;
        }
        if (!ok) break;
        mma_commit(accf(set));
      }
      if (!ok) s_abort = 1;
    }
  } else {
    // ---------------- converters (warps 0..7) ----------------
    const int ct = t;  // 0..255
    auto advance = [&](Cursor& c) {
      if (c.u >= nu) return;
      if (++c.k == ud[c.u].nch) {
        c.k = 0;
        ++c.u;
      }
    };
    auto load = [&](const Cursor& c, float4 (&x)[BG_PER]) {
      if (c.u >= nu) return;
      const GDesc& g = ud[c.u];
      const int r0 = c.k * BG_ROWS;
      const int d = g.d, dp = g.dp, w4 = dp >> 2;
#pragma unroll
      for (int q = 0; q < BG_PER; ++q) {
        const int e = ct + q * BO_CONV * 32;
        const int row = e / w4, c4 = (e - row * w4) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < BG_ROWS && r0 + row < g.rows && c4 < d) {
          v = ldg_stream(g.Y + (int64_t)(r0 + row) * dp + c4);
          if (c4 + 3 >= d) {  // zero the columns past d
            if (c4 + 1 >= d) v.y = 0.f;
            if (c4 + 2 >= d) v.z = 0.f;
            v.w = 0.f;
          }
        }
        x[q] = v;
      }
    };
    // the slab sum of unit u (accumulator u & 1) into the item's
    // partial[slab]: warp w reads Gram rows 32 (w % 4) + lane, 16-column
    // groups c0 = 16 (w / 4) + 32 i, and writes entries (j, i) with
    // i <= j < d at partial[slab][j][i] (lanes: consecutive i)
    const int q4 = warp & 3, h2 = warp >> 2;
    const int i_row = 32 * q4 + lane;
    auto drain_unit = [&](int u) -> bool {
      const uint32_t set = (uint32_t)u & 1u, use = (uint32_t)u >> 1;
      if (!__all_sync(0xffffffffu, wait_bar(accf(set), use & 1u, abort_flag))) return false;
      tc_fence_after();
      const int d = ud[u].d, dp = ud[u].dp;
      double* P = ud[u].P;
      if (32 * q4 < dp) {  // warp-uniform
        for (int c0 = 16 * h2; c0 < dp; c0 += 32) {
          float v[16];
          tmem_ld16(tmem_base + set * 128u + (uint32_t)c0 + ((uint32_t)(32 * q4) << 16), v);
#pragma unroll
          for (int w = 0; w < 16; ++w) {
            const int j = c0 + w;
            if (i_row <= j && j < d) P[(int64_t)j * d + i_row] = (double)v[w];
          }
        }
      }
      tc_fence_before();
      return true;
    };
    uint32_t gi = 0;  // chunks converted
    Cursor cur{0, 0}, ahead{0, 0};
    // one chunk: start the loads of the chunk three ahead (into the buffer
    // the previous step converted), wait for the stage, drain the previous
    // unit's sum when this chunk begins a unit, convert, signal
    auto step = [&](float4 (&xc)[BG_PER], float4 (&xl)[BG_PER]) {
      load(ahead, xl);
      advance(ahead);
      asm volatile("" ::: "memory");  // the loads are issued before the waits
      const uint32_t st = gi % BG_NST;
      if (gi >= BG_NST &&
          !__all_sync(0xffffffffu, wait_bar(empty(st), ((gi / BG_NST) - 1) & 1u, abort_flag))) {
        ok = false;
        return;
      }
      if (cur.k == 0 && cur.u > 0 && !drain_unit(cur.u - 1)) {
        ok = false;
        return;
      }
      const int w4 = ud[cur.u].dp >> 2;
      const uint32_t stage = base + st * BG_STAGE;
#pragma unroll
      for (int q = 0; q < BG_PER; ++q) {
        const int e = ct + q * BO_CONV * 32;
        const int row = e / w4, c4 = (e - row * w4) * 4;
        if (row >= BG_ROWS) continue;
        const int box = c4 >> 6, cb = c4 & 63;
        const uint32_t off = (uint32_t)box * BG_BOX + (uint32_t)row * 128 +
                             ((uint32_t)((cb >> 3) ^ (row & 7)) << 4) + (uint32_t)((cb & 7) * 2);
        st_parts(stage + off, BG_PART, xc[q]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(full(st));
      ++gi;
      advance(cur);
    };
    float4 x0[BG_PER], x1[BG_PER], x2[BG_PER], x3[BG_PER];
    load(ahead, x0);
    advance(ahead);
    load(ahead, x1);
    advance(ahead);
    load(ahead, x2);
    advance(ahead);
    while (ok && cur.u < nu) {
      step(x0, x3);
      if (!ok || cur.u >= nu) break;
      step(x1, x0);
      if (!ok || cur.u >= nu) break;
      step(x2, x1);
      if (!ok || cur.u >= nu) break;
      step(x3, x2);
    }
    if (ok && nu > 0 && !drain_unit(nu - 1)) ok = false;
    if (!ok) s_abort = 1;
  }
  __syncthreads();
  if (warp == BO_CONV) {
    if (lane == 0) {  // every MMA this CTA issued has completed before TMEM is freed
      volatile int never = 0;
      tc_fence_after();
      mma_commit(drain);
      mbar_wait(drain, 0, &never);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "n"(BG_TMEM_COLS)
                 : "memory");
  }
  if (t == 0 && *abort_flag) atomicExch(err, 1);
}

// ========================= Q = Y R^{-1} ===================================
constexpr int BQ_BM = 128;                           // rows of a sub-tile
constexpr int BQ_PER = BQ_BM * 16 / (BO_CONV * 32);  // float4 of a chunk per thread
constexpr uint32_t BQ_APART = BQ_BM * 128;           // A part: [128 rows][64 BF16], 16 KB
constexpr uint32_t BQ_ASTAGE = 3 * BQ_APART;         // 48 KB
constexpr uint32_t BQ_SBOX = BO_DPMAX * 128;         // S part, one K box: [80 n][64 k]
constexpr uint32_t BQ_S_OFF = 2 * BQ_ASTAGE;
constexpr uint32_t BQ_S = 3 * 2 * BQ_SBOX;           // parts x K boxes, 60 KB
constexpr int BQ_SP = 20;                            // epilogue staging pitch (floats)
constexpr uint32_t BQ_STG_OFF = BQ_S_OFF + BQ_S;
constexpr uint32_t BQ_STG = BO_CONV * 32 * BQ_SP * 4;
constexpr uint32_t BQ_BAR = BQ_STG_OFF + BQ_STG;
constexpr int BQ_NBAR = 9;  // a_full[2], a_empty[2], acc_full[2], acc_empty[2], drain
constexpr size_t BQ_SMEM = 1024 + BQ_BAR + 8 * BQ_NBAR + 16;
constexpr uint32_t BQ_TMEM_COLS = 256;

__global__ void __launch_bounds__(BO_THREADS, 1)
k_bqmul_tc(const BMat* __restrict__ T, const BoUnit* __restrict__ units,
           const int* __restrict__ uoff, int src, int dst, int make_bt, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  float* stg_all = reinterpret_cast<float*>(base_ptr + BQ_STG_OFF);
  const uint32_t bar = base + BQ_BAR;
  auto a_full = [&](uint32_t s) { return bar + 8u * s; };
  auto a_empty = [&](uint32_t s) { return bar + 16u + 8u * s; };
  auto acc_full = [&](uint32_t s) { return bar + 32u + 8u * s; };
  auto acc_empty = [&](uint32_t s) { return bar + 48u + 8u * s; };
  const uint32_t drain = bar + 64;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + BQ_BAR + 8 * BQ_NBAR);
  __shared__ int s_abort;
  __shared__ QDesc ud[BO_MAXU];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ub = uoff[blockIdx.x];
  const int nu = min(uoff[blockIdx.x + 1] - ub, BO_MAXU);  // (the host keeps it <= BO_MAXU)
  if (t < nu) {
    const BoUnit un = units[ub + t];
    const BMat& b = T[un.item];
    QDesc q;
    q.Y = bbuf(b, src) + un.row0 * b.dp;
    q.Q = bbuf(b, dst) + un.row0 * b.dp;
    q.Bt = (make_bt && b.use_tc) ? (__nv_bfloat16*)b.Bt + un.row0 : nullptr;
    q.Btl = (make_bt == 2 && b.use_tc) ? (__nv_bfloat16*)b.Btl + un.row0 : nullptr;
    q.St = (const __nv_bfloat16*)b.St;
    q.ldbt = b.ldbt;
    q.rows = un.rows;
    q.d = b.d;
    q.dp = b.dp;
    q.nsub = (un.rows + BQ_BM - 1) / BQ_BM;
    ud[t] = q;
  }
  if (t == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(a_full(s), BO_CONV);
      mbar_init(a_empty(s), 1);
      mbar_init(acc_full(s), 1);
      mbar_init(acc_empty(s), BO_CONV);
    }
    mbar_init(drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == BO_CONV) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "n"(BQ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  bool ok = true;
  auto nsteps = [&](int dp) { return (dp + 63) / 64; };
  // chunks of a unit: (sub-tile g, K chunk c) for k = g * nsteps + c
  auto nchunks = [&](int u) { return ud[u].nsub * nsteps(ud[u].dp); };

  if (warp == BO_CONV) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
      uint32_t j = 0, gt = 0;  // chunks and sub-tiles issued by this CTA
      for (int u = 0; u < nu && ok; ++u) {
        const int dp = ud[u].dp, ns = nsteps(dp), nsb = ud[u].nsub;
        const uint32_t id = idesc_bf16(dp, false);
        for (int g = 0; g < nsb && ok; ++g) {
          const uint32_t set = gt & 1u, v = gt >> 1;
          // the accumulator was drained by the epilogue of its last sub-tile
          if (v >= 1 && !wait_bar(acc_empty(set), (v - 1) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int c = 0; c < ns; ++c) {
            const uint32_t st = j & 1u;
            if (!wait_bar(a_full(st), (j >> 1) & 1u, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const int kw = min(64, dp - 64 * c);
            const uint64_t ad0 = sdesc(base + st * BQ_ASTAGE, 16, 1024);
            for (int kk = 0; kk < kw / 16; ++kk) {
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                const uint64_t ad = ad0 + (uint64_t)((pa[q] * BQ_APART + kk * 32) >> 4);
                const uint64_t bd =
                    sdesc(base + BQ_S_OFF + (uint32_t)(pb[q] * 2 + c) * BQ_SBOX, 16, 1024) +
                    (uint64_t)((kk * 32) >> 4);
                mma_bf16(tmem_base + set * 128u, ad, bd, id, (c > 0 || kk > 0 || q > 0) ? 1u : 0u);
              }
            }
            mma_commit(a_empty(st));
            ++j;
          }
          if (!ok) break;
          mma_commit(acc_full(set));
          ++gt;
        }
      }
      if (!ok) s_abort = 1;
    }
  } else {
    // ---------------- converters + epilogue (warps 0..7) ----------------
    const int ct = t;  // 0..255
    auto advance = [&](Cursor& c) {
      if (c.u >= nu) return;
      if (++c.k == nchunks(c.u)) {
        c.k = 0;
        ++c.u;
      }
    };
    auto load = [&](const Cursor& c, float4 (&x)[BQ_PER]) {
      if (c.u >= nu) return;
      const QDesc& qd = ud[c.u];
      const int d = qd.d, dp = qd.dp;
      const int ns = nsteps(dp), g = c.k / ns, cc = c.k - g * ns;
      const int r0 = g * BQ_BM;
#pragma unroll
      for (int q = 0; q < BQ_PER; ++q) {
        const int e = ct + q * BO_CONV * 32;
        const int row = e >> 4, k = cc * 64 + (e & 15) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + row < qd.rows && k < d) {
          v = ldg_stream(qd.Y + (int64_t)(r0 + row) * dp + k);
          if (k + 3 >= d) {  // zero the columns past d
            if (k + 1 >= d) v.y = 0.f;
            if (k + 2 >= d) v.z = 0.f;
            v.w = 0.f;
          }
        }
        x[q] = v;
      }
    };
    auto load_s = [&](const QDesc& qd) {
      const int dp = qd.dp, per_row = nsteps(dp) * 8;  // 16-byte pieces of a row n
      const __nv_bfloat16* St = qd.St;
      const int total = 3 * dp * per_row;
      for (int e = ct; e < total; e += BO_CONV * 32) {
        const int p = e / (dp * per_row);
        const int r = e - p * dp * per_row;
        const int nr = r / per_row, q = r - nr * per_row;
        const int kb = q >> 3, c16 = q & 7;
        const uint4 v = *reinterpret_cast<const uint4*>(St + ((size_t)(p * dp + nr) * BO_KP +
                                                              kb * 64 + c16 * 8));
        const uint32_t a = base + BQ_S_OFF + (uint32_t)(p * 2 + kb) * BQ_SBOX + (uint32_t)nr * 128 +
                           ((uint32_t)(c16 ^ (nr & 7)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y),
                     "r"(v.z), "r"(v.w)
                     : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    // drain sub-tile g of unit u (accumulator use gt): warp w reads TMEM lanes
    // 32 (w % 4) + lane and the 16-column groups 16 (w / 4) + 32 i, stages
    // them and stores 64-byte row segments of Q
    float* stg = stg_all + warp * 32 * BQ_SP;
    auto epilogue = [&](int u, int g, uint32_t gtp) -> bool {
      const QDesc& qd = ud[u];
      const uint32_t set = gtp & 1u;
      if (!__all_sync(0xffffffffu, wait_bar(acc_full(set), (gtp >> 1) & 1u, abort_flag)))
        return false;
      tc_fence_after();
      const int h = warp >> 2, q4 = warp & 3, dp = qd.dp;
      const int r_end = qd.rows;
      const int rbase = g * BQ_BM + q4 * 32;  // rows relative to the unit's first
      float* Q = qd.Q;
      __nv_bfloat16* Bt = qd.Bt;
      __nv_bfloat16* Btl = qd.Btl;
      const int64_t ldbt = qd.ldbt;
      for (int col = 16 * h; col < dp; col += 32) {
        float v[16];
        tmem_ld16(tmem_base + set * 128u + (uint32_t)col + ((uint32_t)(q4 * 32) << 16), v);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          *reinterpret_cast<float4*>(stg + lane * BQ_SP + 4 * w) =
              make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
        if (Bt != nullptr && rbase + lane < r_end) {
#pragma unroll
          for (int w = 0; w < 16; ++w) {
            const __nv_bfloat16 hv = __float2bfloat16_rn(v[w]);
            Bt[(int64_t)(col + w) * ldbt + rbase + lane] = hv;
            if (Btl != nullptr)
              Btl[(int64_t)(col + w) * ldbt + rbase + lane] =
                  __float2bfloat16_rn(v[w] - __bfloat162float(hv));
          }
        }
        __syncwarp();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const int row = rr * 8 + (lane >> 2), c4 = lane & 3;
          if (rbase + row < r_end)
            *reinterpret_cast<float4*>(Q + (int64_t)(rbase + row) * dp + col + 4 * c4) =
                *reinterpret_cast<const float4*>(stg + row * BQ_SP + 4 * c4);
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(set));
      return true;
    };
    uint32_t j = 0, gt = 0;  // chunks converted; sub-tiles begun
    bool pend = false;       // a sub-tile waiting for its epilogue
    int pu = 0, pg = 0;
    uint32_t pgt = 0;
    Cursor cur{0, 0}, ahead{0, 0};
    auto step = [&](float4 (&xc)[BQ_PER], float4 (&xl)[BQ_PER]) {
      load(ahead, xl);
      advance(ahead);
      asm volatile("" ::: "memory");  // the loads are issued before the waits
      const int ns = nsteps(ud[cur.u].dp), g = cur.k / ns, c = cur.k - g * ns;
      if (cur.k == 0) {
        // a new unit: this warp drains the last sub-tile of the previous one
        // (its wait on acc_full shows that every MMA reading S has completed)
        // and writes its share of the new S; the MMA warp reads S only after
        // a_full has all eight warps' arrivals for the unit's first chunk
        if (pend) {
          if (!epilogue(pu, pg, pgt)) {
            ok = false;
            return;
          }
          pend = false;
        }
        load_s(ud[cur.u]);
      }
      const uint32_t st = j & 1u, use = j >> 1;
      if (use >= 1 &&
          !__all_sync(0xffffffffu, wait_bar(a_empty(st), (use - 1) & 1u, abort_flag))) {
        ok = false;
        return;
      }
      const uint32_t stA = base + st * BQ_ASTAGE;
#pragma unroll
      for (int q = 0; q < BQ_PER; ++q) {
        const int e = ct + q * BO_CONV * 32;
        const int row = e >> 4, kc = (e & 15) * 4;
        const uint32_t off = (uint32_t)row * 128 + ((uint32_t)((kc >> 3) ^ (row & 7)) << 4) +
                             (uint32_t)((kc & 7) * 2);
        st_parts(stA + off, BQ_APART, xc[q]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(a_full(st));
      ++j;
      if (c == 0) {
        // chunk 0 of this sub-tile is in: drain the previous sub-tile
        if (pend && !epilogue(pu, pg, pgt)) {
          ok = false;
          return;
        }
        pend = true;
        pu = cur.u;
        pg = g;
        pgt = gt++;
      }
      advance(cur);
    };
    // (two 32 KB register buffers here: nine warps leave 168 registers a
    // thread, three on one scheduler; one chunk in flight while one converts)
    float4 x0[BQ_PER], x1[BQ_PER];
    load(ahead, x0);
    advance(ahead);
    while (ok && cur.u < nu) {
      step(x0, x1);
      if (!ok || cur.u >= nu) break;
      step(x1, x0);
    }
    if (ok && pend && !epilogue(pu, pg, pgt)) ok = false;
    if (!ok) s_abort = 1;
  }
  __syncthreads();
  if (warp == BO_CONV) {
    if (lane == 0) {
      volatile int never = 0;
      tc_fence_after();
      mma_commit(drain);  // every MMA this CTA issued has completed before TMEM is freed
      mbar_wait(drain, 0, &never);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "n"(BQ_TMEM_COLS)
                 : "memory");
  }
  if (t == 0 && *abort_flag) atomicExch(err, 1);
}

}  // namespace

cudaError_t bgram_tc(const BMat* T, const BoUnit* units, const int* uoff, int grid, int src,
                     int max_slabs, int* err, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_bgram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BG_SMEM);
  if (e != cudaSuccess) return e;
  k_bgram_tc<<<grid, BO_THREADS, BG_SMEM, st>>>(T, units, uoff, src, max_slabs, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t bqmul_tc(const BMat* T, const BoUnit* units, const int* uoff, int grid, int src,
                     int dst, int make_bt, int* err, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_bqmul_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BQ_SMEM);
  if (e != cudaSuccess) return e;
  k_bqmul_tc<<<grid, BO_THREADS, BQ_SMEM, st>>>(T, units, uoff, src, dst, make_bt, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
