// Tensor-core sketch products of RU-QLP on sm_103a (Section III-D: the
// O(mnd) products A X and A^T Y that make up the 2q+2 passes over A):
//
//   Y[m x dp] = A[m x n] X        (A K-major;   "NT" below)
//   Z[n x dp] = A^T[n x m] Y      (A MN-major;  "TN" below)
//
// A is BF16 row-major; the skinny operand is given transposed, Bt[dp x K]
// (BF16, K contiguous), so it is always the K-major B operand.  Outputs are
// FP32 (accumulated in TMEM).
//
// Structure (one CTA per SM, 192 threads):
//   warp 0  : TMA producer (one lane) -- A tile 128 x 64 and Bt tile dp x 64
//             per stage into a 128B-swizzled shared-memory ring;
//   warp 1  : TMEM allocation + tcgen05.mma issue (one lane), M=128, N=dp,
//             K=16 per instruction, two TMEM accumulators (ping-pong);
//   warps 2-5: epilogue -- tcgen05.ld of the accumulator, FP32 stores.
// Work split: output tiles of 128 rows are dealt to the CTAs in whole waves
// (data parallel); the tiles of the last partial wave are split over all
// CTAs along K (stream-K) into FP32 fragments, summed afterwards in CTA
// order by a fix-up kernel (deterministic; no atomics).  With a column split
// ns > 1 every 128-row tile is ns items of dp / ns output columns, dealt to
// consecutive CTAs: they stream the same A tile at the same time (the
// second read comes from L2), and each stage holds only a dp / ns slice of
// the skinny operand, so the ring is deeper and more of A is in flight per
// SM (the product is HBM-latency bound: bytes in flight / latency).  ns and
// the ring depth per shape come from a measured tuner (tc_gemm below).
// Every mbarrier wait is bounded (~2 s of %globaltimer); on timeout the CTA
// sets an error word, stops issuing work, and frees its TMEM before exiting.
#include <algorithm>
#include <array>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <map>
#include <mutex>
#include <stdio.h>
#include <string.h>
#include <string>

#include "internal.h"
#include "tcgen05.cuh"

namespace ruqlp {
namespace {

constexpr int BM = 128;       // rows of an output tile (MMA M)
constexpr int BK = 64;        // K per stage (one 128-byte swizzle row of BF16)
constexpr int NTHREADS = 192;
constexpr int A_TILE_BYTES = BM * BK * 2;  // 16 KB
constexpr int kBatchMaps = 4;              // tensor maps per batched matrix

struct TcParams {
  int64_t Mout;   // output rows
  int64_t K;      // contraction length
  int dp;         // output columns (multiple of 16, <= 256)
  int ns, dpi;    // column split: items of dpi = dp / ns columns (MMA N)
  int stages;
  float* out;
  int64_t ldo;
  float* frag;    // [P][2][BM][dpi]
  int T, KB, full_waves, tail;
  int64_t U;      // stream-K units = tail * KB
  int* err;
  int withhold;   // test hook: CTA 0 never loads its first stage (its waits run out)
};

// A CTA's work, generated on the fly: items 0..full_waves-1 are whole tiles
// (data parallel), then at most two stream-K segments of tail tiles.
struct Item {
  int tile, kb0, kb1, slot;  // slot < 0: write the output; else fragment slot
};

__device__ __forceinline__ int64_t sk_start(int64_t c, int64_t U, int P) { return c * U / P; }

__device__ __forceinline__ int item_count(const TcParams& p) {
  const int P = gridDim.x, c = blockIdx.x;
  int n = p.full_waves;
  if (p.tail > 0) {
    const int64_t u0 = sk_start(c, p.U, P), u1 = sk_start(c + 1, p.U, P);
    if (u1 > u0) n += (u1 > (u0 / p.KB + 1) * (int64_t)p.KB) ? 2 : 1;
  }
  return n;
}

__device__ __forceinline__ Item get_item(const TcParams& p, int i) {
  const int P = gridDim.x, c = blockIdx.x;
  if (i < p.full_waves) return {c + i * P, 0, p.KB, -1};
  const int64_t u0 = sk_start(c, p.U, P), u1 = sk_start(c + 1, p.U, P);
  const int base = p.full_waves * P;
  const int64_t t0 = u0 / p.KB;
  const int64_t e0 = min(u1, (t0 + 1) * (int64_t)p.KB);
  if (i == p.full_waves) return {base + (int)t0, (int)(u0 - t0 * p.KB), (int)(e0 - t0 * p.KB), 0};
  return {base + (int)t0 + 1, 0, (int)(u1 - (t0 + 1) * p.KB), 1};
}

// One unit of work of a CTA: an output tile of 128 rows, K blocks [kb0, kb1),
// written to out (rows < rows_valid) with leading dimension ldo.
struct TcItem {
  const CUtensorMap* mA;
  const CUtensorMap* mB;
  const CUtensorMap* mB2;  // low BF16 part of the skinny operand (two-part products)
  int tile, kb0, kb1, dp;  // 128-row tile, K blocks, output columns (MMA N)
  int bcol;                // first output column (row of the skinny operand Bt)
  float* out;
  int64_t ldo, rows;
  bool a_split;  // K-major A loaded as two 64-row boxes (batched maps)
};

// Single-matrix work: whole tiles, then stream-K segments (fragments).
struct WorkSingle {
  const CUtensorMap* mA;
  const CUtensorMap* mB;
  const CUtensorMap* mB2;
  const TcParams* p;
  static constexpr bool kGlobalMaps = false;
  __device__ int count() const { return item_count(*p); }
  __device__ TcItem get(int i) const {
    const Item it = get_item(*p, i);
    const int mt = it.tile / p->ns, h = it.tile - mt * p->ns;
    TcItem r{mA, mB, mB2, mt, it.kb0, it.kb1, p->dpi, h * p->dpi, nullptr, 0, 0, false};
    if (it.slot < 0) {
      r.out = p->out + (int64_t)mt * BM * p->ldo + r.bcol;
      r.ldo = p->ldo;
      r.rows = p->Mout - (int64_t)mt * BM;
    } else {
      r.out = p->frag + ((int64_t)blockIdx.x * 2 + it.slot) * BM * p->dpi;
      r.ldo = p->dpi;
      r.rows = BM;
    }
    return r;
  }
};

// Batched work: CTA c takes tiles c, c + P, c + 2P, ... of a host-built list
// (whole tiles only, so every tile is one K-ordered accumulation whichever CTA
// runs it).  Tensor maps live in global memory, kBatchMaps per matrix: A
// (64 x 64 boxes), Bt over n (for A X), Bt over m (for A^T Y) and the low
// part Btl over m (the two-part B^T = A^T Q).
struct WorkBatch {
  const BTcTile* list;
  int n;
  const BMat* T;
  const CUtensorMap* maps;
  int dst;
  bool trans;
  static constexpr bool kGlobalMaps = true;
  __device__ int count() const {
    return (int)blockIdx.x < n ? (n - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  }
  __device__ TcItem get(int i) const {
    const BTcTile w = list[blockIdx.x + (int64_t)i * gridDim.x];
    const BMat& b = T[w.mat];
    const int64_t K = trans ? b.m : b.n, Mout = trans ? b.n : b.m;
    TcItem r;
    r.mA = maps + kBatchMaps * (int64_t)w.mat;
    r.mB = maps + kBatchMaps * (int64_t)w.mat + (trans ? 2 : 1);
    r.mB2 = maps + kBatchMaps * (int64_t)w.mat + 3;
    r.tile = w.tile;
    r.kb0 = 0;
    r.kb1 = (int)((K + BK - 1) / BK);
    r.dp = b.dp;
    r.bcol = 0;
    r.out = bbuf(b, dst) + (int64_t)w.tile * BM * b.dp;
    r.ldo = b.dp;
    r.rows = Mout - (int64_t)w.tile * BM;
    r.a_split = true;
    return r;
  }
};

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m)
               : "memory");
}

// The warp-specialised pipeline shared by both kernels.  dpmax sizes the
// shared-memory stages; each item's own dp sets its B bytes and MMA N.
// B2: the skinny operand comes in two BF16 parts, b = h + l (l = bf16(b - h),
// so h + l carries about 16 significant bits of the FP32 value); each stage
// holds both parts' tiles and every A tile is multiplied by both into the same
// accumulator, D += A h + A l.
template <bool TRANS, bool B2, class W>
__device__ __forceinline__ void tc_body(const W& w, int* err, int S, int dpmax,
                                        int withhold = 0) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t b_tile = (uint32_t)dpmax * BK * 2;  // a multiple of 1024 bytes
  const uint32_t stage_bytes = A_TILE_BYTES + (B2 ? 2u : 1u) * b_tile;
  const uint32_t bar_base = base + S * stage_bytes;
  // barriers: full[S], empty[S], tfull[2], tempty[2], drain; then the TMEM address
  auto full_bar = [&](int s) { return bar_base + 8u * s; };
  auto empty_bar = [&](int s) { return bar_base + 8u * (S + s); };
  auto tfull_bar = [&](int a) { return bar_base + 8u * (2 * S + a); };
  auto tempty_bar = [&](int a) { return bar_base + 8u * (2 * S + 2 + a); };
  const uint32_t drain_bar = bar_base + 8u * (2 * S + 4);
  uint32_t* tmem_slot = (uint32_t*)(base_ptr + S * stage_bytes + 8 * (2 * S + 5));
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = w.count();
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 4);  // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!W::kGlobalMaps && nitems > 0) {
      const TcItem it = w.get(0);
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)it.mA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)it.mB) : "memory");
      if (B2) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)it.mB2) : "memory");
    }
  }
  if (warp == 1) {
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

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint64_t pol_a = policy_evict_first(), pol_b = policy_evict_last();
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int64_t issued = 0;
      const CUtensorMap* last_a = nullptr;
      for (int i = 0; i < nitems && ok; ++i) {
        const TcItem it = w.get(i);
        if (W::kGlobalMaps && it.mA != last_a) {  // maps written before the launch
          tmap_acquire(it.mA);
          tmap_acquire(it.mB);
          if (B2) tmap_acquire(it.mB2);
          last_a = it.mA;
        }
        const uint32_t bytes = A_TILE_BYTES + (B2 ? 2u : 1u) * (uint32_t)it.dp * BK * 2;
        for (int kb = it.kb0; kb < it.kb1; ++kb) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag)) { ok = false; break; }
          if (withhold && blockIdx.x == 0 && i == 0 && kb == it.kb0) {
            // test hook: this stage is never loaded, so the MMA warp's bounded
            // wait on it runs out and the CTA takes its timeout path
            if (++stage == S) { stage = 0; phase ^= 1u; }
            continue;
          }
          ++issued;
          const uint32_t sa = base + stage * stage_bytes, sb = sa + A_TILE_BYTES;
          mbar_expect_tx(full_bar(stage), bytes);
          if (!TRANS) {
            if (!it.a_split) {
              tma_load_2d(sa, it.mA, full_bar(stage), kb * BK, it.tile * BM, pol_a);
            } else {
              tma_load_2d(sa, it.mA, full_bar(stage), kb * BK, it.tile * BM, pol_a);
              tma_load_2d(sa + A_TILE_BYTES / 2, it.mA, full_bar(stage), kb * BK,
                          it.tile * BM + 64, pol_a);
            }
          } else {
            tma_load_2d(sa, it.mA, full_bar(stage), it.tile * BM, kb * BK, pol_a);
            tma_load_2d(sa + A_TILE_BYTES / 2, it.mA, full_bar(stage), it.tile * BM + 64,
                        kb * BK, pol_a);
          }
          tma_load_2d(sb, it.mB, full_bar(stage), kb * BK, it.bcol, pol_b);
          if (B2) tma_load_2d(sb + b_tile, it.mB2, full_bar(stage), kb * BK, it.bcol, pol_b);
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 1);
        // let the loads already issued land before the CTA releases its
        // shared memory: wait (bounded) on the newest phase of each stage
        int st2 = stage;
        uint32_t ph2 = phase;
        const int64_t back = issued < S ? issued : S;
        for (int64_t j = 0; j < back; ++j) {
          if (st2 == 0) { st2 = S; ph2 ^= 1u; }
          --st2;
          volatile int never = 0;
          mbar_wait(full_bar(st2), ph2, &never);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int i = 0; i < nitems && ok; ++i) {
        const TcItem it = w.get(i);
        const uint32_t idesc = idesc_bf16(it.dp, TRANS);
        const int acc = i & 1;
        const uint32_t use = (uint32_t)(i >> 1);
        if (!mbar_wait(tempty_bar(acc), (use & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tmem_d = tmem_base + (uint32_t)(acc * 256);
        for (int kb = it.kb0; kb < it.kb1; ++kb) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = base + stage * stage_bytes, sb = sa + A_TILE_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            uint64_t ad, bd;
            if (!TRANS) ad = sdesc(sa + kk * 32, 16, 1024);
            else        ad = sdesc(sa + kk * 2048, A_TILE_BYTES / 2, 1024);
            bd = sdesc(sb + kk * 32, 16, 1024);
            mma_bf16(tmem_d, ad, bd, idesc, (kb > it.kb0 || kk > 0) ? 1u : 0u);
            if (B2) mma_bf16(tmem_d, ad, sdesc(sb + b_tile + kk * 32, 16, 1024), idesc, 1u);
          }
          mma_commit(empty_bar(stage));
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull_bar(acc));
      }
      if (!ok) { *abort_flag = 1; atomicExch(err, 1); }
      // every MMA this thread issued has completed before TMEM is freed
      mma_commit(drain_bar);
      volatile int never = 0;
      mbar_wait(drain_bar, 0, &never);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int g = warp & 3;  // TMEM lane quarter this warp may access
    const int row = g * 32 + lane;
    bool ok = true;
    for (int i = 0; i < nitems && ok; ++i) {
      const TcItem it = w.get(i);
      const int acc = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);
      // the warp agrees on the outcome before its collective TMEM loads
      if (!__all_sync(0xffffffffu, mbar_wait(tfull_bar(acc), use & 1u, abort_flag))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + (uint32_t)(acc * 256) + ((uint32_t)(g * 32) << 16);
      const bool valid = row < it.rows;
      float* dst = it.out + (int64_t)row * it.ldo;
      for (int c = 0; c < it.dp; c += 16) {
        float v[16];
        tmem_ld16(taddr + c, v);
        if (valid) {
          float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
          for (int j = 0; j < 4; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(acc));
    }
    if (!ok) { *abort_flag = 1; if (lane == 0) atomicExch(err, 1); }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base)
                 : "memory");
  }
}

template <bool TRANS, bool B2>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ TcParams p) {
  const WorkSingle w{&tmA, &tmB, &tmB2, &p};
  tc_body<TRANS, B2>(w, p.err, p.stages, p.dpi, p.withhold);
}

template <bool TRANS, bool B2>
__global__ void __launch_bounds__(NTHREADS, 1)
k_btc_gemm(const BTcTile* __restrict__ list, int n, const BMat* __restrict__ T,
           const CUtensorMap* __restrict__ maps, int dst, int stages, int dpmax, int* err) {
  const WorkBatch w{list, n, T, maps, dst, TRANS};
  tc_body<TRANS, B2>(w, err, stages, dpmax);
}

// Sum the stream-K fragments of each tail tile in CTA order into the output.
// One block per (tail tile, 4 rows), one thread per 4 columns (16-byte loads,
// up to 16 contributors in flight), after the block lists the tile's
// contributing CTAs and fragment slots.
__global__ void __launch_bounds__(256) k_tc_fixup(TcParams p, int P) {
  __shared__ int s_src[256];
  __shared__ int s_cnt[8];
  pdl_launch();
  pdl_wait();
  const int tt = blockIdx.x;  // tail tile index
  const int64_t KB = p.KB;
  const int64_t lo = tt * KB, hi = lo + KB;
  // the contributors are consecutive CTAs starting near lo P / U (at most
  // P / tail + 2 of them): thread i tests CTA c0 + i, then an ordered
  // compaction by warp ballots lists them with their fragment slots
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = max(0, (int)((lo * P) / p.U) - 2);
  const int cc = c0 + (int)threadIdx.x;
  bool f = false;
  int slot = 0;
  if (cc < P) {
    const int64_t u0 = sk_start(cc, p.U, P), u1 = sk_start(cc + 1, p.U, P);
    f = u0 < hi && u1 > lo && u1 > u0;
    slot = (u0 / KB == tt) ? 0 : 1;
  }
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_cnt[w] = __popc(b);
  __syncthreads();
  int pos = __popc(b & ((1u << lane) - 1u)), n = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < w) pos += s_cnt[k];
    n += s_cnt[k];
  }
  if (f) s_src[pos] = cc * 2 + slot;
  __syncthreads();
  // block (tt, y): rows 4 y .. 4 y + 3 of the tile, a thread per 4 columns
  const int tile = p.full_waves * P + tt;
  const int mt = tile / p.ns, col0 = (tile - mt * p.ns) * p.dpi;
  const int q4 = p.dpi / 4;
  const int r = blockIdx.y * 4 + threadIdx.x / 64, c4 = threadIdx.x % 64;
  const int64_t gr = (int64_t)mt * BM + r;
  if (gr >= p.Mout || c4 >= q4) return;
  const float4* frag = reinterpret_cast<const float4*>(p.frag);
  // sixteen 16-byte loads in flight, summed in contributor order
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = 0; i < n; i += 16) {
    float4 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (i + u < n) v[u] = frag[((int64_t)s_src[i + u] * BM + r) * q4 + c4];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (i + u < n) {
        s.x += v[u].x;
        s.y += v[u].y;
        s.z += v[u].z;
        s.w += v[u].w;
      }
  }
  *reinterpret_cast<float4*>(p.out + gr * p.ldo + col0 + 4 * c4) = s;
}

// dst[c][r] = bf16(src[r][c]) for c < cols, 0 for cols <= c < dp (r < rows);
// lo (optional): the low part, bf16(src[r][c] - dst[c][r]).
template <typename TS>
__global__ void k_transpose_bf16(const TS* __restrict__ src, int64_t lds, int64_t rows, int cols,
                                 int dp, __nv_bfloat16* __restrict__ dst, int64_t ldd,
                                 __nv_bfloat16* __restrict__ lo) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < rows && c < cols) v = (float)src[r * lds + c];
    t[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (c < dp && r < rows) {
      const float v = t[threadIdx.x][i];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      dst[(int64_t)c * ldd + r] = h;
      if (lo != nullptr) lo[(int64_t)c * ldd + r] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld_elems,
              uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld_elems * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

namespace {

// ---------------------------------------------------------------------------
// Gram of a tall FP32 matrix on the tensor cores (orth()'s Y^T Y, Section II-A):
// Y (M x dp, FP32, dp <= 256) is split on the fly into three BF16 parts,
// y = h + m + l with h = bf16(y), m = bf16(y - h), l = bf16(y - h - m)
// (|y - h - m - l| <= 2^-27 |y|), and
//   Y^T Y ~= h'h + h'm + m'h + m'm + h'l + l'h
// (the dropped m'l, l'm, l'l terms are below 2^-26 of |y_i||y_j|).  Products
// of BF16 parts are exact in FP32, so the result matches an FP32 Gram.
// Each CTA owns a slab of rows.  Warps 0..7 write each chunk's three parts
// into a 128B-swizzled stage of a four-deep ring (both operands MN-major:
// rows of Y are the contraction); warp 8 issues, per chunk, 2 (M tiles of
// 128 Gram rows) x 6 (part pairs) x K/16 MMAs with N = dp into TMEM (M tile
// 1 only over the columns from 128 on: the upper triangle).  Slab sums (FP32)
// go to part[c]; k_gram_tc_reduce adds them in CTA order with compensated
// FP32 summation.
constexpr int GT_CONV = 8;                      // converter / epilogue warps
constexpr int GT_THREADS = 32 * (GT_CONV + 1);  // + the MMA warp
constexpr int GT_NST = 4;                       // ring depth
constexpr uint32_t GT_STAGE = 48 * 1024;        // h, m, l of one (or two) operands
constexpr int GT_SLAB = 32;                     // slab rows: a multiple of this
// Rows per chunk: 32 for Y^T Y, 16 for X^T Y (two operands per stage).
template <bool SYM>
struct GtShape {
  static constexpr int ROWS = SYM ? 32 : 16;
  static constexpr uint32_t BOX = ROWS * 128;     // [ROWS][64 BF16] box
  static constexpr uint32_t SPLIT = 4 * BOX;      // 256 columns
  static constexpr uint32_t OPER = 3 * SPLIT;     // h, m, l
};

// SYM: C = Y^T Y; else C = Y^T Y2 (A operand from Y, B from Y2; only the
// upper block triangle is formed).
template <bool SYM>
__global__ void __launch_bounds__(GT_THREADS, 1)
k_gram_tc(const float* __restrict__ Y, const float* __restrict__ Y2, int64_t ldy, int64_t M,
          int d, int dp, int64_t slab_rows, float* __restrict__ part, int* err) {
  using Sh = GtShape<SYM>;
  constexpr int GT_ROWS = Sh::ROWS;
  constexpr uint32_t GT_BOX = Sh::BOX, GT_SPLIT = Sh::SPLIT;
  constexpr uint32_t B_OFF = SYM ? 0 : Sh::OPER;  // B operand parts
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  // barriers: full[NST] (8 arrivals), empty[NST] (MMA commit), done, drain
  const uint32_t bar = base + GT_NST * GT_STAGE;
  auto full = [&](int s) { return bar + 8u * s; };
  auto empty = [&](int s) { return bar + 8u * (GT_NST + s); };
  const uint32_t done = bar + 16u * GT_NST, drain = done + 8;
  uint32_t* tmem_slot = (uint32_t*)(base_ptr + GT_NST * GT_STAGE + 16 * GT_NST + 32);
  __shared__ int s_abort;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int s2 = 0; s2 < GT_NST; ++s2) {
      mbar_init(full(s2), GT_CONV);
      mbar_init(empty(s2), 1);
    }
    mbar_init(done, 1);
    mbar_init(drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == GT_CONV) {
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
  const int64_t r_begin = (int64_t)blockIdx.x * slab_rows;
  const int64_t r_end = min(M, r_begin + slab_rows);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + GT_ROWS - 1) / GT_ROWS) : 0;
  const int n1 = dp > 128 ? dp - 128 : 16;  // M tile 1: columns 128..dp-1
  bool ok = true;

  if (warp == GT_CONV) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      // kind::f16, BF16 x BF16 -> FP32, A and B MN-major, M = 128, N = dp
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(dp >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t idesc1 = (idesc & ~(0x3Fu << 17)) | ((uint32_t)(n1 >> 3) << 17);
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
      for (int i = 0; i < nchunks; ++i) {
        const int st = i % GT_NST;
        const uint32_t stage = base + st * GT_STAGE;
        if (!mbar_wait(full(st), (uint32_t)((i / GT_NST) & 1), abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // part pairs (A part, B part): hh, hm, mh, mm, hl, lh.  M tile 0 is
        // Gram rows 0..127 against all dp columns; M tile 1 (rows 128..) only
        // needs the columns from 128 on (the upper triangle)
#pragma unroll
        for (int kk = 0; kk < GT_ROWS / 16; ++kk) {
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            if (mt == 1 && dp <= 128) break;
            const uint32_t id = mt == 0 ? idesc : idesc1;
            const uint64_t a0 = sdesc(stage + 2 * mt * GT_BOX + kk * 2048, GT_BOX, 1024);
            const uint64_t b0 = sdesc(stage + B_OFF + 2 * mt * GT_BOX + kk * 2048, GT_BOX, 1024);
#pragma unroll
            for (int q = 0; q < 6; ++q)
              mma_bf16(tmem_base + (uint32_t)(mt * 256), a0 + (uint64_t)((pa[q] * GT_SPLIT) >> 4),
                       b0 + (uint64_t)((pb[q] * GT_SPLIT) >> 4), id,
                       (i > 0 || kk > 0 || q > 0) ? 1u : 0u);
          }
        }
        mma_commit(empty(st));
      }
      if (ok) mma_commit(done);
      else s_abort = 1;
    }
  } else {
    // ---------------- converters (warps 0..7) ----------------
    // per operand GT_ROWS rows x 64 groups of 4 columns (256 columns, zero
    // beyond d) per chunk; chunk i + 1's loads are in flight while chunk i
    // is converted.  Element e: operand e / (GT_ROWS * 64) (always 0 when SYM)
    constexpr int PER = (SYM ? 1 : 2) * GT_ROWS * 64 / (GT_CONV * 32);
    constexpr int OPE = GT_ROWS * 64;  // float4 per operand and chunk
    auto load = [&](int i, float4 (&x)[PER]) {
      const int64_t r0 = r_begin + (int64_t)i * GT_ROWS;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = t + q * GT_CONV * 32;
        const int row = (e % OPE) >> 6, c = (e & 63) * 4;
        const float* src = (SYM || e < OPE) ? Y : Y2;
        x[q] = (r0 + row < r_end && c < dp)
                   ? *reinterpret_cast<const float4*>(src + (r0 + row) * ldy + c)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto step = [&](int i, float4 (&cur)[PER], float4 (&nxt)[PER]) {
      const int st = i % GT_NST;
      const uint32_t stage = base + st * GT_STAGE;
      if (i >= GT_NST &&
          !mbar_wait(empty(st), (uint32_t)(((i / GT_NST) - 1) & 1), abort_flag)) {
        ok = false;
        return;
      }
      if (i + 1 < nchunks) load(i + 1, nxt);
      asm volatile("" ::: "memory");  // the loads are issued before the conversion
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = t + q * GT_CONV * 32;
        const int row = (e % OPE) >> 6, c = (e & 63) * 4;
        const uint32_t obase = (SYM || e < OPE) ? 0u : Sh::OPER;
        float v[4] = {(c < d) ? cur[q].x : 0.f, (c + 1 < d) ? cur[q].y : 0.f,
                      (c + 2 < d) ? cur[q].z : 0.f, (c + 3 < d) ? cur[q].w : 0.f};
        uint32_t hp[2], mp[2], lp[2];
        split3_bf16x4(v, hp, mp, lp);
        const int box = c >> 6, cb = c & 63;
        const uint32_t off = (uint32_t)box * GT_BOX + (uint32_t)row * 128 +
                             ((uint32_t)((cb >> 3) ^ (row & 7)) << 4) + (uint32_t)((cb & 7) * 2);
        const uint32_t a = stage + obase + off;
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(hp[0]), "r"(hp[1])
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + GT_SPLIT), "r"(mp[0]),
                     "r"(mp[1])
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + 2 * GT_SPLIT), "r"(lp[0]),
                     "r"(lp[1])
                     : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(full(st));
    };
    float4 x0[PER], x1[PER];
    if (nchunks > 0) load(0, x0);
    for (int i = 0; i < nchunks && ok; ++i) {
      if (i & 1) step(i, x1, x0);
      else step(i, x0, x1);
    }
    // the accumulators are final once every MMA has completed
    if (ok && nchunks > 0 && !mbar_wait(done, 0, abort_flag)) ok = false;
    if (!ok) s_abort = 1;
  }
  __syncthreads();
  if (*abort_flag) ok = false;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 of M tile w / 4,
  // Gram rows 32 g .. 32 g + 31 with g = w (row block), and stores the
  // columns from 32 g on (the upper block triangle) of its slab sum in the
  // lane-major layout part[c][g][col][32]: lane l of the warp writes row
  // 32 g + l, so each store is one contiguous 128-byte line.
  const int nbr = (dp + 31) / 32;
  float* P = part + (int64_t)blockIdx.x * nbr * dp * 32;
  if (warp < GT_CONV) {
    const int mt = warp >> 2, g4 = warp & 3, g = warp;
    const int c0 = mt * 128, ncol = mt == 0 ? dp : n1;
    if (g < nbr && (mt == 0 || dp > 128)) {
      for (int c = 32 * g4; c < ncol; c += 16) {
        float v[16];
        if (ok && nchunks > 0) {
          tmem_ld16(tmem_base + (uint32_t)(mt * 256 + c) + ((uint32_t)(g4 * 32) << 16), v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        float* dst = P + ((int64_t)g * dp + c0 + c) * 32 + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + c + j < dp) dst[j * 32] = v[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == GT_CONV) {
    if (lane == 0) {  // every MMA this CTA issued has completed before TMEM is freed
      volatile int never = 0;
      tc_fence_after();
      mma_commit(drain);
      mbar_wait(drain, 0, &never);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base)
                 : "memory");
  }
}

// s + c accumulates x: Knuth's TwoSum of s and x, its rounding error
// collected in c (compensated summation in FP32; GB300's FP64 rate is a
// small fraction of its FP32 rate, so the slab sums are not added in FP64).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// C = sum over CTAs of the slab sums, mirrored from the upper triangle, as
// FP64 (s + c of the compensated FP32 sum) and Cf = fl32(s + c).  Block
// (col, g) adds entries (32 g + l, col), l = lane, of the P slab sums (one
// 128-byte line each in the lane-major layout); warp w adds the slab sums
// z = w, w + 8, ... in order, then the 8 warp sums are added in warp order
// (a fixed, deterministic order).
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const float* __restrict__ part, int P,
                                                        int d, int dp, bool sym,
                                                        double* __restrict__ C,
                                                        float* __restrict__ Cf) {
  __shared__ float ws[8][33], wc[8][33];
  pdl_launch();
  pdl_wait();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int col = blockIdx.x, g = blockIdx.y, nbr = gridDim.y;
  if (col >= d || col < 32 * g) return;  // block-uniform
  const int i = 32 * g + lane;
  const int64_t slab = (int64_t)nbr * dp * 32, src = ((int64_t)g * dp + col) * 32 + lane;
  float s = 0.f, c = 0.f;
  int z = w;
  for (; z + 8 * 3 < P; z += 8 * 4) {
    const float a = part[z * slab + src], b = part[(z + 8) * slab + src];
    const float x = part[(z + 16) * slab + src], e = part[(z + 24) * slab + src];
    two_sum_acc(s, c, a);
    two_sum_acc(s, c, b);
    two_sum_acc(s, c, x);
    two_sum_acc(s, c, e);
  }
  for (; z < P; z += 8) two_sum_acc(s, c, part[z * slab + src]);
  ws[w][lane] = s;
  wc[w][lane] = c;
  __syncthreads();
  if (w == 0 && i <= col && i < d) {
    float t = 0.f, tc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      two_sum_acc(t, tc, ws[k][lane]);
      tc += wc[k][lane];
    }
    const double v = (double)t + (double)tc;
    const float f = t + tc;
    C[(int64_t)i * d + col] = v;
    if (i != col) C[(int64_t)col * d + i] = sym ? v : 0.0;
    if (Cf != nullptr) {
      Cf[(int64_t)i * d + col] = f;
      if (i != col) Cf[(int64_t)col * d + i] = sym ? f : 0.f;
    }
  }
}

}  // namespace

bool tc_supported(const void* A, int64_t lda, int dp) {
  return dp >= 16 && dp <= 256 && dp % 16 == 0 && lda % 8 == 0 && ((uintptr_t)A & 15) == 0 &&
         encode_fn() != nullptr;
}

size_t tc_frag_bytes(int dp) { return (size_t)sm_count() * 2 * BM * dp * sizeof(float); }

// Rows per CTA (a multiple of the 64-row chunk) and the number of CTAs, every
// one of which gets rows; functions of M (and the SM count) only.
static int64_t gram_tc_slab(int64_t M) {
  const int64_t chunks = (M + GT_SLAB - 1) / GT_SLAB;
  const int64_t p0 = std::min<int64_t>(sm_count(), std::max<int64_t>(chunks, 1));
  const int64_t slab = (M + p0 - 1) / p0;
  return (slab + GT_SLAB - 1) / GT_SLAB * GT_SLAB;  // a multiple of both kernels' chunk
}

int gram_tc_ctas(int64_t M) {
  const int64_t slab = gram_tc_slab(M);
  return (int)std::max<int64_t>(1, (M + slab - 1) / slab);
}

size_t gram_tc_part_bytes(int d) {
  const int dp = (d + 15) / 16 * 16;
  return (size_t)sm_count() * ((dp + 31) / 32) * dp * 32 * sizeof(float);
}

bool gram_tc_supported(int64_t M, int d, int64_t ldy, const void* Y) {
  const int dp = (d + 15) / 16 * 16;
  return M >= 8192 && d >= 1 && dp <= 256 && ldy % 4 == 0 && ((uintptr_t)Y & 15) == 0 &&
         ldy >= dp;
}

static cudaError_t gram_tc_run(const float* Y, const float* Y2, int64_t ldy, int64_t M, int d,
                               float* part, double* C, float* Cf, int* err, cudaStream_t st) {
  if (!gram_tc_supported(M, d, ldy, Y) || (Y2 != nullptr && ((uintptr_t)Y2 & 15) != 0))
    return cudaErrorInvalidValue;
  const int dp = (d + 15) / 16 * 16;
  const int P = gram_tc_ctas(M);
  const int64_t slab = gram_tc_slab(M);
  const size_t smem = 1024 + GT_NST * (size_t)GT_STAGE + 16 * GT_NST + 64;
  cudaError_t e;
  if (Y2 == nullptr) {
    e = cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_gram_tc<true>, dim3(P), dim3(GT_THREADS), smem, st, Y,
                   (const float*)nullptr, ldy, M, d, dp, slab, part, err);
  } else {
    e = cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_gram_tc<false>, dim3(P), dim3(GT_THREADS), smem, st, Y, Y2, ldy, M, d, dp,
                   slab, part, err);
  }
  count_launch();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_gram_tc_reduce, dim3(d, (dp + 31) / 32), dim3(256), 0, st, (const float*)part,
                 P, d, dp, Y2 == nullptr, C, Cf);
  count_launch();
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t gram_tc(const float* Y, int64_t ldy, int64_t M, int d, float* part, double* C,
                    float* Cf, int* err, cudaStream_t st) {
  return gram_tc_run(Y, nullptr, ldy, M, d, part, C, Cf, err, st);
}

cudaError_t gram_tc_upper(const float* X, const float* Y, int64_t ld, int64_t M, int d,
                          float* part, double* C, int* err, cudaStream_t st) {
  return gram_tc_run(X, Y, ld, M, d, part, C, nullptr, err, st);
}

namespace {
// Dynamic shared memory of the product kernels: 1 KB alignment slack, the
// ring, the 2 S + 5 mbarriers and the TMEM address word.
size_t tc_smem(int stages, size_t stage_bytes) {
  return 1024 + stages * stage_bytes + 8 * (2 * stages + 5) + 16;
}
// The deepest ring (at most 8 stages) within 226 KB of the 227 KB a CTA may
// opt into: 5 stages of 44 KB at dp = 224, 4 of 48 KB at dp = 256.
int tc_stages(size_t stage_bytes) {
  int s = 8;
  while (s > 0 && tc_smem(s, stage_bytes) > 226 * 1024) --s;
  return s;
}
}  // namespace

namespace {

// Launch configuration of one product: column split and ring depth.
struct TcCfg {
  int ns = 1, stages = 0;
};

size_t tc_stage_bytes(int dp, int ns, bool b2) {
  return A_TILE_BYTES + (b2 ? 2 : 1) * (size_t)(dp / ns) * BK * 2;
}

bool tc_ns_valid(int dp, int ns) { return dp % ns == 0 && (dp / ns) % 16 == 0 && dp / ns >= 16; }

// The measured choice per product shape (trans, two-part, output rows, K,
// dp), process-wide, optionally mirrored in a text file (ruqlp_tune_file).
std::mutex g_tune_mu;
std::map<std::array<int64_t, 5>, TcCfg> g_tune;
std::string g_tune_path;

void tune_save_line(const std::array<int64_t, 5>& key, const TcCfg& c, double us) {
  if (g_tune_path.empty()) return;
  FILE* f = fopen(g_tune_path.c_str(), "a");
  if (!f) return;
  fprintf(f, "tc_gemm %lld %lld %lld %lld %lld %d %d %.3f\n", (long long)key[0], (long long)key[1],
          (long long)key[2], (long long)key[3], (long long)key[4], c.ns, c.stages, us);
  fclose(f);
}

struct TcOperands {
  bool trans, b2;
  const void *A, *Bt, *Btl;
  int64_t lda, m, n, ldb, ldo;
  int dp;
  float *out, *frag;
  int* err;
};

// One product launch (and its stream-K fix-up) with configuration c.
cudaError_t tc_launch(const TcOperands& o, const TcCfg& c, cudaStream_t st,
                      const std::function<void(bool)>& mark, int withhold = 0) {
  const int64_t Mout = o.trans ? o.n : o.m, K = o.trans ? o.m : o.n;
  const int dpi = o.dp / c.ns;
  CUtensorMap mA, mB, mB2;
  if (!make_map(&mA, o.A, (uint64_t)o.n, (uint64_t)o.m, (uint64_t)o.lda, 64, o.trans ? 64 : BM))
    return cudaErrorInvalidValue;
  if (!make_map(&mB, o.Bt, (uint64_t)K, (uint64_t)o.dp, (uint64_t)o.ldb, 64, (uint32_t)dpi))
    return cudaErrorInvalidValue;
  if (o.b2) {
    if (!make_map(&mB2, o.Btl, (uint64_t)K, (uint64_t)o.dp, (uint64_t)o.ldb, 64, (uint32_t)dpi))
      return cudaErrorInvalidValue;
  } else {
    mB2 = mB;  // unused
  }
  TcParams p{};
  p.Mout = Mout;
  p.K = K;
  p.dp = o.dp;
  p.ns = c.ns;
  p.dpi = dpi;
  p.out = o.out;
  p.ldo = o.ldo;
  p.frag = o.frag;
  p.err = o.err;
  p.T = ceil_div(Mout, BM) * c.ns;
  p.KB = ceil_div(K, BK);
  int P = sm_count();  // never more CTAs than the fragment buffer has slots for
  if ((int64_t)p.T * p.KB < P) P = p.T * p.KB;
  p.full_waves = p.T / P;
  p.tail = p.T - p.full_waves * P;
  p.U = (int64_t)p.tail * p.KB;
  p.stages = c.stages;
  p.withhold = withhold;
  const size_t smem = tc_smem(c.stages, tc_stage_bytes(o.dp, c.ns, o.b2));
  auto kern = o.trans ? (o.b2 ? k_tc_gemm<true, true> : k_tc_gemm<true, false>)
                      : (o.b2 ? k_tc_gemm<false, true> : k_tc_gemm<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (mark) mark(true);
  e = launch_pdl(kern, dim3(P), dim3(NTHREADS), smem, st, mA, mB, mB2, p);
  if (mark) mark(false);
  count_launch();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess || p.tail == 0) return e;
  e = launch_pdl(k_tc_fixup, dim3(p.tail, BM / 4), dim3(256), 0, st, p, P);
  count_launch();
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

int tune_file(const char* path) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_path = path ? path : "";
  if (g_tune_path.empty()) return 0;
  FILE* f = fopen(g_tune_path.c_str(), "r");
  if (!f) return 0;
  int n = 0;
  char tag[32];
  long long k0, k1, k2, k3, k4;
  int ns, stages;
  double us;
  while (fscanf(f, "%31s %lld %lld %lld %lld %lld %d %d %lf", tag, &k0, &k1, &k2, &k3, &k4, &ns,
                &stages, &us) == 9) {
    if (strcmp(tag, "tc_gemm") != 0 || !tc_ns_valid((int)k4, ns) || stages < 2 ||
        tc_smem(stages, tc_stage_bytes((int)k4, ns, k1 != 0)) > 226 * 1024)
      continue;
    TcCfg c;
    c.ns = ns;
    c.stages = stages;
    g_tune[{k0, k1, k2, k3, k4}] = c;
    ++n;
  }
  fclose(f);
  return n;
}

// Products of one shape run with the configuration measured fastest the
// first time that shape is seen (outside stream capture): every valid
// column split ns in {1, 2, 4} with the deepest ring that fits, each timed
// twice with CUDA events on the stream (the better time counts); the chosen
// configuration then computes the result, so repeated calls are bitwise
// equal.  force_ns > 0 skips the tuner.
cudaError_t tc_gemm(bool trans, const void* A, int64_t lda, int64_t m, int64_t n, const void* Bt,
                    int64_t ldb, int dp, float* out, int64_t ldo, float* frag, int* err,
                    cudaStream_t st, const std::function<void(bool)>& mark, const void* Btl,
                    int force_ns, int withhold) {
  if (dp < 16 || dp > 256 || dp % 16 != 0) return cudaErrorInvalidValue;
  if (lda % 8 != 0 || ldb % 8 != 0 || ((uintptr_t)A & 15) || ((uintptr_t)Bt & 15) || ldo % 4 != 0 ||
      ((uintptr_t)out & 15) || ((uintptr_t)Btl & 15))
    return cudaErrorInvalidValue;
  TcOperands o{trans, Btl != nullptr, A, Bt, Btl, lda, m, n, ldb, ldo, dp, out, frag, err};
  auto cfg_of = [&](int ns) {
    TcCfg c;
    c.ns = ns;
    c.stages = tc_stages(tc_stage_bytes(dp, ns, o.b2));
    return c;
  };
  if (force_ns > 0) {
    if (!tc_ns_valid(dp, force_ns)) return cudaErrorInvalidValue;
    const TcCfg c = cfg_of(force_ns);
    if (c.stages < 2) return cudaErrorInvalidValue;
    return tc_launch(o, c, st, mark, withhold);
  }
  const int64_t Mout = trans ? n : m, K = trans ? m : n;
  const std::array<int64_t, 5> key = {trans ? 1 : 0, o.b2 ? 1 : 0, Mout, K, dp};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return tc_launch(o, it->second, st, mark, withhold);
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return tc_launch(o, cfg_of(1), st, mark);  // no timing inside a capture
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return tc_launch(o, cfg_of(1), st, mark);
  }
  TcCfg best = cfg_of(1);
  float best_ms = 1e30f;
  for (int ns : {1, 2, 4}) {
    if (!tc_ns_valid(dp, ns)) continue;
    const TcCfg c = cfg_of(ns);
    if (c.stages < 2) continue;
    float t = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      cudaError_t e = tc_launch(o, c, st, {});
      cudaEventRecord(e1, st);
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return e != cudaSuccess ? e : cudaErrorUnknown;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, ms);
    }
    if (t < best_ms * 0.99f) {  // a larger split must win clearly
      best_ms = t;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    tune_save_line(key, best, 1e3 * best_ms);
  }
  return tc_launch(o, best, st, mark, withhold);
}

bool btc_encode(void* maps4, const void* A, int64_t lda, int64_t m, int64_t n, const void* Bt,
                const void* Btl, int64_t ldbt, int dp, bool a_only) {
  CUtensorMap t;  // encoded in an aligned temporary, then copied into place
  uint8_t* dst = (uint8_t*)maps4;
  if (!make_map(&t, A, (uint64_t)n, (uint64_t)m, (uint64_t)lda, 64, 64)) return false;
  memcpy(dst, &t, sizeof(t));
  if (a_only) return true;
  if (!make_map(&t, Bt, (uint64_t)n, (uint64_t)dp, (uint64_t)ldbt, 64, (uint32_t)dp)) return false;
  memcpy(dst + sizeof(t), &t, sizeof(t));
  if (!make_map(&t, Bt, (uint64_t)m, (uint64_t)dp, (uint64_t)ldbt, 64, (uint32_t)dp)) return false;
  memcpy(dst + 2 * sizeof(t), &t, sizeof(t));
  if (!make_map(&t, Btl, (uint64_t)m, (uint64_t)dp, (uint64_t)ldbt, 64, (uint32_t)dp)) return false;
  memcpy(dst + 3 * sizeof(t), &t, sizeof(t));
  return true;
}

size_t btc_map_bytes() { return kBatchMaps * sizeof(CUtensorMap); }

cudaError_t btc_gemm(bool trans, const BMat* T, int count, const BTcTile* list, int n,
                     const void* maps, int src, int dst, int dpmax, int* err, cudaStream_t st,
                     bool b2) {
  if (n <= 0) return cudaSuccess;
  if (dpmax < 16 || dpmax > 256 || dpmax % 16) return cudaErrorInvalidValue;
  if (b2 && !trans) return cudaErrorInvalidValue;  // the low part is mapped over m only
  const size_t stage_bytes = A_TILE_BYTES + (b2 ? 2 : 1) * (size_t)dpmax * BK * 2;
  const int stages = tc_stages(stage_bytes);
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = tc_smem(stages, stage_bytes);
  auto kern = trans ? (b2 ? k_btc_gemm<true, true> : k_btc_gemm<true, false>)
                    : k_btc_gemm<false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int P = sm_count();
  if (n < P) P = n;
  const CUtensorMap* mp = (const CUtensorMap*)maps;
  kern<<<P, NTHREADS, smem, st>>>(list, n, T, mp, dst, stages, dpmax, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t transpose_to_bf16(Ty ts, const void* src, int64_t lds, int64_t rows, int cols, int dp,
                              void* dst, int64_t ldd, cudaStream_t st, void* lo) {
  dim3 grid(ceil_div(rows, 32), ceil_div(dp, 32)), block(32, 8);
  if (ts == Ty::F64)
    k_transpose_bf16<double><<<grid, block, 0, st>>>((const double*)src, lds, rows, cols, dp,
                                                     (__nv_bfloat16*)dst, ldd,
                                                     (__nv_bfloat16*)lo);
  else if (ts == Ty::F32)
    k_transpose_bf16<float><<<grid, block, 0, st>>>((const float*)src, lds, rows, cols, dp,
                                                    (__nv_bfloat16*)dst, ldd, (__nv_bfloat16*)lo);
  else
    return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
