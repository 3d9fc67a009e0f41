// Tall-skinny cross products C = X^T W (d1 x d2) for orth() (Section II-A;
// the l x l Gram of CholeskyQR and the R factor of qr(B^T)), FP32 inputs.
//
// One CTA of 64 threads owns a 64 x 64 tile of C; every thread accumulates an
// 8 x 8 sub-tile in FP32 over the CTA's slab of rows (32-row chunks staged in
// shared memory, next chunk prefetched into registers).  The FP32 slab sums
// are written as FP64 partials and summed across slabs in slab order (FP64,
// deterministic).  For X == W only the tiles on or above the diagonal are
// computed and the reduction mirrors them.
#include "internal.h"

namespace ruqlp {
namespace {

constexpr int TM = 64, TK = 32, NT = 64;

__device__ __forceinline__ void gram_tile(const float* __restrict__ X, int64_t ldx,
                                          const float* __restrict__ W, int64_t ldw, int64_t M,
                                          int d1, int d2, bool sym, int64_t slab,
                                          double* __restrict__ partial, int tile_id, int slab_id) {
  __shared__ __align__(16) float Xs[TK][TM];
  __shared__ __align__(16) float Ws[TK][TM];
  // tile coordinates: blockIdx.x enumerates (bi, bj) pairs
  const int nb1 = (d1 + TM - 1) / TM, nb2 = (d2 + TM - 1) / TM;
  int bi, bj;
  if (sym) {  // upper triangle of an nb1 x nb1 tile grid, row by row
    int t = tile_id;
    bi = 0;
    while (t >= nb1 - bi) { t -= nb1 - bi; ++bi; }
    bj = bi + t;
  } else {
    bi = tile_id / nb2;
    bj = tile_id % nb2;
  }
  const int c0 = bi * TM, c1 = bj * TM;
  const bool diag = sym && bi == bj;
  const int64_t r_begin = (int64_t)slab_id * slab;
  const int64_t r_end = min(M, r_begin + slab);
  const int t = threadIdx.x;
  const int ty = t >> 3, tx = t & 7;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // a chunk is 32 rows x 64 columns = 2048 floats: 8 float4s per thread
  auto load = [&](const float* S, int64_t lds, int c0_, int dmax, int64_t r0, float4 (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = (q * NT + t) * 4;  // element index in the 32 x 64 chunk
      const int rr = e / TM, cc = e % TM;
      const int64_t r = r0 + rr;
      const int c = c0_ + cc;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < r_end) {
        const float* p = S + r * lds + c;
        if (c + 3 < dmax) {
          x = *reinterpret_cast<const float4*>(p);
        } else {
          if (c < dmax) x.x = p[0];
          if (c + 1 < dmax) x.y = p[1];
          if (c + 2 < dmax) x.z = p[2];
        }
      }
      v[q] = x;
    }
  };
  auto store = [&](float (*Ss)[TM], const float4 (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = (q * NT + t) * 4;
      *reinterpret_cast<float4*>(&Ss[e / TM][e % TM]) = v[q];
    }
  };

  float4 vx[8], vw[8];
  int64_t r0 = r_begin;
  if (r0 < r_end) {
    load(X, ldx, c0, d1, r0, vx);
    if (!diag) load(W, ldw, c1, d2, r0, vw);
  }
  for (; r0 < r_end; r0 += TK) {
    store(Xs, vx);
    if (!diag) store(Ws, vw);
    __syncthreads();
    if (r0 + TK < r_end) {  // prefetch the next chunk while computing this one
      load(X, ldx, c0, d1, r0 + TK, vx);
      if (!diag) load(W, ldw, c1, d2, r0 + TK, vw);
    }
    const float(*Bs)[TM] = diag ? Xs : Ws;
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* P = partial + (int64_t)slab_id * d1 * d2;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = c0 + ty * 8 + i;
    if (r >= d1) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c1 + tx * 8 + j;
      if (c < d2) P[(int64_t)r * d2 + c] = (double)acc[i][j];
    }
  }
}

// Small-d variant for batches: one dp x dp tile (dp = 8 TPT <= 80) per slab,
// thread (ty, tx) of an 8 x 8 grid owns a TPT x TPT block; both triangles
// are computed (the FP32 products commute, so the lower triangle equals the
// mirror of the upper bitwise).  Every entry is the same sequential FP32 sum
// over the slab's rows as in gram_tile, so results match it bitwise.
constexpr int SMALL_MAX = 80;  // largest dp of the small variant
template <int TPT>
__device__ __forceinline__ void gram_small(const float* __restrict__ X, const float* __restrict__ W,
                                           int64_t ld, int64_t M, int d, bool sym, int64_t slab,
                                           double* __restrict__ partial, int slab_id,
                                           float* __restrict__ sbuf) {
  constexpr int E = 8 * TPT;
  float(*Xs)[E] = reinterpret_cast<float(*)[E]>(sbuf);  // TK x E each
  float(*Ws)[E] = reinterpret_cast<float(*)[E]>(sbuf + TK * E);
  const int64_t r_begin = (int64_t)slab_id * slab;
  const int64_t r_end = min(M, r_begin + slab);
  const int t = threadIdx.x, ty = t >> 3, tx = t & 7;
  float acc[TPT][TPT];
#pragma unroll
  for (int i = 0; i < TPT; ++i)
#pragma unroll
    for (int j = 0; j < TPT; ++j) acc[i][j] = 0.f;
  constexpr int NV = TK * E / 4 / NT;  // float4s per thread per chunk (= TPT)
  auto load = [&](const float* S, int64_t r0, float4 (&v)[NV]) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = (q * NT + t) * 4;
      const int rr = e / E, cc = e % E;
      const int64_t r = r0 + rr;
      v[q] = (r < r_end) ? *reinterpret_cast<const float4*>(S + r * ld + cc)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store = [&](float (*Ss)[E], const float4 (&v)[NV]) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = (q * NT + t) * 4;
      *reinterpret_cast<float4*>(&Ss[e / E][e % E]) = v[q];
    }
  };
  float4 vx[NV], vw[NV];
  int64_t r0 = r_begin;
  if (r0 < r_end) {
    load(X, r0, vx);
    if (!sym) load(W, r0, vw);
  }
  for (; r0 < r_end; r0 += TK) {
    store(Xs, vx);
    if (!sym) store(Ws, vw);
    __syncthreads();
    if (r0 + TK < r_end) {
      load(X, r0 + TK, vx);
      if (!sym) load(W, r0 + TK, vw);
    }
    const float(*Bs)[E] = sym ? Xs : Ws;
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      float a[TPT], b[TPT];
#pragma unroll
      for (int i = 0; i < TPT; i += 2) {
        const float2 x2 = *reinterpret_cast<const float2*>(&Xs[k][ty * TPT + i]);
        const float2 w2 = *reinterpret_cast<const float2*>(&Bs[k][tx * TPT + i]);
        a[i] = x2.x;
        a[i + 1] = x2.y;
        b[i] = w2.x;
        b[i + 1] = w2.y;
      }
#pragma unroll
      for (int i = 0; i < TPT; ++i)
#pragma unroll
        for (int j = 0; j < TPT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* P = partial + (int64_t)slab_id * d * d;
#pragma unroll
  for (int i = 0; i < TPT; ++i) {
    const int r = ty * TPT + i;
    if (r >= d) continue;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
      const int c = tx * TPT + j;
      if (c < d) P[(int64_t)r * d + c] = (double)acc[i][j];
    }
  }
}

// Batched Grams take the small-d variant when dp <= 80.
__host__ __device__ inline bool gram_is_small(int dp) { return dp <= SMALL_MAX; }

__global__ void __launch_bounds__(NT)
k_gram_tiles(const float* __restrict__ X, int64_t ldx, const float* __restrict__ W, int64_t ldw,
             int64_t M, int d1, int d2, bool sym, int64_t slab, double* __restrict__ partial,
             const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  gram_tile(X, ldx, W, ldw, M, d1, d2, sym, slab, partial, blockIdx.x, blockIdx.y);
}

// sum_z P[z * stride + idx] for z < slabs, in slab order, with eight
// independent loads in flight
__device__ __forceinline__ double slab_sum(const double* __restrict__ P, int slabs, int64_t stride,
                                           int64_t idx) {
  double s = 0.0;
  int z = 0;
  for (; z + 8 <= slabs; z += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = P[(int64_t)(z + u) * stride + idx];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; z < slabs; ++z) s += P[(int64_t)z * stride + idx];
  return s;
}

// C[i][j] = sum over slabs of the partials (slab order); with sym the entry
// is taken from the computed upper triangle.
__global__ void k_gram_reduce(const double* __restrict__ P, int slabs, int d1, int d2, bool sym,
                              double* __restrict__ C, float* __restrict__ Cf,
                              const int32_t* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)d1 * d2) return;
  int i = (int)(idx / d2), j = (int)(idx % d2);
  const int64_t src = (sym && j < i) ? ((int64_t)j * d2 + i) : idx;
  const double s = slab_sum(P, slabs, (int64_t)d1 * d2, src);
  C[idx] = s;
  if (Cf != nullptr) Cf[idx] = (float)s;
}

// Batched Grams: tile t of the launch -> (matrix, tile, slab) through prefix;
// M = rows of buf[src] (m for Y, n otherwise).
__global__ void __launch_bounds__(NT)
k_bgram(const BMat* __restrict__ Tb, const int* __restrict__ prefix, int count, int src, int src2,
        int max_slabs) {
  const int t = blockIdx.x;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const BMat& b = Tb[prefix[count + 1 + lo]];  // the launch order's item lo
  const int local = t - prefix[lo];
  const bool sym = src == src2;
  const int64_t M = (src == B_Y) ? b.m : b.n;
  int64_t slab;
  gram_slabs(M, max_slabs, &slab);
  if (gram_is_small(b.dp)) {
    __shared__ __align__(16) float sbuf[2 * TK * SMALL_MAX];
    const float* X = bbuf(b, src);
    const float* W = bbuf(b, src2);
    switch (b.dp / 8) {
      case 2: gram_small<2>(X, W, b.dp, M, b.d, sym, slab, b.partial, local, sbuf); break;
      case 4: gram_small<4>(X, W, b.dp, M, b.d, sym, slab, b.partial, local, sbuf); break;
      case 6: gram_small<6>(X, W, b.dp, M, b.d, sym, slab, b.partial, local, sbuf); break;
      case 8: gram_small<8>(X, W, b.dp, M, b.d, sym, slab, b.partial, local, sbuf); break;
      default: gram_small<10>(X, W, b.dp, M, b.d, sym, slab, b.partial, local, sbuf); break;
    }
    return;
  }
  const int nb = (b.d + TM - 1) / TM;
  const int tiles = sym ? nb * (nb + 1) / 2 : nb * nb;
  gram_tile(bbuf(b, src), b.dp, bbuf(b, src2), b.dp, M, b.d, b.d, sym, slab, b.partial,
            local % tiles, local / tiles);
}

// Batched symmetric Grams of narrow items (dp <= 80), one CTA of NTS threads
// per row slab.  The upper triangle is covered by 4 x 8 blocks (rows 4 bi..,
// columns 8 bj.., the blocks with bj >= bi / 2: those holding an entry on or
// above the diagonal), one block per thread, listed row by row (110 blocks at
// dp = 80, 72 at 64, 42 at 48), so only about half of the square's
// multiply-adds are issued.  Every entry (i <= j) is the same sequential FP32
// sum over the slab's rows as in gram_tile (zero-padded rows of the last
// chunk included), so results match it bitwise; entries below the diagonal
// that a straddling block also forms are never read (the reduction mirrors
// the upper triangle).
constexpr int NTS = 128;
constexpr int packed_blocks(int dp) {
  int n = 0;
  for (int bi = 0; bi < dp / 4; ++bi) n += dp / 8 - bi / 2;
  return n;
}
template <int DP>
__device__ __forceinline__ void gram_sym_packed(const float* __restrict__ X, int64_t ld,
                                                int64_t M, int d, int64_t slab,
                                                double* __restrict__ partial, int slab_id,
                                                float* __restrict__ sbuf) {
  constexpr int NBR = DP / 4, NBC = DP / 8;
  constexpr int NV = TK * DP / 4 / NTS;  // float4s per thread per 32-row chunk
  static_assert(NV * 4 * NTS == TK * DP, "chunk split");
  static_assert(packed_blocks(DP) <= NTS, "one block per thread");
  float(*Xs)[DP] = reinterpret_cast<float(*)[DP]>(sbuf);
  const int64_t r_begin = (int64_t)slab_id * slab;
  const int64_t r_end = min(M, r_begin + slab);
  const int t = threadIdx.x;
  int bi = 0, u = t;
  while (bi < NBR && u >= NBC - bi / 2) {
    u -= NBC - bi / 2;
    ++bi;
  }
  const bool active = bi < NBR;
  const int ra = 4 * (active ? bi : 0), cb = 8 * (active ? bi / 2 + u : 0);
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  auto load = [&](int64_t r0, float4 (&v)[NV]) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = (q * NTS + t) * 4;
      const int rr = e / DP, cc = e % DP;
      const int64_t r = r0 + rr;
      v[q] = (r < r_end) ? *reinterpret_cast<const float4*>(X + r * ld + cc)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  float4 vx[NV];
  int64_t r0 = r_begin;
  if (r0 < r_end) load(r0, vx);
  for (; r0 < r_end; r0 += TK) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = (q * NTS + t) * 4;
      *reinterpret_cast<float4*>(&Xs[e / DP][e % DP]) = vx[q];
    }
    __syncthreads();
    if (r0 + TK < r_end) load(r0 + TK, vx);  // next chunk while computing this one
    if (active) {
#pragma unroll 4
      for (int k = 0; k < TK; ++k) {
        const float4 a4 = *reinterpret_cast<const float4*>(&Xs[k][ra]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Xs[k][cb]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Xs[k][cb + 4]);
        const float a[4] = {a4.x, a4.y, a4.z, a4.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  double* P = partial + (int64_t)slab_id * d * d;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ra + i;
    if (r >= d) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = cb + j;
      if (c < d) P[(int64_t)r * d + c] = (double)acc[i][j];
    }
  }
}

// Batched symmetric Grams of the items with dp <= 80: CTA t of the launch ->
// (item, slab) through prefix (launch order appended, as k_bgram).
__global__ void __launch_bounds__(NTS)
k_bgram_sym(const BMat* __restrict__ Tb, const int* __restrict__ prefix, int count, int src,
            int max_slabs) {
  __shared__ __align__(16) float sbuf[TK * SMALL_MAX];
  const int t = blockIdx.x;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const BMat& b = Tb[prefix[count + 1 + lo]];
  const int local = t - prefix[lo];
  const int64_t M = (src == B_Y) ? b.m : b.n;
  int64_t slab;
  gram_slabs(M, max_slabs, &slab);
  const float* X = bbuf(b, src);
  switch (b.dp / 16) {
    case 1: gram_sym_packed<16>(X, b.dp, M, b.d, slab, b.partial, local, sbuf); break;
    case 2: gram_sym_packed<32>(X, b.dp, M, b.d, slab, b.partial, local, sbuf); break;
    case 3: gram_sym_packed<48>(X, b.dp, M, b.d, slab, b.partial, local, sbuf); break;
    case 4: gram_sym_packed<64>(X, b.dp, M, b.d, slab, b.partial, local, sbuf); break;
    default: gram_sym_packed<80>(X, b.dp, M, b.d, slab, b.partial, local, sbuf); break;
  }
}

__global__ void k_bgram_reduce(const BMat* __restrict__ Tb, int src, int src2, int max_slabs) {
  const BMat& b = Tb[blockIdx.y];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = b.d;
  if (idx >= (int64_t)d * d) return;
  const bool sym = src == src2;
  const int64_t M = (src == B_Y) ? b.m : b.n;
  int64_t slab;
  const int slabs = (int)gram_slabs(M, max_slabs, &slab);
  const int i = (int)(idx / d), j = (int)(idx % d);
  // symmetric partials hold one triangle: the upper one from the CUDA-core
  // tiles, the lower one from the tensor-core kernel (orth_tc items)
  const bool mirror = sym && (b.orth_tc ? j > i : j < i);
  const int64_t so = mirror ? ((int64_t)j * d + i) : idx;
  const double s = slab_sum(b.partial, slabs, (int64_t)d * d, so);
  b.G[idx] = s;
  b.Gf[idx] = (float)s;
}

}  // namespace

int bgram_tiles(int64_t M, int d, bool sym, int max_slabs) {
  const int nb = (d + TM - 1) / TM;
  int64_t slab;
  const int slabs = (int)gram_slabs(M, max_slabs, &slab);
  if (gram_is_small((d + 15) / 16 * 16)) return slabs;
  return (sym ? nb * (nb + 1) / 2 : nb * nb) * slabs;
}

int bgram_sym_ctas(int64_t M, int d, int max_slabs) {
  int64_t slab;
  return gram_is_small((d + 15) / 16 * 16) ? (int)gram_slabs(M, max_slabs, &slab) : 0;
}

cudaError_t bgram_sym(const BMat* T, const int* prefix, int total, int count, int src,
                      int max_slabs, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  k_bgram_sym<<<total, NTS, 0, st>>>(T, prefix, count, src, max_slabs);
  count_launch();
  return cudaGetLastError();
}

cudaError_t bgram_reduce(const BMat* T, int count, int src, int src2, int max_slabs, int dmax,
                         cudaStream_t st) {
  k_bgram_reduce<<<dim3(ceil_div((int64_t)dmax * dmax, 256), count), 256, 0, st>>>(T, src, src2,
                                                                                 max_slabs);
  count_launch();
  return cudaGetLastError();
}

cudaError_t bgram(const BMat* T, const int* prefix, int total, int count, int src, int src2,
                  int max_slabs, int dmax, cudaStream_t st, bool reduce) {
  if (total <= 0) return cudaSuccess;
  k_bgram<<<total, NT, 0, st>>>(T, prefix, count, src, src2, max_slabs);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !reduce) return e;
  return bgram_reduce(T, count, src, src2, max_slabs, dmax, st);
}

cudaError_t gram_f32(const float* X, int64_t ldx, const float* W, int64_t ldw, int64_t M, int d1,
                     int d2, double* C, double* partial, int max_slabs, const int32_t* gate,
                     cudaStream_t st, float* Cf) {
  if (M <= 0 || d1 <= 0 || d2 <= 0) return cudaSuccess;
  const bool sym = (X == W) && (ldx == ldw) && (d1 == d2);
  const int nb1 = (d1 + TM - 1) / TM, nb2 = (d2 + TM - 1) / TM;
  const int tiles = sym ? nb1 * (nb1 + 1) / 2 : nb1 * nb2;
  int64_t slab;
  const int64_t slabs = gram_slabs(M, max_slabs, &slab);
  if ((((uintptr_t)X | (uintptr_t)W) & 15) || (ldx & 3) || (ldw & 3)) return cudaErrorInvalidValue;
  k_gram_tiles<<<dim3(tiles, (unsigned)slabs), NT, 0, st>>>(X, ldx, W, ldw, M, d1, d2, sym, slab,
                                                            partial, gate);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = (int64_t)d1 * d2;
  k_gram_reduce<<<ceil_div(tot, 256), 256, 0, st>>>(partial, (int)slabs, d1, d2, sym, C, Cf, gate);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
