// Householder TSQR: the unconditionally stable orth() / qr() of a tall-skinny
// matrix (Section II-A, the unpivoted QR with diag(R) >= 0), taken when
// CholeskyQR cannot orthonormalise a sketch -- one that is numerically rank
// deficient at the working precision.  Communication-avoiding QR after
// Demmel, Grigori, Hoemmen and Langou (SIAM J. Sci. Comput. 2012):
//
//   1. the rows of Y are cut into P leaf blocks of at least d rows; one CTA
//      per leaf takes a Householder QR of its block (Golub & Van Loan,
//      Algorithm 5.2.1; v = x + sign(x_1) ||x|| e_1, sign(0) = +1);
//   2. the d x d R factors are merged pairwise up a binary tree: one CTA per
//      node takes the QR of its two stacked upper-triangular R's, whose
//      reflectors keep the lower block triangular (structured TSQR);
//   3. the explicit Q comes down the tree: the root's reflectors applied to
//      [I_d; 0], each node's to its parent's d-row block stacked on zeros,
//      and the leaves' to theirs, one CTA per (node, column block);
//   4. Q's columns take the signs of diag(R_root), so that diag(R) >= 0.
//
// Blocks that fit in 200 KB of shared memory are factored there, larger ones
// in place in global memory (slower; the same arithmetic).  Every reduction
// has a fixed order, so results are reproducible run to run.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace ruqlp {
namespace {

constexpr int TS_THREADS = 256;
constexpr int TS_WARPS = TS_THREADS / 32;
constexpr size_t TS_SMEM = 200 * 1024;

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA, the same value (same order) in every thread.
template <typename T> __device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  __syncthreads();  // red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int i = 0; i < TS_WARPS; ++i) s += red[i];
  return s;
}

// Householder reflector of x = (x0, rest) with ||x||^2 = nrm2: H = I - tau v
// v^T, v = (x0 - alpha, rest), H x = alpha e_1 with alpha = -sign(x0) ||x||.
template <typename T>
__device__ __forceinline__ void reflector(T x0, T nrm2, T& alpha, T& v0, T& tau) {
  const T nrm = sqrt(nrm2);
  alpha = (x0 >= T(0)) ? -nrm : nrm;
  v0 = x0 - alpha;
  tau = (nrm2 > T(0)) ? T(1) / (alpha * (alpha - x0)) : T(0);
}

// Householder QR of a dense column-major block M (rows x d, ld, rows >= d),
// in place: R on and above the diagonal (diag = alpha_j), the reflectors'
// tails below it; v0[j], tau[j], diag[j] per column.
template <typename T>
__device__ void house_dense(T* M, int64_t ld, int rows, int d, T* __restrict__ v0s,
                            T* __restrict__ taus, T* __restrict__ diag, T* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ T s_par[3];
  for (int j = 0; j < d; ++j) {
    T* cj = M + (int64_t)j * ld;
    T part = T(0);
    for (int i = j + tid; i < rows; i += TS_THREADS) part += cj[i] * cj[i];
    const T nrm2 = block_sum(part, red);
    if (tid == 0) {
      T alpha, v0, tau;
      reflector(cj[j], nrm2, alpha, v0, tau);
      s_par[0] = alpha;
      s_par[1] = v0;
      s_par[2] = tau;
    }
    __syncthreads();
    const T alpha = s_par[0], v0 = s_par[1], tau = s_par[2];
    if (tau != T(0)) {
      for (int c = j + 1 + warp; c < d; c += TS_WARPS) {
        T* cc = M + (int64_t)c * ld;
        const T top = cc[j];
        T dot = T(0);
        for (int i = j + 1 + lane; i < rows; i += 32) dot += cj[i] * cc[i];
        dot = warp_sum(dot) + v0 * top;
        const T f = tau * dot;
        __syncwarp();
        if (lane == 0) cc[j] = top - f * v0;
        for (int i = j + 1 + lane; i < rows; i += 32) cc[i] -= f * cj[i];
      }
    }
    __syncthreads();
    if (tid == 0) {
      cj[j] = alpha;
      v0s[j] = v0;
      taus[j] = tau;
      diag[j] = alpha;
    }
  }
  __syncthreads();
}

// Leaf i of P covers rows [i M / P, (i + 1) M / P) (at least d rows each).
__host__ __device__ inline int64_t leaf_row0(int64_t i, int64_t M, int64_t P) { return i * M / P; }

// ---- 0. Y (row-major) -> W (column-major, ld M) --------------------------
template <typename T>
__global__ void k_ts_load(const T* __restrict__ Y, int64_t ldy, int64_t M, int d,
                          T* __restrict__ W) {
  __shared__ T t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < M && c < d) ? Y[r * ldy + c] : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (c < d && r < M) W[(int64_t)c * M + r] = t[threadIdx.x][i];
  }
}

// ---- 1. leaf QRs ---------------------------------------------------------
template <typename T, bool SMEM>
__global__ void __launch_bounds__(TS_THREADS)
k_ts_leaf_qr(T* __restrict__ W, int64_t M, int d, int P, T* __restrict__ v0s,
             T* __restrict__ taus, T* __restrict__ diag) {
  extern __shared__ __align__(16) unsigned char ts_smem[];
  __shared__ T red[TS_WARPS];
  const int64_t r0 = leaf_row0(blockIdx.x, M, P), r1 = leaf_row0(blockIdx.x + 1, M, P);
  const int rows = (int)(r1 - r0);
  T* v0 = v0s + (int64_t)blockIdx.x * d;
  T* tau = taus + (int64_t)blockIdx.x * d;
  T* dg = diag + (int64_t)blockIdx.x * d;
  if (SMEM) {
    T* S = reinterpret_cast<T*>(ts_smem);
    for (int64_t e = threadIdx.x; e < (int64_t)rows * d; e += TS_THREADS) {
      const int c = (int)(e / rows), i = (int)(e % rows);
      S[e] = W[(int64_t)c * M + r0 + i];
    }
    __syncthreads();
    house_dense(S, rows, rows, d, v0, tau, dg, red);
    for (int64_t e = threadIdx.x; e < (int64_t)rows * d; e += TS_THREADS) {
      const int c = (int)(e / rows), i = (int)(e % rows);
      W[(int64_t)c * M + r0 + i] = S[e];
    }
  } else {
    house_dense(W + r0, M, rows, d, v0, tau, dg, red);
  }
}

// ---- 2. tree nodes: QR of two stacked upper-triangular R's -----------------
// A node's storage: the top triangle (its R afterwards, diagonal alpha) then
// the bottom triangle (the reflectors' tails), both packed column-major
// (column c holds rows 0..c at offset c (c + 1) / 2), then v0, tau, diag.
__host__ __device__ inline int64_t tri(int c) { return (int64_t)c * (c + 1) / 2; }
__host__ __device__ inline int64_t node_elems(int d) { return 2 * tri(d) + 3 * (int64_t)d; }

struct TsLevel {
  int n;           // nodes at this level
  int nchild;      // nodes (or leaves) at the level below
  int64_t off;     // element offset of node 0 in the tree buffer
  int64_t xoff;    // element offset of this level's Q blocks (2d x d each)
};

// Upper triangle of child c's R, element (i, col), i <= col.
template <typename T>
__device__ __forceinline__ T child_r(bool leaf_children, const T* W, int64_t M, int P,
                                     const T* tree, int64_t child_off, int d, int c, int i,
                                     int col) {
  if (leaf_children)
    return W[(int64_t)col * M + leaf_row0(c, M, P) + i];
  return tree[child_off + (int64_t)c * node_elems(d) + tri(col) + i];
}

template <typename T, bool SMEM>
__global__ void __launch_bounds__(TS_THREADS)
k_ts_node_qr(const T* __restrict__ W, int64_t M, int P, T* tree, TsLevel lv, int64_t child_off,
             int leaf_children, int d) {
  extern __shared__ __align__(16) unsigned char ts_smem[];
  __shared__ T s_par[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int node = blockIdx.x;
  T* gnode = tree + lv.off + (int64_t)node * node_elems(d);
  T* base = SMEM ? reinterpret_cast<T*>(ts_smem) : gnode;
  T* top = base;
  T* bot = base + tri(d);
  T* v0s = gnode + 2 * tri(d);
  T* taus = v0s + d;
  T* diag = taus + d;
  const int c0 = 2 * node, c1 = 2 * node + 1;
  const bool two = c1 < lv.nchild;
  // assemble: top <- R of child c0, bottom <- R of child c1 (or zero)
  for (int64_t e = tid; e < tri(d); e += TS_THREADS) {
    int col = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while (tri(col + 1) <= e) ++col;
    while (tri(col) > e) --col;
    const int i = (int)(e - tri(col));
    top[e] = child_r(leaf_children != 0, W, M, P, tree, child_off, d, c0, i, col);
    bot[e] = two ? child_r(leaf_children != 0, W, M, P, tree, child_off, d, c1, i, col) : T(0);
  }
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    if (two) {
      if (warp == 0) {
        // x = (top_jj, bot_0j .. bot_jj)
        T part = T(0);
        for (int i = lane; i <= j; i += 32) {
          const T b = bot[tri(j) + i];
          part += b * b;
        }
        part = warp_sum(part);
        if (lane == 0) {
          const T x0 = top[tri(j) + j];
          T alpha, v0, tau;
          reflector(x0, x0 * x0 + part, alpha, v0, tau);
          s_par[0] = alpha;
          s_par[1] = v0;
          s_par[2] = tau;
        }
      }
      __syncthreads();
      const T alpha = s_par[0], v0 = s_par[1], tau = s_par[2];
      if (tau != T(0)) {
        for (int c = j + 1 + warp; c < d; c += TS_WARPS) {
          const T tj = top[tri(c) + j];
          T dot = T(0);
          for (int i = lane; i <= j; i += 32) dot += bot[tri(j) + i] * bot[tri(c) + i];
          dot = warp_sum(dot) + v0 * tj;
          const T f = tau * dot;
          __syncwarp();
          if (lane == 0) top[tri(c) + j] = tj - f * v0;
          for (int i = lane; i <= j; i += 32) bot[tri(c) + i] -= f * bot[tri(j) + i];
        }
      }
      __syncthreads();
      if (tid == 0) {
        top[tri(j) + j] = alpha;
        v0s[j] = v0;
        taus[j] = tau;
        diag[j] = alpha;
      }
    } else if (tid == 0) {  // one child: its R passes through (H = I)
      v0s[j] = T(0);
      taus[j] = T(0);
      diag[j] = top[tri(j) + j];
    }
  }
  __syncthreads();
  if (SMEM)
    for (int64_t e = tid; e < 2 * tri(d); e += TS_THREADS) gnode[e] = base[e];
}

// ---- 3. explicit Q, top down ---------------------------------------------
// Column block width of the apply kernels.
template <typename T> struct TsCB { static constexpr int v = sizeof(T) == 8 ? 16 : 32; };

// X (2d x CB block of columns cb0..) = H_node [C; 0], C = the node's d-row
// block of its parent's X (or I_d at the root).  Warp w owns columns w, w +
// TS_WARPS, ... of the block and applies the reflectors j = d-1 .. 0 to them
// on its own (columns are independent).
template <typename T>
__global__ void __launch_bounds__(TS_THREADS)
k_ts_node_apply(const T* __restrict__ tree, TsLevel lv, const T* __restrict__ parent_x,
                int root, int d, T* __restrict__ xout) {
  constexpr int CB = TsCB<T>::v;
  extern __shared__ __align__(16) unsigned char ts_smem[];
  T* X = reinterpret_cast<T*>(ts_smem);  // [CB][2d]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int node = blockIdx.x, cb0 = blockIdx.y * CB;
  const int ncol = min(CB, d - cb0);
  const T* gnode = tree + lv.off + (int64_t)node * node_elems(d);
  const T* bot = gnode + tri(d);
  const T* v0s = gnode + 2 * tri(d);
  const T* taus = v0s + d;
  const int rows = 2 * d;
  // C: rows (node % 2) d .. + d of the parent's X (2d x d, ld 2d)
  const T* C = root ? nullptr : parent_x + (int64_t)(node / 2) * 2 * d * d + (node % 2) * d;
  for (int e = tid; e < CB * rows; e += TS_THREADS) {
    const int c = e / rows, i = e % rows;
    T v = T(0);
    if (c < ncol && i < d) v = root ? T(i == cb0 + c) : C[(int64_t)(cb0 + c) * rows + i];
    X[e] = v;
  }
  __syncthreads();
  for (int c = warp; c < ncol; c += TS_WARPS) {
    T* x = X + c * rows;
    for (int j = d - 1; j >= 0; --j) {
      const T tau = taus[j];
      if (tau == T(0)) continue;
      const T v0 = v0s[j];
      const T* bj = bot + tri(j);
      T dot = T(0);
      for (int i = lane; i <= j; i += 32) dot += bj[i] * x[d + i];
      dot = warp_sum(dot) + v0 * x[j];
      const T f = tau * dot;
      __syncwarp();
      if (lane == 0) x[j] -= f * v0;
      for (int i = lane; i <= j; i += 32) x[d + i] -= f * bj[i];
      __syncwarp();
    }
  }
  __syncthreads();
  T* out = xout + lv.xoff + (int64_t)node * rows * d;
  for (int e = tid; e < ncol * rows; e += TS_THREADS) {
    const int c = e / rows, i = e % rows;
    out[(int64_t)(cb0 + c) * rows + i] = X[e];
  }
}

// Leaf i: Q rows r0..r1 = H_leaf [C; 0] (C = the leaf's d-row block of its
// parent's X, or I_d when the leaf is the root), times the signs of the
// root's diagonal, written row-major to Q.
template <typename T>
__global__ void __launch_bounds__(TS_THREADS)
k_ts_leaf_apply(const T* __restrict__ W, int64_t M, int d, int P, const T* __restrict__ v0s,
                const T* __restrict__ taus, const T* __restrict__ parent_x,
                const T* __restrict__ root_diag, T* __restrict__ Q, int64_t ldq) {
  constexpr int CB = TsCB<T>::v;
  extern __shared__ __align__(16) unsigned char ts_smem[];
  T* X = reinterpret_cast<T*>(ts_smem);  // [CB][rows]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int leaf = blockIdx.x, cb0 = blockIdx.y * CB;
  const int ncol = min(CB, d - cb0);
  const int64_t r0 = leaf_row0(leaf, M, P), r1 = leaf_row0(leaf + 1, M, P);
  const int rows = (int)(r1 - r0);
  const bool root = P == 1;
  const T* C = root ? nullptr : parent_x + (int64_t)(leaf / 2) * 2 * d * d + (leaf % 2) * d;
  for (int e = tid; e < CB * rows; e += TS_THREADS) {
    const int c = e / rows, i = e % rows;
    T v = T(0);
    if (c < ncol && i < d) v = root ? T(i == cb0 + c) : C[(int64_t)(cb0 + c) * 2 * d + i];
    X[e] = v;
  }
  __syncthreads();
  const T* lv0 = v0s + (int64_t)leaf * d;
  const T* ltau = taus + (int64_t)leaf * d;
  for (int c = warp; c < ncol; c += TS_WARPS) {
    T* x = X + c * rows;
    for (int j = d - 1; j >= 0; --j) {
      const T tau = ltau[j];
      if (tau == T(0)) continue;
      const T v0 = lv0[j];
      const T* vj = W + (int64_t)j * M + r0;  // tail rows j+1 .. rows-1
      T dot = T(0);
      for (int i = j + 1 + lane; i < rows; i += 32) dot += vj[i] * x[i];
      dot = warp_sum(dot) + v0 * x[j];
      const T f = tau * dot;
      __syncwarp();
      if (lane == 0) x[j] -= f * v0;
      for (int i = j + 1 + lane; i < rows; i += 32) x[i] -= f * vj[i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * CB; e += TS_THREADS) {
    const int i = e / CB, c = e % CB;
    if (c < ncol) {
      const T s = root_diag[cb0 + c] < T(0) ? T(-1) : T(1);
      Q[(r0 + i) * ldq + cb0 + c] = s * X[c * rows + i];
    }
  }
}

// Tree geometry of a problem: leaves, levels and buffer offsets.
struct TsPlan {
  int P = 1;
  bool leaf_smem = false;
  std::vector<TsLevel> levels;
  size_t off_W, off_v0, off_tau, off_diag, off_tree, off_x, total;  // bytes
};

size_t ts_align(size_t x) { return (x + 255) / 256 * 256; }

TsPlan ts_plan(int64_t M, int d, size_t es) {
  TsPlan p;
  const int64_t bmax = (int64_t)(TS_SMEM / ((size_t)d * es));
  int64_t P = 1;
  if (bmax >= d) P = (M + bmax - 1) / bmax;
  P = std::max<int64_t>(1, std::min<int64_t>(P, M / d));
  // at least one leaf per 128-row block when d is small, for parallelism
  const int64_t b128 = std::max<int64_t>(128, d);
  P = std::max<int64_t>(P, std::min<int64_t>(M / b128, (int64_t)1 << 20));
  P = std::max<int64_t>(1, std::min<int64_t>(P, M / d));
  p.P = (int)P;
  const int64_t rows_max = (M + P - 1) / P;
  p.leaf_smem = (size_t)rows_max * d * es <= TS_SMEM;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = ts_align(off + b); return o; };
  p.off_W = take((size_t)M * d * es);
  p.off_v0 = take((size_t)P * d * es);
  p.off_tau = take((size_t)P * d * es);
  p.off_diag = take((size_t)P * d * es);
  int64_t elems = 0, xel = 0;
  int n = (int)P;
  while (n > 1) {
    TsLevel lv;
    lv.nchild = n;
    lv.n = (n + 1) / 2;
    lv.off = elems;
    lv.xoff = xel;
    elems += (int64_t)lv.n * node_elems(d);
    xel += (int64_t)lv.n * 2 * d * d;
    p.levels.push_back(lv);
    n = lv.n;
  }
  p.off_tree = take((size_t)std::max<int64_t>(elems, 1) * es);
  p.off_x = take((size_t)std::max<int64_t>(xel, 1) * es);
  p.total = off;
  return p;
}

template <typename T>
cudaError_t tsqr_run(const T* Y, int64_t ldy, int64_t M, int d, T* Q, int64_t ldq, char* work,
                     cudaStream_t st) {
  const TsPlan p = ts_plan(M, d, sizeof(T));
  T* W = (T*)(work + p.off_W);
  T* v0s = (T*)(work + p.off_v0);
  T* taus = (T*)(work + p.off_tau);
  T* diag = (T*)(work + p.off_diag);
  T* tree = (T*)(work + p.off_tree);
  T* xb = (T*)(work + p.off_x);
  cudaError_t e;
  {
    dim3 grid(ceil_div(M, 32), ceil_div(d, 32)), block(32, 8);
    k_ts_load<T><<<grid, block, 0, st>>>(Y, ldy, M, d, W);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int64_t rows_max = (M + p.P - 1) / p.P;
  if (p.leaf_smem) {
    const size_t sm = (size_t)rows_max * d * sizeof(T);
    e = cudaFuncSetAttribute(k_ts_leaf_qr<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TS_SMEM);
    if (e != cudaSuccess) return e;
    k_ts_leaf_qr<T, true><<<p.P, TS_THREADS, sm, st>>>(W, M, d, p.P, v0s, taus, diag);
  } else {
    k_ts_leaf_qr<T, false><<<p.P, TS_THREADS, 0, st>>>(W, M, d, p.P, v0s, taus, diag);
  }
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t node_sm = (size_t)2 * tri(d) * sizeof(T);
  const bool node_smem = node_sm <= TS_SMEM;
  for (size_t l = 0; l < p.levels.size(); ++l) {
    const TsLevel& lv = p.levels[l];
    const int64_t child_off = l == 0 ? 0 : p.levels[l - 1].off;
    if (node_smem) {
      e = cudaFuncSetAttribute(k_ts_node_qr<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TS_SMEM);
      if (e != cudaSuccess) return e;
      k_ts_node_qr<T, true><<<lv.n, TS_THREADS, node_sm, st>>>(W, M, p.P, tree, lv, child_off,
                                                               l == 0, d);
    } else {
      k_ts_node_qr<T, false><<<lv.n, TS_THREADS, 0, st>>>(W, M, p.P, tree, lv, child_off, l == 0,
                                                          d);
    }
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  constexpr int CB = TsCB<T>::v;
  const int ncb = ceil_div(d, CB);
  const size_t xsm = (size_t)CB * 2 * d * sizeof(T);
  if (xsm > TS_SMEM) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_ts_node_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TS_SMEM);
  if (e != cudaSuccess) return e;
  for (int l = (int)p.levels.size() - 1; l >= 0; --l) {
    const TsLevel& lv = p.levels[l];
    const bool root = l == (int)p.levels.size() - 1;
    const T* parent = root ? nullptr : xb + p.levels[l + 1].xoff;
    k_ts_node_apply<T><<<dim3(lv.n, ncb), TS_THREADS, xsm, st>>>(tree, lv, parent, root ? 1 : 0,
                                                                d, xb);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const size_t lsm = (size_t)CB * rows_max * sizeof(T);
  if (lsm > TS_SMEM) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_ts_leaf_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TS_SMEM);
  if (e != cudaSuccess) return e;
  const T* root_diag = p.levels.empty()
                           ? diag
                           : tree + p.levels.back().off + 2 * tri(d) + 2 * (int64_t)d;
  const T* parent = p.levels.empty() ? nullptr : xb + p.levels[0].xoff;
  k_ts_leaf_apply<T><<<dim3(p.P, ncb), TS_THREADS, lsm, st>>>(W, M, d, p.P, v0s, taus, parent,
                                                             root_diag, Q, ldq);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

size_t tsqr_work_bytes(Ty t, int64_t M, int d) {
  if (M < 1 || d < 1 || M < d) return 0;
  return ts_plan(M, d, ty_size(t)).total;
}

bool tsqr_supported(Ty t, int64_t M, int d) {
  if (M < d || d < 1 || (t != Ty::F32 && t != Ty::F64)) return false;
  const TsPlan p = ts_plan(M, d, ty_size(t));
  const size_t es = ty_size(t);
  const size_t cb = t == Ty::F64 ? 16 : 32;
  const int64_t rows_max = (M + p.P - 1) / p.P;
  return cb * 2 * d * es <= TS_SMEM && cb * rows_max * es <= TS_SMEM;
}

cudaError_t tsqr(Ty t, const void* Y, int64_t ldy, int64_t M, int d, void* Q, int64_t ldq,
                 void* work, cudaStream_t st) {
  if (!tsqr_supported(t, M, d)) return cudaErrorInvalidValue;
  if (t == Ty::F64)
    return tsqr_run<double>((const double*)Y, ldy, M, d, (double*)Q, ldq, (char*)work, st);
  return tsqr_run<float>((const float*)Y, ldy, M, d, (float*)Q, ldq, (char*)work, st);
}

}  // namespace ruqlp
