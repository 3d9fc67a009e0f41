// Device generation of the Gaussian test matrix Omega (philox.cuh).
#include <algorithm>

#include "internal.h"
#include "philox.cuh"

namespace ruqlp {
namespace {

// out[i * ldo + j] = Omega_ij, i < n, j < d (FP64, row-major).
__global__ void k_omega_philox(uint64_t seed, int64_t n, int d, double* __restrict__ out,
                               int64_t ldo) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < d; j += blockDim.x) out[i * ldo + j] = omega_entry(seed, i, j);
}

}  // namespace

cudaError_t omega_philox(uint64_t seed, int64_t n, int d, double* out, int64_t ldo,
                         cudaStream_t st) {
  if (n <= 0 || d <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>(n, 152 * 32);
  k_omega_philox<<<grid, 128, 0, st>>>(seed, n, d, out, ldo);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ruqlp
