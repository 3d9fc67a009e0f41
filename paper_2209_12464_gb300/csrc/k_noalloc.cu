// Gram entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a Gram matrix:
// code that is recording a CUDA graph (an allocation inside stream capture is
// refused), host programs whose own memory manager owns the whole device and
// forbids allocations it does not account for, and latency-critical loops
// where the implicit synchronisation of cudaMalloc/cudaFree is unacceptable.
// ruqlp_gram_noalloc computes the same G = Y^T Y as ruqlp_gram with the same
// split-K kernel, but its FP64 partial sums live in a fixed device array
// compiled into the library instead of a handle's workspace arena.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "../../include/ruqlp.h"
#include "internal.h"

namespace {

// Scratch for the FP64 partial Grams: 4 MiB, i.e. ruqlp_gram_noalloc's stated
// maximum.  Every GPU that loads the library holds this array until the
// process exits.
constexpr int64_t kScratchDoubles = 524288;
constexpr int kMaxD = 256;
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The calling thread's current CUDA context (driver entry point, looked up
// once); nullptr when it cannot be read.
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuCtxGetCurrent_v4000)ptr;
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the calling thread's current device,
// looked up with that device current the first time it is used there, and
// again whenever the device's context has changed since (a cudaDeviceReset
// tears the context down and reloads the module, which can move the array).
// In host code the name g_gram_scratch is only a host-side stand-in, so
// kernels must be given this address instead.
ruqlp_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RUQLP_ERR_CUDA;
  // (before the runtime has made a context current there is none: then the
  // lookup below creates it and the next call records it)
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev] || ctx == nullptr || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || !p) return RUQLP_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return RUQLP_OK;
}

}  // namespace

extern "C" ruqlp_status ruqlp_gram_noalloc(const void* Y, int64_t M, int d, int64_t ldy,
                                           ruqlp_dtype dtype, double* G, void* cuda_stream) {
  using namespace ruqlp;
  if (!Y || !G || M < 1 || d < 1 || ldy < d) return RUQLP_ERR_INVALID;
  if (dtype != RUQLP_F64 && dtype != RUQLP_F32) return RUQLP_ERR_INVALID;
  if (d > kMaxD) return RUQLP_ERR_BUDGET;
  double* scratch = nullptr;
  const ruqlp_status s = scratch_address(&scratch);
  if (s != RUQLP_OK) return s;
  const Ty ty = dtype == RUQLP_F64 ? Ty::F64 : Ty::F32;
  int splits = tn_splits(d, M, d, 64);
  const int64_t fit = kScratchDoubles / ((int64_t)d * d);
  if (splits > fit) splits = (int)fit;
  // Every slab writes all d x d entries of its partial, so nothing in the
  // scratch has to start at zero; the previous call's contents are overwritten.
  const cudaError_t e = simt_gemm_tn(ty, ty, Ty::F64, Mul::F64, Y, ldy, Y, ldy, G, d, d, M, d,
                                     splits, scratch, nullptr, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? RUQLP_OK : RUQLP_ERR_CUDA;
}
