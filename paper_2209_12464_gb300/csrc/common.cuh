// Shared definitions of the RU-QLP CUDA library (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <utility>

namespace ruqlp {

// Element type of a buffer inside the library.
enum class Ty : int { F64 = 0, F32 = 1, BF16 = 2 };

inline size_t ty_size(Ty t) { return t == Ty::F64 ? 8 : (t == Ty::F32 ? 4 : 2); }

// Device status word written by kernels (one per decomposition).
struct DevStatus {
  int32_t flags;      // RUQLP_FLAG_* bits
  int32_t breakdown;  // non-zero: an orth() failed after its fallbacks
  int32_t shifted;    // set by the Cholesky of the current orth when it shifted
  int32_t timeout;    // a bounded device wait ran out
  int32_t invalid;    // input checks on the device (CSR structure) failed
  int32_t pad[3];
};

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename T> struct Cvt;
template <> struct Cvt<float> {
  template <typename S> __device__ __forceinline__ static float from(S v) { return to_f32(v); }
};
template <> struct Cvt<double> {
  __device__ __forceinline__ static double from(double v) { return v; }
  __device__ __forceinline__ static double from(float v) { return (double)v; }
  __device__ __forceinline__ static double from(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
  }
};
template <> struct Cvt<__nv_bfloat16> {
  __device__ __forceinline__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  __device__ __forceinline__ static __nv_bfloat16 from(double v) {
    return __float2bfloat16_rn((float)v);
  }
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Programmatic dependent launch along the orth() / product chain: a kernel
// lets its successor start (launch_dependents) once its own resources (TMEM)
// are held, and waits for its predecessor's completion and memory (wait)
// before touching global memory.  Both are no-ops for a kernel launched
// without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialization (the kernel may start while
// its predecessor in the stream finishes; it waits in pdl_wait()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Process-wide count of kernels this library has launched (read through the
// ABI to report how many of the library's kernels a timed region ran).
void count_launch(int n = 1);
int64_t launch_count();

}  // namespace ruqlp
