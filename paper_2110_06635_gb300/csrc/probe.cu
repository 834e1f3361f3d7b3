// Atomic-throughput probe: a measurement aid, not part of the method.  The
// depth and accumulate passes are bound by L2 atomics on per-pixel buffers,
// so their roofline needs the rate at which this GPU completes atomics on a
// buffer of the same size; this kernel issues `ops` atomics of one kind at
// uniformly random elements of a caller-owned buffer, for the caller to time.
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {
namespace {

// SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014): a well-mixed 64-bit hash of k.
__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k += 0x9E3779B97F4A7C15ull;
  k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
  k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
  return k ^ (k >> 31);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_atomic_probe(void* buf, uint32_t elems, int64_t ops, uint64_t seed) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ops; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed + (uint64_t)k);
    const uint32_t e = (uint32_t)(((h >> 32) * (uint64_t)elems) >> 32);  // uniform in [0, elems)
    if constexpr (KIND == 0) {
      atomicMin(reinterpret_cast<unsigned long long*>(buf) + e, (unsigned long long)h);
    } else if constexpr (KIND == 1) {
      atomicAdd(reinterpret_cast<unsigned int*>(buf) + e, 1u);
    } else if constexpr (KIND == 2) {
      atomicAdd(reinterpret_cast<float4*>(buf) + e, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
    } else {
      atomicAdd(reinterpret_cast<float*>(buf) + e, 1.0f);
    }
  }
}

}  // namespace
}  // namespace adop

using namespace adop;

extern "C" adop_status adop_atomic_probe(int32_t kind, void* buf, int64_t elems, int64_t ops, uint64_t seed,
                                         adop_stream stream) {
  if (kind < 0 || kind > 3) {
    set_last_error("kind outside [0, 3]");
    return ADOP_ERR_INVALID_ARG;
  }
  if (!buf || elems < 1 || elems > 0xFFFFFFFFll || ops < 0) {
    set_last_error("buf must be non-NULL, elems in [1, 2^32), ops >= 0");
    return ADOP_ERR_INVALID_ARG;
  }
  const uintptr_t align = kind == 2 ? 16 : (kind == 0 ? 8 : 4);
  if (((uintptr_t)buf & (align - 1)) != 0) {
    set_last_error("buf misaligned for the kind's element size");
    return ADOP_ERR_INVALID_ARG;
  }
  if (ops == 0) return ADOP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t want = (ops + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 16;
  const dim3 grid((unsigned)(want < cap ? want : cap));
  const uint32_t n = (uint32_t)elems;
  switch (kind) {
    case 0: k_atomic_probe<0><<<grid, kThreads, 0, s>>>(buf, n, ops, seed); break;
    case 1: k_atomic_probe<1><<<grid, kThreads, 0, s>>>(buf, n, ops, seed); break;
    case 2: k_atomic_probe<2><<<grid, kThreads, 0, s>>>(buf, n, ops, seed); break;
    default: k_atomic_probe<3><<<grid, kThreads, 0, s>>>(buf, n, ops, seed); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return ADOP_ERR_CUDA;
  }
  return ADOP_OK;
}
