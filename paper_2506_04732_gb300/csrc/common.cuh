// Shared helpers for the sm_103a kernels and their host launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdint>

#include "../../include/t2s2.h"

#define T2S2_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      t2s2::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return (_e == cudaErrorMemoryAllocation) ? T2S2_ENOMEM : T2S2_ECUDA; \
    }                                                         \
  } while (0)

// With T2S2_VERBOSE=1 every level a failure passes through is printed to
// stderr (innermost first); the check costs nothing on the success path.
#define T2S2_TRY(expr)                                      \
  do {                                                      \
    t2s2_status _s = (expr);                                \
    if (_s != T2S2_OK) {                                    \
      t2s2::note_failure(_s, #expr, __FILE__, __LINE__);    \
      return _s;                                            \
    }                                                       \
  } while (0)

namespace t2s2 {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void note_failure(int status, const char* what, const char* file, int line);

// Programmatic dependent launch.  A kernel started by launch_pdl may begin
// (its CTAs become resident) while the previous kernel of its stream is still
// running.  Such a kernel calls pdl_wait() before its first global memory
// access; the wait returns once that previous kernel has completed and its
// writes are visible, so memory order stays plain stream order and only the
// launch itself overlaps.  pdl_trigger() lets the next dependent kernel start
// launching; both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// T2S2_PDL=0 turns the attribute off (every launch_pdl is then a plain launch).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }
constexpr int kNumSMs = 152;
}  // namespace t2s2
