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

#define T2S2_TRY(expr)                 \
  do {                                 \
    t2s2_status _s = (expr);           \
    if (_s != T2S2_OK) return _s;      \
  } while (0)

namespace t2s2 {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }
constexpr int kNumSMs = 152;
}  // namespace t2s2
