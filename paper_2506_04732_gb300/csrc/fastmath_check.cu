// t2s2_fastmath: runs the FP64 reciprocal and reciprocal square root of
// fastmath.cuh (binary32 seed, two binary64 Newton steps; IEEE operations
// outside the binary32 normal range) on a device array, so that they can be
// compared with correctly rounded results directly rather than only through
// the factorisations that use them.
#include <algorithm>

#include "api_internal.h"
#include "fastmath.cuh"

namespace t2s2 {
namespace {

__global__ void fastmath_kernel(const double* x, double* rs, double* rc, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (rs) rs[i] = drsqrt(v);
    if (rc) rc[i] = drcp(v);
  }
}

}  // namespace
}  // namespace t2s2

extern "C" t2s2_status t2s2_fastmath(const double* x, double* rsqrt_out, double* rcp_out, long n, void* stream) {
  if (n < 0 || (n > 0 && !x)) return T2S2_EINVAL;
  if (n == 0) return T2S2_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long blocks = std::min<long>((n + 255) / 256, 4096);
  t2s2::fastmath_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, rsqrt_out, rcp_out, n);
  T2S2_CUDA_TRY(cudaGetLastError());
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  return T2S2_OK;
}
