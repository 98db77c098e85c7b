// FP64 reciprocal and reciprocal square root for latency-bound single-CTA
// kernels.  GB300 runs FP64 at 2 DFMA/clk/SM, so IEEE double division and
// square root (long FP64 instruction sequences) dominate the small Jacobi and
// Cholesky kernels.  Here the FP32 hardware approximation gives a seed with
// ~23 correct bits and two Newton-Raphson steps in FP64 (each squares the
// relative error) bring it to full double precision:
//     rsqrt: y <- y (3 - x y^2) / 2,      rcp: y <- y (2 - x y).
// Inputs outside the FP32 normal range fall back to IEEE FP64 operations.
#pragma once

namespace t2s2 {

__device__ __forceinline__ bool f32_range(double x) {
  const double ax = fabs(x);
  return ax > 1e-36 && ax < 1e36;
}

__device__ __forceinline__ double drsqrt(double x) {
  if (!(x > 0.0) || !f32_range(x)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double hx = 0.5 * x;
  y = y * fma(-hx * y, y, 1.5);
  y = y * fma(-hx * y, y, 1.5);
  return y;
}

__device__ __forceinline__ double dsqrt(double x) {
  if (x == 0.0) return 0.0;
  return x * drsqrt(x);
}

__device__ __forceinline__ double drcp(double x) {
  if (!f32_range(x)) return 1.0 / x;
  double y = (double)__frcp_rn((float)x);
  y = y * fma(-x, y, 2.0);
  y = y * fma(-x, y, 2.0);
  return y;
}

}  // namespace t2s2
