// t2s2_tt_fibre: the values of a TT along one mode with the other indices
// fixed, X(i_0, .., i_k = t, .., i_{d-1}) for every t (eq.
// TT-format:elementwise: the product of the core slices).  One CTA: the slice
// products left and right of mode k as vector-matrix products in shared
// memory, then one value per thread.
#include <algorithm>

#include "api_internal.h"

namespace t2s2 {
namespace {

struct FibreArgs {
  const double* c[T2S2_MAX_D];
  int r[T2S2_MAX_D + 1];
  int m[T2S2_MAX_D];
  int idx[T2S2_MAX_D];
  int d, mode, rmax;
  double* out;
};

__global__ void fibre_kernel(FibreArgs a) {
  extern __shared__ double sh[];
  double* lv = sh;               // left vector, r[mode] entries
  double* rv = sh + a.rmax;      // right vector, r[mode + 1] entries
  double* tv = sh + 2 * a.rmax;  // scratch
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) lv[0] = 1.0, rv[0] = 1.0;
  __syncthreads();
  // left: v <- v G_k[:, idx_k, :] for k < mode
  for (int k = 0; k < a.mode; ++k) {
    const int ra = a.r[k], rb = a.r[k + 1], m = a.m[k], i = a.idx[k];
    for (int b = t; b < rb; b += nt) {
      double s = 0.0;
      for (int q = 0; q < ra; ++q) s = fma(lv[q], a.c[k][((long)q * m + i) * rb + b], s);
      tv[b] = s;
    }
    __syncthreads();
    for (int b = t; b < rb; b += nt) lv[b] = tv[b];
    __syncthreads();
  }
  // right: v <- G_k[:, idx_k, :] v for k > mode, from the last core inwards
  for (int k = a.d - 1; k > a.mode; --k) {
    const int ra = a.r[k], rb = a.r[k + 1], m = a.m[k], i = a.idx[k];
    for (int q = t; q < ra; q += nt) {
      double s = 0.0;
      for (int b = 0; b < rb; ++b) s = fma(a.c[k][((long)q * m + i) * rb + b], rv[b], s);
      tv[q] = s;
    }
    __syncthreads();
    for (int q = t; q < ra; q += nt) rv[q] = tv[q];
    __syncthreads();
  }
  const int k = a.mode, ra = a.r[k], rb = a.r[k + 1], m = a.m[k];
  for (int i = t; i < m; i += nt) {
    double s = 0.0;
    for (int q = 0; q < ra; ++q) {
      const double* g = a.c[k] + ((long)q * m + i) * rb;
      double u = 0.0;
      for (int b = 0; b < rb; ++b) u = fma(g[b], rv[b], u);
      s = fma(lv[q], u, s);
    }
    a.out[i] = s;
  }
}

}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" t2s2_status t2s2_tt_fibre(t2s2_op op, const t2s2_tt* x, int mode, const int* idx, double* out,
                                     void* stream) {
  if (!op || !x || !idx || !out) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, x));
  if (mode < 0 || mode >= x->d) return T2S2_EINVAL;
  int rmax = 1;
  for (int k = 0; k <= x->d; ++k) rmax = std::max(rmax, x->r[k]);
  for (int k = 0; k < x->d; ++k)
    if (k != mode && (idx[k] < 0 || idx[k] >= x->m[k])) return T2S2_EINVAL;
  const size_t smem = 3 * (size_t)rmax * sizeof(double);
  if (smem > 200 * 1024) return T2S2_EINVAL;
  T2S2_TRY(ensure_arena(op, tt_bytes(x) + sizeof(double) * x->m[mode] + ((size_t)1 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT dx;
  T2S2_TRY(bind_tt(cx, x, dx, true));
  double* dout = aget<double>(cx, x->m[mode]);
  if (!dout) return T2S2_ENOMEM;
  FibreArgs a;
  a.d = x->d;
  a.mode = mode;
  a.rmax = rmax;
  a.out = dout;
  for (int k = 0; k <= x->d; ++k) a.r[k] = x->r[k];
  for (int k = 0; k < x->d; ++k) {
    a.c[k] = dx.c[k];
    a.m[k] = x->m[k];
    a.idx[k] = k == mode ? 0 : idx[k];
  }
  static bool attr = false;
  if (!attr) {
    T2S2_CUDA_TRY(cudaFuncSetAttribute(fibre_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  fibre_kernel<<<1, 256, smem, cx.st>>>(a);
  T2S2_CUDA_TRY(cudaGetLastError());
  T2S2_CUDA_TRY(cudaMemcpyAsync(out, dout, sizeof(double) * x->m[mode], cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  return T2S2_OK;
}
