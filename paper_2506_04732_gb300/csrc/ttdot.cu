// TT inner products <u_p, v_p> (up to kMaxDots of them) in ONE cooperative
// launch.
//
// The residual screens of the solver need <b, y>, <y, y> and <b, b> (y = A x)
// at once.  As separate GEMM chains they cost two launches per core and
// product plus a host read-back each; here every product's left-to-right
// contraction (Methods: TT inner products through the interface matrices)
// runs in the same grid, with two grid barriers per core:
//
//   stage 1:  W_p[a', i, b]  = sum_a        phi_p[a, a'] U_p[a, i, b]
//   stage 2:  phi_p[b, b']   = sum_{a', i}  W_p[a', i, b] V_p[a', i, b']
//
// starting from phi_p = 1 and ending with the 1 x 1 phi_p = <u_p, v_p>.
// Stage 1 gives each W entry to one thread (two accumulators), stage 2 each
// phi entry to one warp (lanes over (a', i), then a fixed shuffle tree), so
// the sums are taken in an order that does not depend on timing.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "api_internal.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int kDotThreads = 256;
constexpr int kMaxDots = 4;

struct DotArgs {
  int n, d;
  int m[T2S2_MAX_D];
  int ru[kMaxDots][T2S2_MAX_D + 1], rv[kMaxDots][T2S2_MAX_D + 1];
  const double* u[kMaxDots][T2S2_MAX_D];
  const double* v[kMaxDots][T2S2_MAX_D];
  double* phi[kMaxDots];  // ru_k x rv_k
  double* w[kMaxDots];    // rv_k x m_k x ru_{k+1}
  double* out;            // n values
};

__global__ void __launch_bounds__(kDotThreads) tt_dots_kernel(DotArgs a) {
  pdl_trigger();
  cg::grid_group grid = cg::this_grid();
  const long gt = (long)blockIdx.x * kDotThreads + threadIdx.x;
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < a.d; ++k) {
    const int m = a.m[k];
    long tot = 0;
    for (int p = 0; p < a.n; ++p) tot += (long)a.rv[p][k] * m * a.ru[p][k + 1];
    for (long slot = threadIdx.x;; slot += kDotThreads) {
      const long e = slot * gridDim.x + blockIdx.x;  // item j on CTA j mod G
      if (e >= tot) break;
      int p = 0;
      long q = e;
      while (q >= (long)a.rv[p][k] * m * a.ru[p][k + 1]) q -= (long)a.rv[p][k] * m * a.ru[p][k + 1], ++p;
      const int ra = a.ru[p][k], rb = a.ru[p][k + 1], sa = a.rv[p][k];
      const int b = (int)(q % rb);
      const long ai = q / rb;  // a' * m + i
      const int i = (int)(ai % m), ap = (int)(ai / m);
      const double* U = a.u[p][k];
      double s0 = 0.0, s1 = 0.0;
      if (k == 0) {
        s0 = U[(long)i * rb + b];  // phi = 1, ra = sa = 1
      } else {
        const double* ph = a.phi[p];
        int x = 0;
        for (; x + 1 < ra; x += 2) {
          s0 = fma(ph[(long)x * sa + ap], U[((long)x * m + i) * rb + b], s0);
          s1 = fma(ph[(long)(x + 1) * sa + ap], U[((long)(x + 1) * m + i) * rb + b], s1);
        }
        if (x < ra) s0 = fma(ph[(long)x * sa + ap], U[((long)x * m + i) * rb + b], s0);
      }
      a.w[p][q] = s0 + s1;
    }
    grid.sync();
    long tot2 = 0;
    for (int p = 0; p < a.n; ++p) tot2 += (long)a.ru[p][k + 1] * a.rv[p][k + 1];
    for (long slot = threadIdx.x >> 5;; slot += kDotThreads / 32) {
      const long it = slot * gridDim.x + blockIdx.x;
      if (it >= tot2) break;
      int p = 0;
      long q = it;
      while (q >= (long)a.ru[p][k + 1] * a.rv[p][k + 1]) q -= (long)a.ru[p][k + 1] * a.rv[p][k + 1], ++p;
      const int rb = a.ru[p][k + 1], sb = a.rv[p][k + 1], sa = a.rv[p][k];
      const int b = (int)(q / sb), bp = (int)(q % sb);
      const double* W = a.w[p];
      const double* V = a.v[p][k];
      const int K = sa * m;
      double s0 = 0.0, s1 = 0.0;
      int x = lane;
      for (; x + 32 < K; x += 64) {
        s0 = fma(W[(long)x * rb + b], V[(long)x * sb + bp], s0);
        s1 = fma(W[(long)(x + 32) * rb + b], V[(long)(x + 32) * sb + bp], s1);
      }
      if (x < K) s0 = fma(W[(long)x * rb + b], V[(long)x * sb + bp], s0);
      double s = s0 + s1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) a.phi[p][q] = s;
    }
    grid.sync();
  }
  if (gt < a.n) a.out[gt] = a.phi[gt][0];
}

// ---------------------------------------------------------------------------
// <u, v> in double-double arithmetic: every product of binary64 inputs is
// split exactly (p + e = a b through an FMA) and every sum is an error-free
// two-sum, so the environments carry ~2^-104 relative precision.  The
// residual |b - A x|^2 = |b|^2 - 2<b, A x> + |A x|^2 has terms of the size
// |b|^2 while the result is many orders smaller; in binary64 the cancellation
// leaves noise of ~1e-16 |b|^2, in double-double ~1e-28 |b|^2, so a residual
// of 1e-12 |b| comes out to about four digits.  When v is u the environments
// are symmetric and only their upper triangles are computed.

struct DDArgs {
  int n, d;
  int m[T2S2_MAX_D];
  int r[kMaxDots][T2S2_MAX_D + 1];   // ranks of u_p
  int s[kMaxDots][T2S2_MAX_D + 1];   // ranks of v_p
  int sym[kMaxDots];                 // 1: v_p is u_p (phi symmetric)
  const double* u[kMaxDots][T2S2_MAX_D];
  const double* v[kMaxDots][T2S2_MAX_D];
  double* phh[kMaxDots];  // phi, high and low parts (r_k x s_k)
  double* phl[kMaxDots];
  double* wh[kMaxDots];   // W, high and low parts (s_k x m_k x r_{k+1})
  double* wl[kMaxDots];
  double* out;            // n (hi, lo) pairs
};

// The error-free steps use explicitly rounded operations, which the compiler
// never fuses into an FMA (a fused a*b + c would break the exact splits).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// (hi, lo) += (xh + xl) y
__device__ __forceinline__ void dd_fma(double& hi, double& lo, double xh, double xl, double y) {
  const double p = __dmul_rn(xh, y);
  double pe = fma(xh, y, -p);
  pe = fma(xl, y, pe);
  double s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __dadd_rn(lo, __dadd_rn(e, pe));
}

__device__ __forceinline__ void dd_add(double& hi, double& lo, double h2, double l2) {
  double s, e;
  two_sum(hi, h2, s, e);
  hi = s;
  lo = __dadd_rn(lo, __dadd_rn(l2, e));
}

// Item j of a stage goes to CTA j mod G: the binary64 work of the items
// spreads over every SM instead of filling the first CTAs.
__device__ __forceinline__ long spread_item(long slot, int G, int g) { return slot * G + g; }

// number of phi entries computed for product p at bond k+1: the upper
// triangle when phi is symmetric
__device__ __forceinline__ long dd_phi_items(const DDArgs& a, int p, int k) {
  const long r1 = a.r[p][k + 1], s1 = a.s[p][k + 1];
  return a.sym[p] ? r1 * (r1 + 1) / 2 : r1 * s1;
}

__global__ void __launch_bounds__(kDotThreads) tt_norm2_dd_kernel(DDArgs a) {
  pdl_trigger();
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x, g = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < a.d; ++k) {
    const int m = a.m[k];
    long tot = 0;
    for (int p = 0; p < a.n; ++p) tot += (long)a.s[p][k] * m * a.r[p][k + 1];
    // W[a', i, b] = sum_a phi[a, a'] U[a, i, b]
    for (long slot = threadIdx.x;; slot += kDotThreads) {
      const long e = spread_item(slot, G, g);
      if (e >= tot) break;
      int p = 0;
      long q = e;
      while (q >= (long)a.s[p][k] * m * a.r[p][k + 1]) q -= (long)a.s[p][k] * m * a.r[p][k + 1], ++p;
      const int ra = a.r[p][k], rb = a.r[p][k + 1], sa = a.s[p][k];
      const int b = (int)(q % rb);
      const int ai = (int)(q / rb);
      const int i = ai % m, ap = ai / m;
      const double* U = a.u[p][k];
      double h0 = 0.0, l0 = 0.0, h1 = 0.0, l1 = 0.0;
      if (k == 0) {
        h0 = U[(long)i * rb + b];
      } else {
        const double *ph = a.phh[p], *pl = a.phl[p];
        int x = 0;
        for (; x + 1 < ra; x += 2) {
          dd_fma(h0, l0, ph[(long)x * sa + ap], pl[(long)x * sa + ap], U[((long)x * m + i) * rb + b]);
          dd_fma(h1, l1, ph[(long)(x + 1) * sa + ap], pl[(long)(x + 1) * sa + ap],
                 U[((long)(x + 1) * m + i) * rb + b]);
        }
        if (x < ra) dd_fma(h0, l0, ph[(long)x * sa + ap], pl[(long)x * sa + ap], U[((long)x * m + i) * rb + b]);
        dd_add(h0, l0, h1, l1);
      }
      a.wh[p][q] = h0;
      a.wl[p][q] = l0;
    }
    grid.sync();
    // phi[b, b'] = sum_{a', i} W[a', i, b] V[a', i, b'] (upper triangle only
    // when V is U; both halves are written)
    long tot2 = 0;
    for (int p = 0; p < a.n; ++p) tot2 += dd_phi_items(a, p, k);
    for (long slot = warp;; slot += kDotThreads / 32) {
      const long it = spread_item(slot, G, g);
      if (it >= tot2) break;
      int p = 0;
      long q = it;
      while (q >= dd_phi_items(a, p, k)) q -= dd_phi_items(a, p, k), ++p;
      const int rb = a.r[p][k + 1], sb = a.s[p][k + 1], sa = a.s[p][k];
      int b, bp;
      if (a.sym[p]) {
        // q -> (b, b') with b <= b', row-major over the upper triangle
        b = (int)((2.0f * rb + 1.0f - sqrtf((2.0f * rb + 1.0f) * (2.0f * rb + 1.0f) - 8.0f * (float)q)) * 0.5f);
        b = max(0, min(rb - 1, b));
        while (b > 0 && (long)b * (2 * rb - b + 1) / 2 > q) --b;
        while ((long)(b + 1) * (2 * rb - b) / 2 <= q) ++b;
        bp = b + (int)(q - (long)b * (2 * rb - b + 1) / 2);
      } else {
        b = (int)(q / sb);
        bp = (int)(q % sb);
      }
      const double *Wh = a.wh[p], *Wl = a.wl[p];
      const double* V = a.v[p][k];
      const int K = sa * m;
      double h0 = 0.0, l0 = 0.0, h1 = 0.0, l1 = 0.0;
      int x = lane;
      for (; x + 32 < K; x += 64) {
        dd_fma(h0, l0, Wh[(long)x * rb + b], Wl[(long)x * rb + b], V[(long)x * sb + bp]);
        dd_fma(h1, l1, Wh[(long)(x + 32) * rb + b], Wl[(long)(x + 32) * rb + b], V[(long)(x + 32) * sb + bp]);
      }
      if (x < K) dd_fma(h0, l0, Wh[(long)x * rb + b], Wl[(long)x * rb + b], V[(long)x * sb + bp]);
      dd_add(h0, l0, h1, l1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double h2 = __shfl_xor_sync(0xffffffffu, h0, o), l2 = __shfl_xor_sync(0xffffffffu, l0, o);
        dd_add(h0, l0, h2, l2);
      }
      if (lane == 0) {
        double sh, se;
        two_sum(h0, l0, sh, se);  // renormalise
        a.phh[p][(long)b * sb + bp] = sh;
        a.phl[p][(long)b * sb + bp] = se;
        if (a.sym[p]) {
          a.phh[p][(long)bp * sb + b] = sh;
          a.phl[p][(long)bp * sb + b] = se;
        }
      }
    }
    grid.sync();
  }
  if (g == 0 && threadIdx.x < a.n) {
    a.out[2 * threadIdx.x] = a.phh[threadIdx.x][0];
    a.out[2 * threadIdx.x + 1] = a.phl[threadIdx.x][0];
  }
}

}  // namespace

t2s2_status tt_dots_dd(Ctx& cx, int n, const DevTT* const* u, const DevTT* const* v, double* hi, double* lo) {
  if (n < 1 || n > kMaxDots) return T2S2_EINVAL;
  const int d = u[0]->d;
  DDArgs a;
  a.n = n;
  a.d = d;
  for (int k = 0; k < d; ++k) a.m[k] = u[0]->m[k];
  size_t mark = cx.ar->mark();
  double fl = 0.0;
  for (int p = 0; p < n; ++p) {
    if (u[p]->d != d || v[p]->d != d) return T2S2_EINVAL;
    a.sym[p] = (u[p] == v[p]) ? 1 : 0;
    size_t phi_n = 1, w_n = 1;
    for (int k = 0; k < d; ++k) {
      if (u[p]->m[k] != a.m[k] || v[p]->m[k] != a.m[k]) return T2S2_EINVAL;
      a.u[p][k] = u[p]->c[k];
      a.v[p][k] = v[p]->c[k];
      phi_n = std::max(phi_n, (size_t)u[p]->r[k + 1] * v[p]->r[k + 1]);
      w_n = std::max(w_n, (size_t)v[p]->r[k] * a.m[k] * u[p]->r[k + 1]);
      fl += 2.0 * v[p]->r[k] * a.m[k] * (double)u[p]->r[k + 1] * (u[p]->r[k] + v[p]->r[k + 1]);
    }
    for (int k = 0; k <= d; ++k) {
      a.r[p][k] = u[p]->r[k];
      a.s[p][k] = v[p]->r[k];
    }
    a.phh[p] = aget<double>(cx, phi_n);
    a.phl[p] = aget<double>(cx, phi_n);
    a.wh[p] = aget<double>(cx, w_n);
    a.wl[p] = aget<double>(cx, w_n);
    if (!a.phh[p] || !a.phl[p] || !a.wh[p] || !a.wl[p]) return T2S2_ENOMEM;
  }
  a.out = aget<double>(cx, 2 * (size_t)n);
  if (!a.out) return T2S2_ENOMEM;
  int dev = 0, sms = 0, per_sm = 0;
  T2S2_CUDA_TRY(cudaGetDevice(&dev));
  T2S2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_norm2_dd_kernel, kDotThreads, 0));
  long cap = std::min<long>((long)std::max(1, per_sm) * sms, sms);
  if (cx.coop_ctas > 0) cap = std::min<long>(cap, cx.coop_ctas);
  // ~11 binary64 operations per product term: binary64 issue, not the item
  // count, sets the time, so every SM takes a share
  const int G = (int)std::max(1L, cap);
  {
    TraceScope ts(kTrDots, cx.st, fl, 0.0);  // algorithmic: 2 per product term
    void* args[] = {&a};
    T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)tt_norm2_dd_kernel, dim3(G), dim3(kDotThreads), args, 0,
                                              cx.st));
  }
  T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, a.out, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  for (int p = 0; p < n; ++p) {
    hi[p] = cx.hbuf[2 * p];
    lo[p] = cx.hbuf[2 * p + 1];
  }
  cx.ar->release(mark);
  return T2S2_OK;
}

t2s2_status tt_dots(Ctx& cx, int n, const DevTT* const* u, const DevTT* const* v, double* out) {
  if (n < 1 || n > kMaxDots) return T2S2_EINVAL;
  const int d = u[0]->d;
  DotArgs a;
  a.n = n;
  a.d = d;
  for (int k = 0; k < d; ++k) a.m[k] = u[0]->m[k];
  size_t mark = cx.ar->mark();
  long st1 = 0, st2 = 0;
  double fl = 0.0;
  for (int p = 0; p < n; ++p) {
    if (u[p]->d != d || v[p]->d != d) return T2S2_EINVAL;
    size_t phi_n = 1, w_n = 1;
    for (int k = 0; k < d; ++k) {
      if (u[p]->m[k] != a.m[k] || v[p]->m[k] != a.m[k]) return T2S2_EINVAL;
      a.u[p][k] = u[p]->c[k];
      a.v[p][k] = v[p]->c[k];
      phi_n = std::max(phi_n, (size_t)u[p]->r[k + 1] * v[p]->r[k + 1]);
      w_n = std::max(w_n, (size_t)v[p]->r[k] * a.m[k] * u[p]->r[k + 1]);
      fl += 2.0 * v[p]->r[k] * a.m[k] * (double)u[p]->r[k + 1] * (u[p]->r[k] + v[p]->r[k + 1]);
    }
    for (int k = 0; k <= d; ++k) {
      a.ru[p][k] = u[p]->r[k];
      a.rv[p][k] = v[p]->r[k];
    }
    a.phi[p] = aget<double>(cx, phi_n);
    a.w[p] = aget<double>(cx, w_n);
    if (!a.phi[p] || !a.w[p]) return T2S2_ENOMEM;
  }
  for (int k = 0; k < d; ++k) {
    long s1 = 0, s2 = 0;
    for (int p = 0; p < n; ++p) {
      s1 += (long)a.rv[p][k] * a.m[k] * a.ru[p][k + 1];
      s2 += (long)a.ru[p][k + 1] * a.rv[p][k + 1];
    }
    st1 = std::max(st1, s1);
    st2 = std::max(st2, s2);
  }
  a.out = aget<double>(cx, n);
  if (!a.out) return T2S2_ENOMEM;
  int dev = 0, sms = 0, per_sm = 0;
  T2S2_CUDA_TRY(cudaGetDevice(&dev));
  T2S2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_dots_kernel, kDotThreads, 0));
  long cap = (long)std::max(1, per_sm) * sms;
  cap = std::min<long>(cap, sms);
  if (cx.coop_ctas > 0) cap = std::min<long>(cap, cx.coop_ctas);
  // sized by the work (one item per thread, one phi entry per warp): every
  // grid barrier costs more with more CTAs
  const long want = std::max((st1 + kDotThreads - 1) / kDotThreads, (32 * st2 + kDotThreads - 1) / kDotThreads);
  const int G = (int)std::max(1L, std::min(cap, want));
  {
    TraceScope ts(kTrDots, cx.st, fl, 0.0);
    void* args[] = {&a};
    T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)tt_dots_kernel, dim3(G), dim3(kDotThreads), args, 0,
                                              cx.st));
  }
  T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, a.out, sizeof(double) * n, cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  for (int p = 0; p < n; ++p) out[p] = cx.hbuf[p];
  cx.ar->release(mark);
  return T2S2_OK;
}

}  // namespace t2s2
