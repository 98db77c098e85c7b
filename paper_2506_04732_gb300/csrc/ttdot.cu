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
#include <mutex>
#include <atomic>

#include "api_internal.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int kDotThreads = 256;
constexpr int kMaxDots = 4;
constexpr int kMaxClusterDots = 16;  // grids of at most this many CTAs run as one cluster
// double-double products up to which one cluster beats the full grid: 16 SMs
// issue ~32 binary64 lane operations per clock, ~11 per product term, against
// ~24 us of grid barriers for a d = 6 train
constexpr double kDDClusterTerms = 60000.0;

// Barrier between the stages: a grid barrier of a cooperative launch (~2 us
// on this part), or, when the whole grid is one thread-block cluster, a
// cluster barrier (~0.2 us; release/acquire at cluster scope orders the
// stages' global-memory writes and reads).
template <bool kCluster>
__device__ __forceinline__ void stage_barrier(cg::grid_group& grid) {
  if constexpr (kCluster) cg::this_cluster().sync();
  else grid.sync();
}

__device__ __forceinline__ void stage_stamp(unsigned long long* ts, int k) {
  if (ts && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    ts[k] = t;
  }
}

struct DotArgs {
  int n, d;
  int m[T2S2_MAX_D];
  int ru[kMaxDots][T2S2_MAX_D + 1], rv[kMaxDots][T2S2_MAX_D + 1];
  const double* u[kMaxDots][T2S2_MAX_D];
  const double* v[kMaxDots][T2S2_MAX_D];
  double* phi[kMaxDots];  // ru_k x rv_k
  double* w[kMaxDots];    // rv_k x m_k x ru_{k+1}
  double* out;            // n values
  unsigned long long* tstamp;  // diagnostics: stage end times of CTA 0 (null: off)
};

template <bool kCluster>
__global__ void __launch_bounds__(kDotThreads) tt_dots_kernel(DotArgs a) {
  pdl_wait();  // a cluster launch may overlap the previous kernel of the stream
  pdl_trigger();
  stage_stamp(a.tstamp, 0);
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
    stage_barrier<kCluster>(grid);
    stage_stamp(a.tstamp, 1 + 2 * k);
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
    stage_barrier<kCluster>(grid);
    stage_stamp(a.tstamp, 2 + 2 * k);
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
  unsigned long long* tstamp;  // diagnostics: stage end times of CTA 0 (null: off)
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

template <bool kCluster>
__global__ void __launch_bounds__(kDotThreads) tt_norm2_dd_kernel(DDArgs a) {
  pdl_wait();  // a cluster launch may overlap the previous kernel of the stream
  pdl_trigger();
  stage_stamp(a.tstamp, 0);
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x, g = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < a.d; ++k) {
    const int m = a.m[k];
    long tot = 0;
    for (int p = 0; p < a.n; ++p) tot += (long)a.s[p][k] * m * a.r[p][k + 1];
    // W[a', i, b] = sum_a phi[a, a'] U[a, i, b]; when the items are fewer
    // than half the grid's threads, S2 adjacent lanes share one (the sum over
    // a split S2 ways, combined by shuffles within the group)
    int S2 = 1;
    if (k > 0)
      while (S2 < 8 && tot * (S2 * 2) <= (long)G * kDotThreads) S2 *= 2;
    const unsigned gmask = (S2 == 32 ? 0xffffffffu : ((1u << S2) - 1u)) << (lane & ~(S2 - 1));
    const int gpart = lane & (S2 - 1);
    for (long slot = threadIdx.x / S2;; slot += kDotThreads / S2) {
      const long e = spread_item(slot, G, g);
      if (e >= tot) break;  // the same for the S2 lanes of a group
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
        int x = gpart;
        for (; x + S2 < ra; x += 2 * S2) {
          dd_fma(h0, l0, ph[(long)x * sa + ap], pl[(long)x * sa + ap], U[((long)x * m + i) * rb + b]);
          dd_fma(h1, l1, ph[(long)(x + S2) * sa + ap], pl[(long)(x + S2) * sa + ap],
                 U[((long)(x + S2) * m + i) * rb + b]);
        }
        if (x < ra) dd_fma(h0, l0, ph[(long)x * sa + ap], pl[(long)x * sa + ap], U[((long)x * m + i) * rb + b]);
        dd_add(h0, l0, h1, l1);
        for (int o = S2 >> 1; o > 0; o >>= 1) {
          const double h2 = __shfl_xor_sync(gmask, h0, o), l2 = __shfl_xor_sync(gmask, l0, o);
          dd_add(h0, l0, h2, l2);
        }
      }
      if (gpart == 0) {
        a.wh[p][q] = h0;
        a.wl[p][q] = l0;
      }
    }
    stage_barrier<kCluster>(grid);
    stage_stamp(a.tstamp, 1 + 2 * k);
    // phi[b, b'] = sum_{a', i} W[a', i, b] V[a', i, b'] (upper triangle only
    // when V is U; both halves are written)
    long tot2 = 0;
    for (int p = 0; p < a.n; ++p) tot2 += dd_phi_items(a, p, k);
    // CTA g takes entries g, g + G, ...; when it has fewer entries than warps,
    // P warps share one entry (P = 1, 2, 4, 8: the k sum split P ways) so
    // that every SM sub-partition issues, and the P partial sums are added
    // in shared memory in a fixed order
    const long mine = tot2 > g ? (tot2 - 1 - g) / G + 1 : 0;  // entries of this CTA
    constexpr int NWd = kDotThreads / 32;
    int P = 1;
    while (P < NWd && mine * (P * 2) <= NWd) P *= 2;
    const int per_round = NWd / P;
    const long rounds = (mine + per_round - 1) / per_round;  // the same for every warp of the CTA
    const int part = warp % P;
    for (long round = 0; round < rounds; ++round) {
      const long slot = round * per_round + warp / P;
      const long it = spread_item(slot, G, g);
      const bool valid = slot < mine;  // warp-uniform
      int p = 0, b = 0, bp = 0, sb = 1;
      double h0 = 0.0, l0 = 0.0;
      if (valid) {
        long q = it;
        while (q >= dd_phi_items(a, p, k)) q -= dd_phi_items(a, p, k), ++p;
        const int rb = a.r[p][k + 1], sa = a.s[p][k];
        sb = a.s[p][k + 1];
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
        const int K = sa * m, stride = 32 * P;
        double h1 = 0.0, l1 = 0.0;
        int x = part * 32 + lane;
        for (; x + stride < K; x += 2 * stride) {
          dd_fma(h0, l0, Wh[(long)x * rb + b], Wl[(long)x * rb + b], V[(long)x * sb + bp]);
          dd_fma(h1, l1, Wh[(long)(x + stride) * rb + b], Wl[(long)(x + stride) * rb + b],
                 V[(long)(x + stride) * sb + bp]);
        }
        if (x < K) dd_fma(h0, l0, Wh[(long)x * rb + b], Wl[(long)x * rb + b], V[(long)x * sb + bp]);
        dd_add(h0, l0, h1, l1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double h2 = __shfl_xor_sync(0xffffffffu, h0, o), l2 = __shfl_xor_sync(0xffffffffu, l0, o);
          dd_add(h0, l0, h2, l2);
        }
      }
      if (P > 1) {
        __shared__ double ph_part[NWd], pl_part[NWd];
        if (lane == 0) {
          ph_part[warp] = h0;
          pl_part[warp] = l0;
        }
        __syncthreads();
        if (valid && part == 0 && lane == 0)
          for (int w = 1; w < P; ++w) dd_add(h0, l0, ph_part[warp + w], pl_part[warp + w]);
        __syncthreads();
      }
      if (valid && part == 0 && lane == 0) {
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
    stage_barrier<kCluster>(grid);
    stage_stamp(a.tstamp, 2 + 2 * k);
  }
  if (g == 0 && threadIdx.x < a.n) {
    a.out[2 * threadIdx.x] = a.phh[threadIdx.x][0];
    a.out[2 * threadIdx.x + 1] = a.phl[threadIdx.x][0];
  }
}

}  // namespace

// T2S2_DOT_TIMING=N: the N-th inner-product launch of the process (both
// kernels counted) prints the end time of every stage of its CTA 0
// (diagnostics; synchronises that one call).
static unsigned long long* dot_stamps(cudaStream_t st, bool* on) {
  static const int at = [] {
    const char* e = std::getenv("T2S2_DOT_TIMING");
    return (e && e[0] >= '0' && e[0] <= '9') ? std::atoi(e) : -1;
  }();
  static std::atomic<int> calls{0};
  static unsigned long long* buf = nullptr;
  *on = at >= 0 && calls.fetch_add(1) == at;
  if (!*on) return nullptr;
  if (!buf && cudaMalloc(&buf, sizeof(unsigned long long) * (1 + 2 * T2S2_MAX_D)) != cudaSuccess) {
    cudaGetLastError();
    *on = false;
    return nullptr;
  }
  cudaMemsetAsync(buf, 0, sizeof(unsigned long long) * (1 + 2 * T2S2_MAX_D), st);
  return buf;
}

static void dot_stamps_print(unsigned long long* buf, int d, int G, const char* what, cudaStream_t st) {
  unsigned long long h[1 + 2 * T2S2_MAX_D];
  if (cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  fprintf(stderr, "[t2s2] %s stage times (ns), %d CTAs:", what, G);
  for (int k = 0; k < d; ++k)
    fprintf(stderr, " | core %d: %lld %lld", k, (long long)(h[1 + 2 * k] - h[2 * k]),
            (long long)(h[2 + 2 * k] - h[1 + 2 * k]));
  fprintf(stderr, "\n");
}

// Launch one of the stage kernels: as one thread-block cluster with
// programmatic dependent launch when the grid has at most kMaxClusterDots
// CTAs and such a cluster can be resident, else as a cooperative grid.
template <typename Args>
static t2s2_status launch_stages(void (*coop)(Args), void (*clus)(Args), Args& a, int G, cudaStream_t st) {
  static std::once_flag once;
  static bool attr_ok = false;
  std::call_once(once, [&] {
    attr_ok = cudaFuncSetAttribute(clus, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    if (!attr_ok) cudaGetLastError();
  });
  if (attr_ok && G <= kMaxClusterDots) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kDotThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static std::atomic<signed char> fits[kMaxClusterDots + 1];  // 0 unknown, 1 yes, -1 no
    signed char f = fits[G].load();
    if (f == 0) {
      int nc = 0;
      const bool ok = cudaOccupancyMaxActiveClusters(&nc, clus, &cfg) == cudaSuccess && nc > 0;
      if (!ok) cudaGetLastError();
      f = ok ? 1 : -1;
      fits[G].store(f);
    }
    if (f > 0) {
      cfg.numAttrs = pdl_enabled() ? 2 : 1;
      T2S2_CUDA_TRY(cudaLaunchKernelEx(&cfg, clus, a));
      return T2S2_OK;
    }
  }
  void* args[] = {&a};
  T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)coop, dim3(G), dim3(kDotThreads), args, 0, st));
  return T2S2_OK;
}

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
  T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_norm2_dd_kernel<false>, kDotThreads, 0));
  long cap = std::min<long>((long)std::max(1, per_sm) * sms, sms);
  if (cx.coop_ctas > 0) cap = std::min<long>(cap, cx.coop_ctas);
  // ~11 binary64 operations per product term: binary64 issue, not the item
  // count, sets the time, so every SM takes a share -- unless the products
  // are few enough that the grid barriers (two per core) would cost more than
  // the binary64 issue of one cluster: then one cluster sized by the items
  int G = (int)std::max(1L, cap);
  if (fl * 0.5 <= kDDClusterTerms) {
    long st1 = 0, st2 = 0;
    for (int k = 0; k < d; ++k) {
      long s1 = 0, s2 = 0;
      for (int p = 0; p < n; ++p) {
        s1 += (long)a.s[p][k] * a.m[k] * a.r[p][k + 1];
        s2 += (long)a.r[p][k + 1] * a.s[p][k + 1];
      }
      st1 = std::max(st1, s1);
      st2 = std::max(st2, s2);
    }
    const long want = std::max((st1 + kDotThreads - 1) / kDotThreads, (32 * st2 + kDotThreads - 1) / kDotThreads);
    G = (int)std::max(1L, std::min<long>(kMaxClusterDots, std::min<long>(cap, want)));
  }
  {
    TraceScope ts(kTrDots, cx.st, fl, 0.0);  // algorithmic: 2 per product term
    bool on = false;
    a.tstamp = dot_stamps(cx.st, &on);
    T2S2_TRY(launch_stages(tt_norm2_dd_kernel<false>, tt_norm2_dd_kernel<true>, a, G, cx.st));
    if (on) dot_stamps_print(a.tstamp, d, G, "double-double dots", cx.st);
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
  T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_dots_kernel<false>, kDotThreads, 0));
  long cap = (long)std::max(1, per_sm) * sms;
  cap = std::min<long>(cap, sms);
  if (cx.coop_ctas > 0) cap = std::min<long>(cap, cx.coop_ctas);
  // sized by the work (one item per thread, one phi entry per warp): every
  // grid barrier costs more with more CTAs
  const long want = std::max((st1 + kDotThreads - 1) / kDotThreads, (32 * st2 + kDotThreads - 1) / kDotThreads);
  const int G = (int)std::max(1L, std::min(cap, want));
  {
    TraceScope ts(kTrDots, cx.st, fl, 0.0);
    bool on = false;
    a.tstamp = dot_stamps(cx.st, &on);
    T2S2_TRY(launch_stages(tt_dots_kernel<false>, tt_dots_kernel<true>, a, G, cx.st));
    if (on) dot_stamps_print(a.tstamp, d, G, "binary64 dots", cx.st);
  }
  T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, a.out, sizeof(double) * n, cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  for (int p = 0; p < n; ++p) out[p] = cx.hbuf[p];
  cx.ar->release(mark);
  return T2S2_OK;
}

}  // namespace t2s2
