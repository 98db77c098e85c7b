// TT-matrix-by-TT product for the rank-2 collocation operator (eq.
// tt-matrix-format): y = (c_mass M + c_op A) x with
//     A = sum_k Rt_1 x ... x Lt_k x ... x Rt_d,   M = Rt_1 x ... x Rt_d.
// Core k of y needs the two mode-k contractions S X_k and G X_k with
// S = Rt_k and G = c_op Lt_k (+ c_mass Rt_1 on the first core).  Each CTA
// computes a 64 x 64 tile of [S; G] X_k (rows: the 2m stacked output rows,
// columns: the (a, b) = (left, right) rank pairs of the core) and writes it
// straight into the block pattern of Y_k:
//     first  [G X, S X]            (1      x m x 2 r1)
//     middle [[S X, 0], [G X, S X]] (2 r0  x m x 2 r1)
//     last   [S X; G X]            (2 r0  x m x 1)
//     d = 1  G X                   (1      x m x 1)
// All d cores go in one launch; the zero block of middle cores is written by
// the S-row tiles.
#include <algorithm>

#include "apply.h"
#include "trace.h"

namespace t2s2 {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
// small trains: 16 x 16 tiles, one output per thread, so that the few
// tiles of a small problem still spread over the SMs
constexpr int BMS = 16, BNS = 16;

struct ParamWork {
  ApplyBatch p;
  int start[T2S2_MAX_D + 1];  // first tile of each core; start[ncores] = total
  __device__ int n() const { return p.ncores; }
  __device__ int first(int i) const { return start[i]; }
  __device__ ApplyCore core(int i) const { return p.c[i]; }
};
struct GlobalWork {
  const ApplyCore* c;
  const int* start;
  int ncores;
  __device__ int n() const { return ncores; }
  __device__ int first(int i) const { return start[i]; }
  __device__ ApplyCore core(int i) const { return c[i]; }
};

template <class Work>
__device__ __forceinline__ int find_core(const Work& w, int tile) {
  int lo = 0, hi = w.n() - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.first(mid) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Persistent over tiles: CTA b takes tiles b, b + gridDim.x, ...  A tile is
// 64 rows of [S; G] by 64 (a, b) pairs of the core (column g = a rb + b), so
// small right ranks waste no columns.
template <class Work, int TBM, int TBN>
__global__ void __launch_bounds__(NT) apply_kernel(Work w, int total) {
  pdl_wait();
  pdl_trigger();
  constexpr int TM = TBM / 16, TN = TBN / 16;
  __shared__ double As[BK][TBM + 1];
  __shared__ double Bs[BK][TBN + 1];
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int ci = find_core(w, tile);
    const ApplyCore c = w.core(ci);
    const int local = tile - w.first(ci);
    const long npairs = (long)c.ra * c.rb;
    const int nt = (int)((npairs + TBN - 1) / TBN);
    const int m0 = (local / nt) * TBM;
    const long n0 = (long)(local % nt) * TBN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < c.m; k0 += BK) {
      for (int e = threadIdx.x; e < TBM * BK; e += NT) {
        int kk = e % BK, mm = e / BK;
        int row = m0 + mm, col = k0 + kk;
        double v = 0.0;
        if (row < 2 * c.m && col < c.m) {
          if (row < c.m) {
            v = c.S[(long)row * c.m + col];
          } else {
            long o = (long)(row - c.m) * c.m + col;
            v = c.g_op * c.L[o];
            if (c.g_mass != 0.0) v += c.g_mass * c.S[o];
          }
        }
        As[kk][mm] = v;
      }
      for (int e = threadIdx.x; e < TBN * BK; e += NT) {
        const int nn = e % TBN, kk = e / TBN;
        const long g = n0 + nn;
        const int j = k0 + kk;
        double v = 0.0;
        if (j < c.m && g < npairs) {
          const long a = g / c.rb, b = g % c.rb;
          v = c.X[(a * c.m + j) * c.rb + b];
        }
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    // scatter into the block pattern of Y
    const int ra = c.ra, rb = c.rb, m = c.m;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const long g = n0 + tx + 16 * j;
      if (g >= npairs) continue;
      const long a = g / rb, b = g % rb;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int row = m0 + ty + 16 * i;
        if (row >= 2 * m) continue;
        const bool gpart = row >= m;
        const int ii = gpart ? row - m : row;
        const double v = acc[i][j];
        double* Y = c.Y;
        switch (c.kind) {
          case kApplySingle:  // 1 x m x 1
            if (gpart) Y[ii] = v;
            break;
          case kApplyFirst: {  // 1 x m x 2rb: [G X, S X]
            const long base = (long)ii * 2 * rb;
            if (gpart) Y[base + b] = v; else Y[base + rb + b] = v;
            break;
          }
          case kApplyLast: {  // 2ra x m x 1: [S X; G X]
            const long r = gpart ? (ra + a) : a;
            Y[r * m + ii] = v;
            break;
          }
          default: {  // middle: 2ra x m x 2rb
            const long wd = 2L * rb;
            if (gpart) {
              Y[((ra + a) * m + ii) * wd + b] = v;            // (1,0): G X
            } else {
              Y[(a * m + ii) * wd + b] = v;                   // (0,0): S X
              Y[((ra + a) * m + ii) * wd + rb + b] = v;       // (1,1): S X
              Y[(a * m + ii) * wd + rb + b] = 0.0;            // (0,1): 0
            }
          }
        }
      }
    }
  }
}
}  // namespace

int apply_fp64_tiles(const ApplyCore& c) { return cdiv(2 * c.m, BM) * cdiv((long)c.ra * c.rb, BN); }

t2s2_status apply_fp64(const ApplyBatch& p, cudaStream_t st) {
  ParamWork w;
  w.p = p;
  int total = 0;
  double fl = 0.0, by = 0.0;
  for (int k = 0; k < p.ncores; ++k) {
    total += apply_fp64_tiles(p.c[k]);
    apply_work_totals(p.c[k], &fl, &by);
  }
  if (total == 0) return T2S2_OK;
  // fewer 64 x 64 tiles than SMs: take 16 x 16 tiles instead (a 64 x 64
  // tile of K = m costs its SM 64 x 64 x m / 2 cycles of binary64 issue)
  const bool small = total < kNumSMs;
  const int tbm = small ? BMS : BM, tbn = small ? BNS : BN;
  total = 0;
  for (int k = 0; k < p.ncores; ++k) {
    w.start[k] = total;
    const ApplyCore& c = p.c[k];
    total += cdiv(2 * c.m, tbm) * cdiv((long)c.ra * c.rb, tbn);
  }
  w.start[p.ncores] = total;
  TraceScope ts(kTrApply, st, fl, by);
  if (small) (void)launch_pdl(apply_kernel<ParamWork, BMS, BNS>, total, NT, 0, st, w, total);
  else (void)launch_pdl(apply_kernel<ParamWork, BM, BN>, total, NT, 0, st, w, total);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

t2s2_status apply_fp64_grouped(const ApplyCore* dcores, const int* dstart, int ncores, int total, int grid,
                               double flops, double bytes, cudaStream_t st) {
  if (ncores < 1 || total < 0 || grid < 1) return T2S2_EINVAL;
  if (total == 0) return T2S2_OK;
  GlobalWork w{dcores, dstart, ncores};
  TraceScope ts(kTrApply, st, flops, bytes);
  (void)launch_pdl(apply_kernel<GlobalWork, BM, BN>, std::min(grid, total), NT, 0, st, w, total);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

}  // namespace t2s2
