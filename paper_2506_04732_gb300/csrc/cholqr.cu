// Shifted CholeskyQR (up to four passes) in ONE cooperative launch.
//
// The orthogonalisations of the TT sweeps (Methods: QR of the unfoldings
// before every truncation) factor tall-skinny blocks of nlong vectors of
// length c <= 96.  One grid does every pass:
//
//   pass p = 0, 1, 2:
//     every CTA:  partial Gram of its own vectors (compact lower triangle)
//                                                             (grid sync)
//     CTA b:      sums its slice of the Gram over all partials (grid sync)
//     every CTA:  loads the Gram; if it is within kOrthDev / c of the identity
//                 this pass is the last one (and pass 0 runs unshifted);
//                 (Gram + shift I) = L D L^T, semidefinite (pivots below
//                 64 u max diag zeroed), with L^{-1} built in the same
//                 elimination steps; v <- D^{-1/2} L^{-1} v for its own
//                 vectors; its own rows of Lacc <- Lacc L D^{1/2}
//
// with the shift of the first pass as in Fukaya et al.'s shifted
// CholeskyQR3, and the same shift in the second pass when it is not the last
// (kCqrShiftedPasses, small.h: a plain second pass would zero the pivots of
// directions that the first shift pushed to roundoff in column order, and
// lose more of W than those directions hold).  The stopping test is the CholeskyQR2 argument: a Gram close
// to the identity means a condition number close to 1, for which one more
// CholeskyQR pass yields Q orthonormal to working precision; blocks with one
// column need a single unshifted pass.  "Vectors" are the rows of a row-major
// rows x c block (tall: W = Q R with R = Lacc^T) or the columns of a
// row-major c x cols block (wide: W = L Q with L = Lacc).  Sums run in a
// fixed order, so results do not depend on timing.
//
// Binary64 on this part issues one warp instruction per ~64 cycles per SM
// sub-partition, so the small c x c work is shaped around that: one barrier
// per elimination step, the next pivot's reciprocal computed by one thread
// while the others update (binary32 seed, one Newton step in binary64 -- the
// pivots are exact binary64 values and decide zeroing; a reciprocal good to
// 2^-46 only perturbs L's off-diagonal entries, which are O(1e-3) or smaller
// in the final pass), exact power-of-4 scaling of the Gram so that binary32
// comparisons and seeds stay in range, and maxima taken as integer
// reductions of bit patterns.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <atomic>

#include "fastmath.cuh"
#include "small.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int kThreads = 256;
constexpr int kCholQrMaxSmem = 200 * 1024;
constexpr int kMaxGrid = 128;    // CTAs of one factorisation
constexpr int kPerTarget = 8;    // vectors per CTA
// a pass is the last one when every entry of its Gram is within kOrthDev / c
// of the identity's: then the spectral distance is at most kOrthDev, the
// block's condition number at most sqrt(3), and one more CholeskyQR pass
// leaves Q orthonormal to working precision (the CholeskyQR2 argument)
constexpr float kOrthDev = 0.5f;
constexpr double kUnitRoundoff = 1.1102230246251565e-16;  // 2^-53

struct CholQrArgs {
  const double* W;
  const double* W2;  // tall only: columns c1 .. c-1 in a second block (null: one block)
  int c1;
  double* Q;
  double* R;     // c x c output (R = Lacc^T for tall, L = Lacc for wide)
  double* part;  // grid x T partial Grams (T = c (c + 1) / 2)
  double* gsum;  // T: the summed Gram
  int* status;   // set to 1 when a pivot was zeroed (rank deficiency)
  int nlong, c, per;  // vectors, their length, vectors per CTA
  int tall;
  double shift_rel;
  unsigned long long* tstamp;  // diagnostics: phase times of CTA 0 (null: off)
};

constexpr int kQrStamps = 2 + 6 * kCqrMaxPass + 1;

#define QR_STAMP(k)                                                                   \
  do {                                                                                \
    if (a.tstamp && blockIdx.x == 0 && threadIdx.x == 0) {                            \
      unsigned long long ts_;                                                         \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ts_));                         \
      a.tstamp[k] = ts_;                                                              \
    }                                                                                 \
  } while (0)

__host__ __device__ inline int tri_count(int c) { return c * (c + 1) / 2; }

__host__ __device__ inline size_t smem_bytes(int per, int c, int grid) {
  const int rpc = (c + grid - 1) / grid;
  return sizeof(double) * (2 * (size_t)per * c + 2 * (size_t)c * c + 2 * (size_t)rpc * c + 4 * (size_t)c) +
         sizeof(int) * ((tri_count(c) + 1) & ~1);
}

// element j of vector i in a tall (i-th row) or wide (i-th column) block
__device__ __forceinline__ long vidx(const CholQrArgs& a, int i, int j) {
  return a.tall ? (long)i * a.c + j : (long)j * a.nlong + i;
}

// element j of input vector i (a tall input may come in two column blocks)
__device__ __forceinline__ double win(const CholQrArgs& a, int i, int j) {
  if (a.W2) return j < a.c1 ? a.W[(long)i * a.c1 + j] : a.W2[(long)i * (a.c - a.c1) + (j - a.c1)];
  return a.W[vidx(a, i, j)];
}

// binary32 seed and one binary64 Newton step: 1/v to about 2^-46
__device__ __forceinline__ double pivot_rcp(double v, float f) {
  double y = (double)__frcp_rn(f);
  return y * fma(-v, y, 2.0);
}

__global__ void __launch_bounds__(kThreads) cholqr3_kernel(CholQrArgs a) {
  pdl_trigger();
  QR_STAMP(0);
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  const int c = a.c, T = tri_count(c);
  const int b = blockIdx.x, t = threadIdx.x, G = gridDim.x, lane = t & 31, warp = t >> 5;
  const int i0 = b * a.per, cnt = max(0, min(a.per, a.nlong - i0));
  const int rpc = (c + G - 1) / G;
  const int nrow = b < c ? (c - 1 - b) / G + 1 : 0;  // own rows b, b + G, ... of Lacc
  double* V = sm;                // per x c: own vectors
  double* V2 = V + a.per * c;    // per x c
  double* A = V2 + a.per * c;    // c x c lower: scaled Gram, LDL^T work, then L D^{1/2}
  double* B = A + c * c;         // c x c lower: unit L^{-1}
  double* Lr = B + c * c;        // rpc x c: own rows of Lacc
  double* Lr2 = Lr + rpc * c;    // rpc x c
  double* rv = Lr2 + rpc * c;    // 1/d_j (0 for a zeroed pivot), scaled units
  double* dv = rv + c;           // d_j (0 for a zeroed pivot), scaled units
  double* sdn = dv + c;          // sqrt(d_j), scaled units
  double* isdn = sdn + c;        // 1/sqrt(d_j), scaled units
  int* tri = reinterpret_cast<int*>(isdn + c);  // (row << 8) | col, lower triangle row by row
  __shared__ unsigned ired[2][kThreads / 32];
  __shared__ double shift, sc, isc;
  __shared__ float tauf;
  __shared__ int bad, last;
  for (int e = t; e < cnt * c; e += kThreads) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    V[r * c + j] = win(a, i0 + r, j);
  }
  for (int ia = t; ia < c; ia += kThreads)
    for (int ib = 0; ib <= ia; ++ib) tri[ia * (ia + 1) / 2 + ib] = (ia << 8) | ib;
  if (t == 0) bad = 0;
  __syncthreads();
  QR_STAMP(1);
  const int sl = (T + G - 1) / G;  // Gram entries summed by each CTA
  int pass = 0;
  for (;; ++pass) {
    // (1) partial Gram of own vectors, entries (k, j) with j <= k
    for (int e = t; e < T; e += kThreads) {
      const int rc = tri[e], k = rc >> 8, j = rc & 255;
      double s = 0.0;
      for (int r = 0; r < cnt; ++r) s = fma(V[r * c + j], V[r * c + k], s);
      a.part[(long)b * T + e] = s;
    }
    grid.sync();
    QR_STAMP(2 + 6 * pass + 0);
    // (2) this CTA's slice of the Gram: lanes over the partials, then a fixed
    // shuffle tree
    for (int e = b * sl + warp; e < min(T, (b + 1) * sl); e += kThreads / 32) {
      double s = 0.0;
      for (int p = lane; p < G; p += 32) s += a.part[(long)p * T + e];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) a.gsum[e] = s;
    }
    grid.sync();
    QR_STAMP(2 + 6 * pass + 1);
    // (3) load the Gram; the largest diagonal and the distance from the
    // identity as integer maxima of bit patterns (non-negative values order
    // like their bits); exactly zero columns, left by zeroed pivots, do not
    // count against the identity
    {
      unsigned mxh = 0, devb = 0;
      for (int e = t; e < T; e += kThreads) {
        const int rc = tri[e], k = rc >> 8, j = rc & 255;
        const double g = a.gsum[e];
        A[k * c + j] = g;
        B[k * c + j] = (k == j) ? 1.0 : 0.0;
        const float gf = (float)g;
        if (k == j) {
          mxh = max(mxh, (unsigned)max(__double2hiint(g), 0));
          if ((__double_as_longlong(g) << 1) != 0) devb = max(devb, __float_as_uint(fabsf(gf - 1.0f)));
        } else {
          devb = max(devb, __float_as_uint(fabsf(gf)));
        }
      }
      mxh = __reduce_max_sync(0xffffffffu, mxh);
      devb = __reduce_max_sync(0xffffffffu, devb);
      if (lane == 0) ired[0][warp] = mxh, ired[1][warp] = devb;
    }
    __syncthreads();
    if (t == 0) {
      unsigned M = 0, D = 0;
      for (int w = 0; w < kThreads / 32; ++w) M = max(M, ired[0][w]), D = max(D, ired[1][w]);
      const bool fin = (__uint_as_float(D) * c <= kOrthDev) || c == 1 || pass == kCqrMaxPass - 1;
      const double mx = __hiloint2double((int)M, 0);
      // shift of the first pass, with c * (largest diagonal) >= trace
      const double sh = (pass < kCqrShiftedPasses && !fin) ? a.shift_rel * c * mx : 0.0;
      shift = sh;
      last = fin;
      // exact power-of-4 scaling: the largest diagonal lands in [1, 4)
      const int ex = (int)((M >> 20) & 0x7FF);
      const int k2 = (ex > 0 && ex < 0x7FF) ? ((ex - 1023) >> 1) : 0;
      sc = __longlong_as_double((long long)(1023 + k2) << 52);
      isc = __longlong_as_double((long long)(1023 - k2) << 52);
      const double s2 = __longlong_as_double((long long)(1023 - 2 * k2) << 52);
      tauf = (float)(64.0 * kUnitRoundoff * (mx + sh) * s2);
    }
    __syncthreads();
    {
      const double s2 = isc * isc, sh = shift;
      for (int e = t; e < T; e += kThreads) {
        const int rc = tri[e], k = rc >> 8, j = rc & 255;
        const double v = (A[k * c + j] + (k == j ? sh : 0.0)) * s2;
        A[k * c + j] = v;
        if (e == 0) {  // tri[0] is (0, 0): the first pivot
          const float f = (float)v;
          const bool z = !(f > tauf);
          rv[0] = z ? 0.0 : pivot_rcp(v, f);
          dv[0] = z ? 0.0 : v;
          if (z) bad = 1;
        }
      }
    }
    __syncthreads();
    QR_STAMP(2 + 6 * pass + 2);
    // (4) L D L^T: step j takes column j out of the trailing block and out of
    // the rows of L^{-1} below j.  Thread 0 updates the next pivot and takes
    // its reciprocal; the other threads do the rest.
    for (int j = 0; j + 1 < c; ++j) {
      const int rem = c - 1 - j, nt = rem * (rem + 1) / 2, ni = rem * (j + 1);
      const double r = rv[j];
      if (t == 0) {
        const int i = j + 1;
        const double l = A[i * c + j];
        const double v = fma(-(l * r), l, A[i * c + i]);
        A[i * c + i] = v;
        const float f = (float)v;
        const bool z = !(f > tauf);
        rv[i] = z ? 0.0 : pivot_rcp(v, z ? 1.0f : f);
        dv[i] = z ? 0.0 : v;
        if (z) bad = 1;
      } else {
        for (int e = t; e < nt + ni; e += kThreads - 1) {
          if (e < nt) {
            const int rc = tri[e], i = j + 1 + (rc >> 8), k = j + 1 + (rc & 255);
            A[i * c + k] = fma(-(A[i * c + j] * r), A[k * c + j], A[i * c + k]);
          } else {
            const int q = e - nt, i = j + 1 + q / (j + 1), l = q % (j + 1);
            B[i * c + l] = fma(-(A[i * c + j] * r), B[j * c + l], B[i * c + l]);
          }
        }
      }
      __syncthreads();
    }
    for (int i = t; i < c; i += kThreads) {
      const double d = dv[i];
      const double is = d > 0.0 ? drsqrt(d) : 0.0;
      isdn[i] = is;
      sdn[i] = d * is;
    }
    __syncthreads();
    QR_STAMP(2 + 6 * pass + 3);
    // (5) v <- D^{-1/2} L^{-1} v for own vectors; rows i and c-1-i together,
    // so that every thread runs c + 1 products
    {
      const int h = (c + 1) / 2;
      const double sci = isc;
      for (int e = t; e < cnt * h; e += kThreads) {
        const int r = e / h, i1 = e % h, i2 = c - 1 - i1;
        const double* vr = V + r * c;
        double s1 = 0.0;
        for (int l = 0; l <= i1; ++l) s1 = fma(B[i1 * c + l], vr[l], s1);
        V2[r * c + i1] = s1 * isdn[i1] * sci;
        if (i2 != i1) {
          double s2 = 0.0;
          for (int l = 0; l <= i2; ++l) s2 = fma(B[i2 * c + l], vr[l], s2);
          V2[r * c + i2] = s2 * isdn[i2] * sci;
        }
      }
    }
    // the factor L D^{1/2} in unscaled units into A's lower part
    for (int e = t; e < T; e += kThreads) {
      const int rc = tri[e], i = rc >> 8, j = rc & 255;
      A[i * c + j] = (i == j) ? sdn[j] * sc : A[i * c + j] * isdn[j] * sc;
    }
    __syncthreads();
    QR_STAMP(2 + 6 * pass + 4);
    // (6) own rows of Lacc <- Lacc L D^{1/2}
    for (int e = t; e < nrow * c; e += kThreads) {
      const int q = e / c, k = e % c, i = b + q * G;
      double s = 0.0;
      if (pass == 0) {
        s = (k <= i) ? A[i * c + k] : 0.0;
      } else if (k <= i) {
        for (int l = k; l <= i; ++l) s = fma(Lr[q * c + l], A[l * c + k], s);
      }
      Lr2[q * c + k] = s;
    }
    __syncthreads();
    QR_STAMP(2 + 6 * pass + 5);
    double* tmp = Lr;
    Lr = Lr2;
    Lr2 = tmp;
    tmp = V;
    V = V2;
    V2 = tmp;
    if (last) break;  // the same decision in every CTA: same Gram, same code
  }
  for (int e = t; e < cnt * c; e += kThreads) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    a.Q[vidx(a, i0 + r, j)] = V[r * c + j];
  }
  for (int e = t; e < nrow * c; e += kThreads) {
    const int q = e / c, k = e % c, i = b + q * G;
    if (a.tall) a.R[k * c + i] = Lr[q * c + k];
    else a.R[i * c + k] = Lr[q * c + k];
  }
  QR_STAMP(kQrStamps - 1);
  if (b == 0 && t == 0 && a.status) *a.status = bad;
}

}  // namespace

size_t cholqr3_scratch_doubles(int nlong, int c, int grid) {
  (void)nlong;
  return (size_t)(grid + 1) * tri_count(c);  // partial Grams and their sum
}

// Grid size and shared memory for a fused CholeskyQR of nlong vectors of
// length c; returns false if no co-resident grid fits.
bool cholqr3_plan(int nlong, int c, int max_grid, int* grid_out, int* per_out, size_t* smem_out) {
  if (c < 1 || c > kSmallMax || nlong < c) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // about kPerTarget vectors per CTA: the Gram and the triangular product
  // scale with the vectors per CTA, the Gram sums are spread over the CTAs
  const int cap = std::min(kMaxGrid, max_grid > 0 ? std::min(sms, max_grid) : sms);
  int grid = std::max(1, std::min(cap, (nlong + kPerTarget - 1) / kPerTarget));
  const int per = (nlong + grid - 1) / grid;
  grid = (nlong + per - 1) / per;
  const size_t smem = smem_bytes(per, c, grid);
  if (smem > kCholQrMaxSmem) return false;
  // the attribute is set once per device to the largest size ever used: a
  // per-call value would race with concurrent solves on other host threads
  static std::atomic<unsigned long long> set_mask{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(set_mask.load() & bit)) {
    if (cudaFuncSetAttribute(cholqr3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholQrMaxSmem) !=
        cudaSuccess) {
      cudaGetLastError();  // leave no stale error behind
      return false;
    }
    set_mask.fetch_or(bit);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholqr3_kernel, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (per_sm * sms < grid) return false;
  *grid_out = grid;
  *per_out = per;
  *smem_out = smem;
  return true;
}

t2s2_status cholqr3_fused(const double* W, double* Q, double* R, int nlong, int c, bool tall, double shift_rel,
                          double* scratch, int* status, int grid, int per, size_t smem, cudaStream_t st,
                          const double* W2, int c1) {
  CholQrArgs a;
  a.W = W;
  a.W2 = (tall && W2) ? W2 : nullptr;
  a.c1 = c1;
  a.Q = Q;
  a.R = R;
  a.part = scratch;
  a.gsum = scratch + (size_t)grid * tri_count(c);
  a.status = status;
  a.nlong = nlong;
  a.c = c;
  a.per = per;
  a.tall = tall ? 1 : 0;
  a.shift_rel = shift_rel;
  a.tstamp = nullptr;
  // T2S2_QR_TIMING=N: the N-th fused factorisation of the process prints the
  // phase times of its CTA 0 (diagnostics; synchronises that one call)
  static const int stamp_at = [] {
    const char* e = std::getenv("T2S2_QR_TIMING");
    return (e && e[0] >= '0' && e[0] <= '9') ? std::atoi(e) : -1;
  }();
  static std::atomic<int> calls{0};
  static unsigned long long* stamp_buf = nullptr;
  const bool stamp_this = stamp_at >= 0 && calls.fetch_add(1) == stamp_at;
  if (stamp_this) {
    if (!stamp_buf) T2S2_CUDA_TRY(cudaMalloc(&stamp_buf, sizeof(unsigned long long) * kQrStamps));
    T2S2_CUDA_TRY(cudaMemsetAsync(stamp_buf, 0, sizeof(unsigned long long) * kQrStamps, st));
    a.tstamp = stamp_buf;
  }
  // work of two passes (the common case): Gram and triangular product
  // 2 n c^2 each, the L D L^T with its inverse 2 c^3 / 3
  const double fl = 2.0 * (4.0 * nlong * (double)c * c) + 2.0 * (2.0 * (double)c * c * c / 3.0);
  TraceScope ts(kTrCholQR, st, fl, 16.0 * nlong * c);
  void* args[] = {&a};
  T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cholqr3_kernel, dim3(grid), dim3(kThreads), args, smem, st));
  if (stamp_this) {
    unsigned long long h[kQrStamps];
    T2S2_CUDA_TRY(cudaMemcpyAsync(h, stamp_buf, sizeof(h), cudaMemcpyDeviceToHost, st));
    T2S2_CUDA_TRY(cudaStreamSynchronize(st));
    fprintf(stderr, "[t2s2] cholqr3 phase times (ns) nlong=%d c=%d grid=%d: load %lld", nlong, c, grid,
            (long long)(h[1] - h[0]));
    unsigned long long prev = h[1];
    for (int p = 0; p < kCqrMaxPass && h[2 + 6 * p]; ++p) {
      fprintf(stderr, " | pass %d:", p);
      for (int k = 0; k < 6; ++k) {
        fprintf(stderr, " %lld", (long long)(h[2 + 6 * p + k] - prev));
        prev = h[2 + 6 * p + k];
      }
    }
    fprintf(stderr, " | store %lld total %lld\n", (long long)(h[kQrStamps - 1] - prev),
            (long long)(h[kQrStamps - 1] - h[0]));
  }
  return T2S2_OK;
}

}  // namespace t2s2
