// Shifted CholeskyQR3 in ONE cooperative launch.
//
// The orthogonalisations of the TT sweeps (Methods: QR of the unfoldings
// before every truncation) factor tall-skinny blocks of nlong vectors of
// length c <= 96.  As separate launches each of the three CholeskyQR passes
// needs a Gram GEMM (plus split-K sum), a one-CTA Cholesky, the triangular
// product and the factor update: about sixteen launches per QR, each a few
// microseconds of mostly idle GPU.  Here one grid does all three passes:
//
//   for pass = 1..3:
//     every CTA:  partial Gram of its own vectors             (grid sync)
//     every CTA:  Gram = sum of all partials in CTA order, then
//                 (Gram + shift I) = L L^T (semidefinite; pivots below
//                 64 u max diag zeroed), L^{-1}, Lacc <- Lacc L -- the same
//                 numbers in every CTA, so no second barrier is needed
//     every CTA:  v <- L^{-1} v for its own vectors (kept in shared memory)
//
// with the shift of the first pass as in Fukaya et al.'s shifted CholeskyQR3.
// "Vectors" are the rows of a row-major rows x c block (tall: W = Q R with
// R = Lacc^T) or the columns of a row-major c x cols block (wide: W = L Q with
// L = Lacc).  Sums run in a fixed order, so results do not depend on timing.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "fastmath.cuh"
#include "small.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int kThreads = 256;
constexpr int kCholQrMaxSmem = 200 * 1024;

struct CholQrArgs {
  const double* W;
  double* Q;
  double* R;     // c x c output (R = Lacc^T for tall, L = Lacc for wide)
  double* part;  // 2 x grid x c x c partial Grams (alternating by pass)
  int* status;   // set to 1 when a pivot was zeroed (rank deficiency)
  int nlong, c, per;  // vectors, their length, vectors per CTA
  int tall;
  double shift_rel;
};

// element j of vector i in a tall (i-th row) or wide (i-th column) block
__device__ __forceinline__ long vidx(const CholQrArgs& a, int i, int j) {
  return a.tall ? (long)i * a.c + j : (long)j * a.nlong + i;
}

__global__ void __launch_bounds__(kThreads) cholqr3_kernel(CholQrArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  const int c = a.c, cc = c * c;
  const int b = blockIdx.x, t = threadIdx.x, G = gridDim.x;
  const int i0 = b * a.per, cnt = max(0, min(a.per, a.nlong - i0));
  double* V = sm;                 // per x c: own vectors
  double* V2 = V + a.per * c;     // per x c
  double* A = V2 + a.per * c;     // c x c: Gram, then L
  double* Iv = A + cc;            // c x c: L^{-1}
  double* Lacc = Iv + cc;         // c x c (kept by every CTA; CTA 0 writes it out)
  __shared__ double shift, tau;
  __shared__ int bad;
  // own vectors of W
  for (int e = t; e < cnt * c; e += kThreads) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    V[r * c + j] = a.W[vidx(a, i0 + r, j)];
  }
  if (t == 0) bad = 0;
  __syncthreads();
  for (int pass = 0; pass < 3; ++pass) {
    // partials alternate between two buffers: a CTA may still be reading the
    // previous pass's partials while a faster one writes this pass's
    double* part = a.part + (size_t)(pass & 1) * G * cc;
    // (1) partial Gram of own vectors (upper triangle)
    for (int e = t; e < cc; e += kThreads) {
      const int j = e / c, k = e % c;
      double s = 0.0;
      if (k >= j)
        for (int r = 0; r < cnt; ++r) s = fma(V[r * c + j], V[r * c + k], s);
      part[(long)b * cc + e] = s;
    }
    grid.sync();
    // (2) every CTA: Gram = sum of the partials in CTA order, then the same
    // shifted semidefinite Cholesky and inverse (identical in all CTAs)
    for (int e = t; e < cc; e += kThreads) {
      const int j = e / c, k = e % c;
      double s = 0.0;
      if (k <= j) {
#pragma unroll 8
        for (int p = 0; p < G; ++p) s += part[(long)p * cc + k * c + j];
      }
      A[e] = s;  // lower triangle (row j >= column k) from the upper partials
    }
    __syncthreads();
    if (t == 0) {
      double tr = 0.0, mx = 0.0;
      for (int i = 0; i < c; ++i) {
        tr += A[i * c + i];
        mx = fmax(mx, A[i * c + i]);
      }
      shift = (pass == 0) ? a.shift_rel * tr : 0.0;
      tau = 64.0 * 1.1102230246251565e-16 * (mx + shift);
    }
    __syncthreads();
    for (int i = t; i < c; i += kThreads) A[i * c + i] += shift;
    __syncthreads();
    for (int j = 0; j < c; ++j) {
      const double v = A[j * c + j];
      const bool zero = !(v > tau);
      __syncthreads();
      if (zero) {
        for (int i = j + t; i < c; i += kThreads) A[i * c + j] = 0.0;
        if (t == 0) bad = 1;
        __syncthreads();
        continue;
      }
      const double rinv = drsqrt(v);
      for (int i = j + 1 + t; i < c; i += kThreads) A[i * c + j] *= rinv;
      if (t == 0) A[j * c + j] = v * rinv;
      __syncthreads();
      const int rem = c - j - 1;
      for (int e = t; e < rem * rem; e += kThreads) {
        const int i = j + 1 + e / rem, k = j + 1 + e % rem;
        if (k <= i) A[i * c + k] -= A[i * c + j] * A[k * c + j];
      }
      __syncthreads();
    }
    // pseudo-inverse of lower-triangular L (x_i = 0 where L_ii = 0)
    for (int e = t; e < cc; e += kThreads) Iv[e] = 0.0;
    __syncthreads();
    for (int k = t; k < c; k += kThreads) {
      for (int i = k; i < c; ++i) {
        const double dii = A[i * c + i];
        if (dii == 0.0) continue;
        double s = (i == k) ? 1.0 : 0.0;
        for (int l = k; l < i; ++l) s -= A[i * c + l] * Iv[l * c + k];
        Iv[i * c + k] = s * drcp(dii);
      }
    }
    __syncthreads();
    // (3) v <- L^{-1} v for own vectors
    for (int e = t; e < cnt * c; e += kThreads) {
      const int r = e / c, j = e % c;
      double s = 0.0;
      for (int k = 0; k <= j; ++k) s = fma(Iv[j * c + k], V[r * c + k], s);
      V2[e] = s;
    }
    __syncthreads();
    // Lacc <- Lacc L (lower triangular product), staged in Iv (now free)
    if (pass == 0) {
      for (int e = t; e < cc; e += kThreads) Lacc[e] = (e % c <= e / c) ? A[e] : 0.0;
    } else {
      for (int e = t; e < cc; e += kThreads) {
        const int i = e / c, k = e % c;
        double s = 0.0;
        if (k <= i)
          for (int l = k; l <= i; ++l) s = fma(Lacc[i * c + l], A[l * c + k], s);
        Iv[e] = s;
      }
      __syncthreads();
      for (int e = t; e < cc; e += kThreads) Lacc[e] = Iv[e];
    }
    __syncthreads();
    double* tmp = V;
    V = V2;
    V2 = tmp;
  }
  // own vectors of Q
  for (int e = t; e < cnt * c; e += kThreads) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    a.Q[vidx(a, i0 + r, j)] = V[r * c + j];
  }
  if (b == 0) {
    for (int e = t; e < cc; e += kThreads) {
      const int i = e / c, k = e % c;
      a.R[e] = a.tall ? Lacc[k * c + i] : Lacc[e];
    }
    if (t == 0 && a.status) *a.status = bad;
  }
}

}  // namespace

size_t cholqr3_scratch_doubles(int nlong, int c, int grid) {
  (void)nlong;
  return 2 * (size_t)grid * c * c;  // two alternating sets of partial Grams
}

// Grid size and shared memory for a fused CholeskyQR3 of nlong vectors of
// length c; returns false if no co-resident grid fits.
bool cholqr3_plan(int nlong, int c, int max_grid, int* grid_out, int* per_out, size_t* smem_out) {
  if (c < 1 || c > kSmallMax || nlong < c) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // about 16 vectors per CTA and at most 64 CTAs: the Gram reduction reads one
  // partial per CTA for every entry, so a wider grid costs more than it saves
  const int cap = std::min(64, max_grid > 0 ? std::min(sms, max_grid) : sms);
  int grid = std::max(1, std::min(cap, (nlong + 15) / 16));
  const int per = (nlong + grid - 1) / grid;
  grid = (nlong + per - 1) / per;
  const size_t smem = sizeof(double) * (2 * (size_t)per * c + 3 * (size_t)c * c);
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
                          double* scratch, int* status, int grid, int per, size_t smem, cudaStream_t st) {
  CholQrArgs a;
  a.W = W;
  a.Q = Q;
  a.R = R;
  a.part = scratch;
  a.status = status;
  a.nlong = nlong;
  a.c = c;
  a.per = per;
  a.tall = tall ? 1 : 0;
  a.shift_rel = shift_rel;
  const double fl = 3.0 * (4.0 * nlong * (double)c * c) + 3.0 * (double)c * c * c;
  TraceScope ts(kTrSmall, st, fl, 16.0 * nlong * c);
  void* args[] = {&a};
  T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cholqr3_kernel, dim3(grid), dim3(kThreads), args, smem, st));
  return T2S2_OK;
}

}  // namespace t2s2
