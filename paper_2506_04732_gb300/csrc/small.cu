// Small dense factorisations (c x c, c <= kSmallMax) done by one CTA in
// shared memory, FP64:
//  * chol_inv: G + s I = L L^T (Cholesky) and L^{-1}, for CholeskyQR.  The
//    shift s makes the shifted passes of CholeskyQR (Fukaya, Kannan,
//    Nakatsukasa, Yamamoto, Yanagisawa 2020) succeed for any conditioning.
//  * jacobi_svd: one-sided Jacobi SVD A = U diag(s) V^T of a p x q matrix
//    (Hestenes' method, columns orthogonalised by plane rotations in a
//    round-robin ordering; singular values sorted in decreasing order).
#include "fastmath.cuh"
#include "small.h"
#include "trace.h"

#include <cmath>

namespace t2s2 {

namespace {

constexpr int kThreads = 512;
// the sweeps' column pairs: kPairLanes lanes each, kPairsPerWarp per warp
constexpr int kPairLanes = 8;
constexpr int kPairsPerWarp = 32 / kPairLanes;
constexpr size_t kJacobiSepSmem = 200 * 1024;  // pre-rotation with separate product buffers
constexpr size_t kJacobiMaxSmem = 224 * 1024;  // pre-rotation with in-place products

// G (c x c, row-major, ld c) -> L lower (G + shift I = L L^T), Linv = L^{-1}.
__global__ void __launch_bounds__(kThreads) chol_inv_kernel(const double* __restrict__ G, int c,
                                                            double shift_rel, double* __restrict__ L,
                                                            double* __restrict__ Linv, int* status) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double sm[];
  double* A = sm;           // c x c
  double* Iv = sm + c * c;  // c x c
  __shared__ double shift, tau;
  __shared__ int bad;
  const int t = threadIdx.x;
  for (int e = t; e < c * c; e += blockDim.x) A[e] = G[e];
  if (t == 0) {
    double tr = 0.0, mx = 0.0;
    for (int i = 0; i < c; ++i) {
      tr += G[i * c + i];
      mx = fmax(mx, G[i * c + i]);
    }
    shift = shift_rel * tr;
    // pivots below tau are roundoff-level directions (the matrix is only
    // positive semidefinite): their column of L is zeroed, so W = L Q still
    // holds and the matching row / column of Q is zero
    tau = 64.0 * 1.1102230246251565e-16 * (mx + shift);
    bad = 0;
  }
  __syncthreads();
  for (int i = t; i < c; i += blockDim.x) A[i * c + i] += shift;
  __syncthreads();
  // right-looking semidefinite Cholesky, lower triangle
  for (int j = 0; j < c; ++j) {
    const double v = A[j * c + j];
    const bool zero = !(v > tau);
    __syncthreads();
    if (zero) {
      for (int i = j + t; i < c; i += blockDim.x) A[i * c + j] = 0.0;
      if (t == 0) bad = 1;
      __syncthreads();
      continue;
    }
    const double rinv = drsqrt(v);  // 1 / L_jj
    for (int i = j + 1 + t; i < c; i += blockDim.x) A[i * c + j] *= rinv;
    if (t == 0) A[j * c + j] = v * rinv;
    __syncthreads();
    int rem = c - j - 1;
    for (int e = t; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) A[i * c + k] -= A[i * c + j] * A[k * c + j];
    }
    __syncthreads();
  }
  // pseudo-inverse of the lower-triangular L: column k solves L x = e_k with
  // x_i = 0 wherever L_ii = 0 (one thread per column)
  for (int e = t; e < c * c; e += blockDim.x) Iv[e] = 0.0;
  __syncthreads();
  for (int k = t; k < c; k += blockDim.x) {
    for (int i = k; i < c; ++i) {
      const double dii = A[i * c + i];
      if (dii == 0.0) {
        Iv[i * c + k] = 0.0;
        continue;
      }
      double s = (i == k) ? 1.0 : 0.0;
      for (int l = k; l < i; ++l) s -= A[i * c + l] * Iv[l * c + k];
      Iv[i * c + k] = s * drcp(dii);
    }
  }
  __syncthreads();
  for (int e = t; e < c * c; e += blockDim.x) {
    int i = e / c, k = e % c;
    L[e] = (k <= i) ? A[e] : 0.0;
    Linv[e] = (k <= i) ? Iv[e] : 0.0;
  }
  if (t == 0 && status) *status = bad;
}

// One-sided Jacobi on the columns of W (p x q, p >= q) held in shared memory.
// V (q x q) accumulates the rotations.  Returns sorted s, U = W / s, V.
__global__ void __launch_bounds__(kThreads) jacobi_svd_kernel(const double* __restrict__ A, int p,
                                                              int q, int transpose,
                                                              double* __restrict__ U,
                                                              double* __restrict__ s_out,
                                                              double* __restrict__ V, int* sweeps_out,
                                                              int prerotate) {
  pdl_wait();
  pdl_trigger();
  // Working matrix W is rows x cols with rows >= cols (transposed input if p < q).
  extern __shared__ double sm[];
  const int rows = transpose ? q : p, cols = transpose ? p : q;
  double* W = sm;                        // rows x cols, column-major for rotations
  double* Vs = sm + rows * cols;         // cols x cols, column-major
  double* nrm = Vs + cols * cols;        // cols
  __shared__ int rotated;
  __shared__ unsigned top32;
  __shared__ int order[kSmallMax];
  const int t = threadIdx.x;
  for (int e = t; e < rows * cols; e += blockDim.x) {
    int i = e % rows, j = e / rows;  // W(i,j)
    W[j * rows + i] = transpose ? A[j * q + i] : A[i * q + j];
  }
  for (int e = t; e < cols * cols; e += blockDim.x) Vs[e] = (e % cols == e / cols) ? 1.0 : 0.0;
  __shared__ double fro2;
  __shared__ double wsum[kThreads / 32];
  __syncthreads();
  {
    double acc = 0.0;
    for (int e = t; e < rows * cols; e += blockDim.x) acc = fma(W[e], W[e], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) wsum[t / 32] = acc;
  }
  __syncthreads();
  if (t == 0) {  // fixed order: the result does not depend on timing
    double acc = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) acc += wsum[w];
    fro2 = acc;
  }
  __syncthreads();
  // a column whose squared norm is below this is zero to working precision
  // (e.g. a direction the semidefinite Cholesky zeroed): rotating it only
  // stirs roundoff, and the sweeps would never settle
  const double negligible = 1e-32 * fro2;
  const int warp = t / 32, lane = t % 32, nwarps = blockDim.x / 32;
  const int grp = lane / kPairLanes, gl = lane % kPairLanes;  // pair group, lane in it
  const int npair = (cols + 1) / 2;  // round-robin with a dummy column when cols is odd
  const int ncol = 2 * npair;
  // Binary32 pre-rotation.  A binary64 instruction costs a warp ~64 issue
  // cycles on this part (2 DFMA/clk/SM), binary32 one: the sweeps run in
  // binary32 on a rounded copy until its columns are orthogonal to ~1e-6
  // (or the binary32 noise stops them), W <- W V32 in binary64, and one
  // binary64 sweep below (starting from V = V32) converges quadratically
  // to the stopping test.  Small
  // singular values keep full binary64 relative accuracy: they come from
  // binary64 column norms after the binary64 rotations.
  if (prerotate) {
    // prerotate 1: separate binary64 buffers for V^T V, the Newton-Schulz
    // iterate and W V; prerotate 2 (blocks too large for those): V^T V over
    // the binary32 copies (cols^2 doubles <= (rows + cols) cols floats) and
    // both products row by row in place -- a warp reads a row of V (or W)
    // whole before it writes it, and no other warp touches that row
    const bool inplace = prerotate == 2;
    float* Wf = reinterpret_cast<float*>(nrm + cols);
    float* Vf = Wf + rows * cols;
    // keep Wt 8-byte aligned: pad the float arrays to an even count
    double* Wt = inplace ? reinterpret_cast<double*>(Wf)
                         : reinterpret_cast<double*>(Vf + cols * cols + ((rows * cols + cols * cols) & 1));
    for (int e = t; e < rows * cols; e += blockDim.x) Wf[e] = (float)W[e];
    for (int e = t; e < cols * cols; e += blockDim.x) Vf[e] = (e % cols == e / cols) ? 1.f : 0.f;
    const float negl32 = (float)(1e-14 * fro2);
    // the sweeps stop when no rotation exceeds |gamma| = 1e-6 sqrt(alpha beta),
    // or when the largest one is below ~3e-5 and no longer shrinks tenfold a
    // sweep: binary32 dot products carry ~1e-7 relative noise per term, so the
    // last rotations can stall at the noise (without this stop such blocks
    // ran all 30 sweeps), and the binary64 sweeps below converge from there
    float prev_top = 1.f;
    for (int sw = 0; sw < 30; ++sw) {
      if (t == 0) {
        rotated = 0;
        top32 = 0u;
      }
      __syncthreads();
      for (int round = 0; round < ncol - 1; ++round) {
        for (int pr0 = warp * kPairsPerWarp; pr0 < npair; pr0 += nwarps * kPairsPerWarp) {
          // kPairsPerWarp pairs per warp, kPairLanes lanes each (the shuffle
          // trip counts stay warp-uniform: idle groups reduce zeros)
          const int pr = pr0 + grp;
          int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (ncol - 1);
          int b = 1 + (ncol - 2 - pr + round) % (ncol - 1);
          const bool act = pr < npair && a < cols && b < cols;
          if (a > b) { int tmp = a; a = b; b = tmp; }
          float* wa = Wf + (act ? a : 0) * rows;
          float* wb = Wf + (act ? b : 0) * rows;
          float alpha = 0.f, beta = 0.f, gamma = 0.f;
          if (act) {
            for (int i = gl; i < rows; i += kPairLanes) {
              alpha = fmaf(wa[i], wa[i], alpha);
              beta = fmaf(wb[i], wb[i], beta);
              gamma = fmaf(wa[i], wb[i], gamma);
            }
          }
          for (int o = kPairLanes / 2; o > 0; o >>= 1) {
            alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
            beta += __shfl_xor_sync(0xffffffffu, beta, o);
            gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
          }
          if (act && gamma != 0.f && gamma * gamma > 1e-12f * alpha * beta && alpha > negl32 && beta > negl32) {
            const float diff = beta - alpha, g2 = 2.f * gamma;
            const float tf = (diff >= 0.f ? g2 : -g2) / (fabsf(diff) + sqrtf(fmaf(diff, diff, g2 * g2)));
            const float cs = rsqrtf(fmaf(tf, tf, 1.f)), sn = cs * tf;
            for (int i = gl; i < rows; i += kPairLanes) {
              const float x = wa[i], y = wb[i];
              wa[i] = cs * x - sn * y;
              wb[i] = sn * x + cs * y;
            }
            float* va = Vf + a * cols;
            float* vb = Vf + b * cols;
            for (int i = gl; i < cols; i += kPairLanes) {
              const float x = va[i], y = vb[i];
              va[i] = cs * x - sn * y;
              vb[i] = sn * x + cs * y;
            }
            if (gl == 0) {
              rotated = 1;
              // non-negative binary32 values order like their bit patterns
              atomicMax(&top32, __float_as_uint(gamma * gamma / (alpha * beta)));
            }
          }
        }
        __syncthreads();
      }
      const float top = __uint_as_float(top32);
      if (!rotated || (top < 1e-9f && top > 0.01f * prev_top)) break;
      prev_top = top;
      __syncthreads();
    }
    // V32 is orthogonal only to ~1e-7: make it orthogonal in binary64 with
    // two Newton-Schulz steps V <- V (3 I - V^T V) / 2 (quadratic: 1e-7 ->
    // 1e-14 -> roundoff), so that W0 = W V^T stays exact for the caller
    for (int e = t; e < cols * cols; e += blockDim.x) Vs[e] = (double)Vf[e];
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
      for (int e = t; e < cols * cols; e += blockDim.x) {  // Wt <- V^T V
        const int i = e % cols, j = e / cols;
        double acc = 0.0;
        for (int k = 0; k < cols; ++k) acc = fma(Vs[i * cols + k], Vs[j * cols + k], acc);
        Wt[e] = acc;
      }
      __syncthreads();
      if (inplace) {
        for (int r = warp; r < cols; r += nwarps) {  // row r of V <- 1.5 V_r - 0.5 V_r Wt
          double o[kSmallMax / 32];
#pragma unroll
          for (int u = 0; u < kSmallMax / 32; ++u) {
            const int j = lane + 32 * u;
            if (j < cols) {
              double acc = 0.0;
              for (int c = 0; c < cols; ++c) acc = fma(Vs[c * cols + r], Wt[j * cols + c], acc);
              o[u] = fma(1.5, Vs[j * cols + r], -0.5 * acc);
            }
          }
          __syncwarp();
#pragma unroll
          for (int u = 0; u < kSmallMax / 32; ++u) {
            const int j = lane + 32 * u;
            if (j < cols) Vs[j * cols + r] = o[u];
          }
        }
        __syncthreads();
      } else {
        double* V2 = Wt + rows * cols;  // cols x cols
        for (int e = t; e < cols * cols; e += blockDim.x) {  // V2 <- V (3 I - V^T V) / 2
          const int k = e % cols, j = e / cols;
          double acc = 0.0;
          for (int i = 0; i < cols; ++i) acc = fma(Vs[i * cols + k], ((i == j) ? 3.0 : 0.0) - Wt[j * cols + i], acc);
          V2[e] = 0.5 * acc;
        }
        __syncthreads();
        for (int e = t; e < cols * cols; e += blockDim.x) Vs[e] = V2[e];
        __syncthreads();
      }
    }
    // W <- W V, in binary64
    if (inplace) {
      for (int r = warp; r < rows; r += nwarps) {
        double o[kSmallMax / 32];
#pragma unroll
        for (int u = 0; u < kSmallMax / 32; ++u) {
          const int j = lane + 32 * u;
          if (j < cols) {
            double acc = 0.0;
            for (int k = 0; k < cols; ++k) acc = fma(W[k * rows + r], Vs[j * cols + k], acc);
            o[u] = acc;
          }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kSmallMax / 32; ++u) {
          const int j = lane + 32 * u;
          if (j < cols) W[j * rows + r] = o[u];
        }
      }
      __syncthreads();
    } else {
      for (int e = t; e < rows * cols; e += blockDim.x) {
        const int i = e % rows, j = e / rows;
        double acc = 0.0;
        for (int k = 0; k < cols; ++k) acc = fma(W[k * rows + i], Vs[j * cols + k], acc);
        Wt[e] = acc;
      }
      __syncthreads();
      for (int e = t; e < rows * cols; e += blockDim.x) W[e] = Wt[e];
      __syncthreads();
    }
  }
  int sweep = 0;
  for (sweep = 0; sweep < 60; ++sweep) {
    if (t == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < ncol - 1; ++round) {
      for (int pr0 = warp * kPairsPerWarp; pr0 < npair; pr0 += nwarps * kPairsPerWarp) {
        // round-robin pairing: position 0 fixed, others rotate; kPairsPerWarp
        // pairs per warp share each binary64 instruction (a binary64 warp
        // instruction costs the same ~64 cycles with 8 or 32 lanes busy)
        const int pr = pr0 + grp;
        int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (ncol - 1);
        int b = 1 + (ncol - 2 - pr + round) % (ncol - 1);
        const bool act = pr < npair && a < cols && b < cols;
        if (a > b) { int tmp = a; a = b; b = tmp; }
        double* wa = W + (act ? a : 0) * rows;
        double* wb = W + (act ? b : 0) * rows;
        double alpha = 0, beta = 0, gamma = 0;
        if (act) {
          for (int i = gl; i < rows; i += kPairLanes) {
            alpha += wa[i] * wa[i];
            beta += wb[i] * wb[i];
            gamma += wa[i] * wb[i];
          }
        }
        for (int o = kPairLanes / 2; o > 0; o >>= 1) {
          alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
          beta += __shfl_xor_sync(0xffffffffu, beta, o);
          gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
        }
        if (act && gamma != 0.0 && gamma * gamma > 1e-30 * alpha * beta && alpha > negligible && beta > negligible) {
          // Rotation angle in binary32 (only its orthogonality must be exact):
          // t = 2 gamma sign(beta - alpha) / (|beta - alpha| + sqrt((beta - alpha)^2 + 4 gamma^2)).
          // Near convergence a binary32 angle still cuts gamma by ~1e-7 per sweep.
          const double diff = beta - alpha, g2 = 2.0 * gamma;
          const double mm = fmax(fabs(diff), fabs(g2));
          float df, gf;
          if (mm > 1e-30 && mm < 1e30) {
            const float inv = 1.0f / (float)mm;
            df = (float)diff * inv;
            gf = (float)g2 * inv;
          } else {
            const double inv = 1.0 / mm;
            df = (float)(diff * inv);
            gf = (float)(g2 * inv);
          }
          const float tf = (df >= 0.f ? gf : -gf) / (fabsf(df) + sqrtf(fmaf(df, df, gf * gf)));
          double cs = (double)rsqrtf(fmaf(tf, tf, 1.0f));
          double sn = cs * (double)tf;
          // renormalise in binary64: two Newton steps on 1/sqrt(cs^2 + sn^2)
          double n2 = fma(cs, cs, sn * sn);
          double f = fma(-0.5, n2, 1.5);
          cs *= f;
          sn *= f;
          n2 = fma(cs, cs, sn * sn);
          f = fma(-0.5, n2, 1.5);
          cs *= f;
          sn *= f;
          for (int i = gl; i < rows; i += kPairLanes) {
            double x = wa[i], y = wb[i];
            wa[i] = cs * x - sn * y;
            wb[i] = sn * x + cs * y;
          }
          double* va = Vs + a * cols;
          double* vb = Vs + b * cols;
          for (int i = gl; i < cols; i += kPairLanes) {
            double x = va[i], y = vb[i];
            va[i] = cs * x - sn * y;
            vb[i] = sn * x + cs * y;
          }
          // a sweep whose rotations were all below 1e-4 (relative) leaves
          // off-diagonals of ~1e-8 (quadratic convergence): it is the last.
          // The column norms then carry ~1e-16 relative error as singular
          // values, W = U diag(s) V^T holds with V orthogonal to roundoff,
          // and the left vectors are orthogonal to ~1e-8 (the sweeps that
          // consume them re-orthogonalise with CholeskyQR anyway).  After
          // the binary32 pre-rotation this is the first binary64 sweep.
          if (gl == 0 && gamma * gamma > 1e-8 * alpha * beta) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  for (int j = warp; j < cols; j += nwarps) {
    double s = 0;
    for (int i = lane; i < rows; i += 32) s += W[j * rows + i] * W[j * rows + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[j] = dsqrt(s);
  }
  __syncthreads();
  if (t == 0) {  // selection sort of column order by decreasing norm (cols <= kSmallMax)
    for (int j = 0; j < cols; ++j) order[j] = j;
    for (int j = 0; j < cols; ++j) {
      int best = j;
      for (int l = j + 1; l < cols; ++l)
        if (nrm[order[l]] > nrm[order[best]]) best = l;
      int tmp = order[j]; order[j] = order[best]; order[best] = tmp;
    }
    if (sweeps_out) *sweeps_out = sweep;
  }
  __syncthreads();
  // Outputs: A = U diag(s) V^T with U p x k, V q x k, k = cols (= min(p,q)).
  // Working problem: W0 = Wfinal V^T.  If transpose, A = W0^T = V diag(s) U_w^T.
  const int k = cols;
  for (int j = t; j < k; j += blockDim.x) s_out[j] = nrm[order[j]];
  for (int e = t; e < rows * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    int cj = order[j];
    double sj = nrm[cj];
    double u = (sj > 0) ? W[cj * rows + i] / sj : ((i == j) ? 1.0 : 0.0);
    if (!transpose) U[i * k + j] = u;   // U: p x k
    else V[i * k + j] = u;              // V: q x k (rows == q)
  }
  for (int e = t; e < cols * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    double v = Vs[order[j] * cols + i];
    if (!transpose) V[i * k + j] = v;   // V: q x k
    else U[i * k + j] = v;              // U: p x k (cols == p)
  }
}

}  // namespace

t2s2_status chol_inv(const double* G, int c, double shift_rel, double* L, double* Linv, int* status,
                     cudaStream_t st) {
  if (c <= 0 || c > kSmallMax) return T2S2_EINVAL;
  size_t smem = (size_t)2 * c * c * sizeof(double);
  static bool attr = false;
  if (!attr) {
    T2S2_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * kSmallMax * kSmallMax * (int)sizeof(double)));
    attr = true;
  }
  TraceScope ts(kTrSmall, st, (double)c * c * c, 8.0 * 3 * c * c);
  const int nt = c <= 32 ? 32 : (c <= 64 ? 128 : 256);
  (void)launch_pdl(chol_inv_kernel, 1, nt, smem, st, G, c, shift_rel, L, Linv, status);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

t2s2_status jacobi_svd(const double* A, int p, int q, double* U, double* s, double* V, int* sweeps,
                       cudaStream_t st) {
  if (p <= 0 || q <= 0 || p > kSmallMax || q > kSmallMax) return T2S2_EINVAL;
  int transpose = p < q;
  int rows = transpose ? q : p, cols = transpose ? p : q;
  size_t smem = ((size_t)rows * cols + (size_t)cols * cols + cols) * sizeof(double);
  // binary32 pre-rotation: with separate product buffers when they fit in
  // kJacobiSepSmem, else with the products in place when the binary32
  // copies fit in kJacobiMaxSmem
  const size_t copies = ((size_t)rows * cols + (size_t)cols * cols + 1) * sizeof(float) + 16;
  const size_t buffers = ((size_t)rows * cols + (size_t)cols * cols) * sizeof(double);
  int prerotate = 0;
  if (smem + copies + buffers <= kJacobiSepSmem) {
    prerotate = 1;
    smem += copies + buffers;
  } else if (smem + copies <= kJacobiMaxSmem) {
    prerotate = 2;
    smem += copies;
  }
  static bool attr = false;
  if (!attr) {
    T2S2_CUDA_TRY(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kJacobiMaxSmem));
    attr = true;
  }
  TraceScope ts(kTrSmall, st, 6.0 * 8 * (double)rows * cols * cols, 8.0 * (2.0 * p * q + q * q));
  (void)launch_pdl(jacobi_svd_kernel, 1, kThreads, smem, st, A, p, q, transpose, U, s, V, sweeps, prerotate);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

}  // namespace t2s2
