// Local solve with a right interface of rank one, in one CTA.
//
// With rb = 1 the local system of the sweep, (P_L (+) B' (+) P_R) X = F, is the
// Sylvester equation
//     P_L X + X B'^T + pi X = F,      X: ra x m,  pi = P_R (a scalar).
// In the complex Schur basis of the 1D operator, B' = Z Ts Z^H with
// Ts = c_op T + shift I (computed once per operator), Y = X conj(Z) and
// G = F conj(Z) satisfy
//     (P_L + (Ts_ii + pi) I) y_i = g_i - sum_{j > i} Ts_ij y_j,   i = m-1 .. 0,
// m shifted ra x ra systems solved one after another.  The kernel inverts the
// m shifted matrices once (Gauss-Jordan with partial pivoting, complex
// binary32, one warp each), uses the resulting binary32 solver as the
// preconditioner of a binary64 iterative refinement X <- X + M^{-1}(F - K X),
// and stops when ||F - K X|| <= tol ||F||.  A vanishing pivot, a step that cuts
// the residual less than tenfold, or the step cap ends it with status 1: the
// iterate stays in x, and the general solver queued behind this kernel (the
// interface eigendecompositions and the GMRES team) runs from it.  On status 0
// those kernels return at once.
#include <cuda_runtime.h>

#include <algorithm>

#include "eig.cuh"
#include "local.h"
#include "trace.h"

namespace t2s2 {

namespace {

constexpr int kSylvThreads = 256;
constexpr int kSylvMaxRa = 32;
constexpr int kSylvMaxSteps = 6;
constexpr size_t kSylvMaxSmem = 160 * 1024;

size_t sylv_smem_bytes(int ra, int m) {
  const size_t dbl = (size_t)ra * ra + (size_t)m * m + 3 * (size_t)ra * m;
  const size_t cpx = 2 * (size_t)m * m + (size_t)m * ra * ra + (size_t)ra * m + kSylvMaxRa;
  return sizeof(double) * dbl + sizeof(cf) * cpx;
}

__device__ __forceinline__ cf cinv(cf a) {
  const float d = __frcp_rn(cabs2(a));
  return cmk(a.x * d, -a.y * d);
}

__global__ void __launch_bounds__(kSylvThreads) sylv_rb1_kernel(SylvProblem P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ra = P.ra, m = P.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double* PL = reinterpret_cast<double*>(smem);  // ra x ra
  double* Bp = PL + ra * ra;                      // m x m
  double* X = Bp + m * m;                         // ra x m
  double* R = X + ra * m;                         // ra x m
  double* F = R + ra * m;                         // ra x m
  cf* Ts = reinterpret_cast<cf*>(F + ra * m);     // m x m (upper triangle)
  cf* Z = Ts + m * m;                             // m x m
  cf* Inv = Z + m * m;                            // m matrices ra x ra
  cf* G = Inv + (size_t)m * ra * ra;              // ra x m: G, then Y in place
  cf* tv = G + ra * m;                            // kSylvMaxRa: one right-hand side
  __shared__ double red[kSylvThreads / 32];
  __shared__ int fail;
  const double pi = P.PR[0];
  const float cop = (float)P.c_op, sh = (float)P.shift;
  for (int e = t; e < ra * ra; e += kSylvThreads) PL[e] = P.PL[e];
  for (int e = t; e < m * m; e += kSylvThreads) {
    Bp[e] = P.Bp[e];
    const int i = e / m, j = e % m;
    Ts[e] = cmk(cop * P.Tr[e] + (i == j ? sh : 0.f), cop * P.Ti[e]);
    Z[e] = cmk(P.Zr[e], P.Zi[e]);
  }
  for (int e = t; e < ra * m; e += kSylvThreads) {
    X[e] = P.x[e];
    F[e] = P.rhs[e];
  }
  if (t == 0) fail = 0;
  __syncthreads();
  // inverses of A_i = P_L + (Ts_ii + pi) I, one warp each; lane = row
  for (int i = warp; i < m; i += kSylvThreads / 32) {
    cf* A = Inv + (size_t)i * ra * ra;
    const cf s = cadd(Ts[i * m + i], cmk((float)pi, 0.f));
    for (int e = lane; e < ra * ra; e += 32) {
      const int p = e / ra, q = e % ra;
      A[e] = cadd(cmk((float)PL[e], 0.f), p == q ? s : cmk(0.f, 0.f));
    }
    __syncwarp();
    float amax = 0.f;
    for (int e = lane; e < ra * ra; e += 32) amax = fmaxf(amax, cabs2(A[e]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    int perm[kSylvMaxRa];
    bool bad = false;
    for (int p = 0; p < ra; ++p) {
      // pivot: largest |a_qp| over q >= p (ties: smallest q)
      // (non-negative binary32 values order like their bit patterns)
      const unsigned mine = (lane >= p && lane < ra) ? __float_as_uint(cabs2(A[lane * ra + p])) : 0u;
      const unsigned top = __reduce_max_sync(0xffffffffu, mine);
      const unsigned who = __ballot_sync(0xffffffffu, lane >= p && lane < ra && mine == top);
      const int arg = __ffs(who) - 1;
      const float best = __uint_as_float(top);
      perm[p] = arg;
      if (!(best > 1e-24f * amax)) bad = true;
      if (arg != p)
        for (int c = lane; c < ra; c += 32) {
          const cf u = A[p * ra + c];
          A[p * ra + c] = A[arg * ra + c];
          A[arg * ra + c] = u;
        }
      __syncwarp();
      const cf ip = bad ? cmk(0.f, 0.f) : cinv(A[p * ra + p]);
      __syncwarp();
      for (int c = lane; c < ra; c += 32) A[p * ra + c] = cmul(c == p ? cmk(1.f, 0.f) : A[p * ra + c], ip);
      __syncwarp();
      if (lane < ra && lane != p) {
        const cf f = A[lane * ra + p];
        A[lane * ra + p] = cmk(0.f, 0.f);
        for (int c = 0; c < ra; ++c) A[lane * ra + c] = csub(A[lane * ra + c], cmul(f, A[p * ra + c]));
      }
      __syncwarp();
    }
    // undo the row swaps as column swaps, last first
    for (int p = ra - 1; p >= 0; --p) {
      const int q = perm[p];
      if (q != p)
        for (int r = lane; r < ra; r += 32) {
          const cf u = A[r * ra + p];
          A[r * ra + p] = A[r * ra + q];
          A[r * ra + q] = u;
        }
      __syncwarp();
    }
    if (bad && lane == 0) fail = 1;
  }
  __syncthreads();
  int status = fail ? 1 : 0;
  double rr = 0.0, ff = 0.0, rr_prev = -1.0;
  int its = 0;
  for (int step = 0; status == 0; ++step) {
    // R = F - K X in binary64, ||R||^2 (and ||F||^2 at first)
    double pr = 0.0, pf = 0.0;
    for (int e = t; e < ra * m; e += kSylvThreads) {
      const int a = e / m, i = e % m;
      double s0 = pi * X[e], s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int p = 0; p < ra; ++p) s0 = fma(PL[a * ra + p], X[p * m + i], s0);
      int j = 0;
      for (; j + 2 < m; j += 3) {
        s1 = fma(Bp[i * m + j], X[a * m + j], s1);
        s2 = fma(Bp[i * m + j + 1], X[a * m + j + 1], s2);
        s3 = fma(Bp[i * m + j + 2], X[a * m + j + 2], s3);
      }
      for (; j < m; ++j) s1 = fma(Bp[i * m + j], X[a * m + j], s1);
      const double r = F[e] - ((s0 + s1) + (s2 + s3));
      R[e] = r;
      pr = fma(r, r, pr);
      if (step == 0) pf = fma(F[e], F[e], pf);
    }
    for (int o = 16; o > 0; o >>= 1) {
      pr += __shfl_xor_sync(0xffffffffu, pr, o);
      pf += __shfl_xor_sync(0xffffffffu, pf, o);
    }
    if (lane == 0) red[warp] = pr;
    __syncthreads();
    rr = 0.0;
    for (int w = 0; w < kSylvThreads / 32; ++w) rr += red[w];
    __syncthreads();
    if (step == 0) {
      if (lane == 0) red[warp] = pf;
      __syncthreads();
      for (int w = 0; w < kSylvThreads / 32; ++w) ff += red[w];
      __syncthreads();
    }
    if (rr <= P.tol_rel * P.tol_rel * ff || rr == 0.0) break;  // converged
    if ((rr_prev >= 0.0 && rr > 0.01 * rr_prev) || step == kSylvMaxSteps) {
      status = 1;  // not paying off: the general solver takes over
      break;
    }
    rr_prev = rr;
    // G = R conj(Z)
    for (int e = t; e < ra * m; e += kSylvThreads) {
      const int a = e / m, i = e % m;
      float gr = 0.f, gi = 0.f;
      for (int j = 0; j < m; ++j) {
        const float rv = (float)R[a * m + j];
        const cf z = Z[j * m + i];
        gr = fmaf(rv, z.x, gr);
        gi = fmaf(-rv, z.y, gi);
      }
      G[e] = cmk(gr, gi);
    }
    __syncthreads();
    // y_i = A_i^{-1} (g_i - sum_{j > i} Ts_ij y_j), i = m-1 .. 0 (warp 0;
    // lane = row a), Y over G in place
    if (warp == 0) {
      for (int i = m - 1; i >= 0; --i) {
        if (lane < ra) {
          cf s = G[lane * m + i];
          for (int j = i + 1; j < m; ++j) s = csub(s, cmul(Ts[i * m + j], G[lane * m + j]));
          tv[lane] = s;
        }
        __syncwarp();
        if (lane < ra) {
          const cf* A = Inv + (size_t)i * ra * ra + lane * ra;
          cf y = cmk(0.f, 0.f);
          for (int q = 0; q < ra; ++q) y = cadd(y, cmul(A[q], tv[q]));
          G[lane * m + i] = y;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // X += Re(Y Z^T)
    for (int e = t; e < ra * m; e += kSylvThreads) {
      const int a = e / m, i = e % m;
      float d = 0.f;
      for (int j = 0; j < m; ++j) {
        const cf y = G[a * m + j], z = Z[i * m + j];
        d = fmaf(y.x, z.x, fmaf(-y.y, z.y, d));
      }
      X[e] += (double)d;
    }
    ++its;
    __syncthreads();
  }
  for (int e = t; e < ra * m; e += kSylvThreads) P.x[e] = X[e];
  if (t == 0) {
    *P.status = status;
    if (P.iters_out) *P.iters_out = its;
    if (P.res_out) {
      P.res_out[0] = sqrt(rr);
      P.res_out[1] = sqrt(ff);
    }
  }
}

}  // namespace

bool sylv_rb1_fits(int ra, int m) {
  return ra >= 1 && ra <= kSylvMaxRa && m >= 1 && sylv_smem_bytes(ra, m) <= kSylvMaxSmem;
}

t2s2_status sylv_rb1(const SylvProblem& P, cudaStream_t st) {
  if (!sylv_rb1_fits(P.ra, P.m) || !P.status) return T2S2_EINVAL;
  static bool attr = false;
  if (!attr) {
    T2S2_CUDA_TRY(cudaFuncSetAttribute(sylv_rb1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSylvMaxSmem));
    attr = true;
  }
  const size_t smem = sylv_smem_bytes(P.ra, P.m);
  const double N = (double)P.ra * P.m;
  TraceScope ts(kTrLocal, st, 2.0 * N * (P.ra + P.m) * 3.0, 0.0);
  sylv_rb1_kernel<<<1, kSylvThreads, smem, st>>>(P);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

}  // namespace t2s2
