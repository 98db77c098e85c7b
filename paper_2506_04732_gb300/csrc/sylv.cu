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

constexpr int kSylvThreads = 512;
constexpr int kSylvMaxRa = 32;
constexpr int kSylvMaxSteps = 6;
constexpr int kSylvBlock = 8;  // columns of the backward substitution per serial block
constexpr size_t kSylvMaxSmem = 160 * 1024;

// Leading dimensions: odd counts of 8-byte words per row, so that lanes
// walking down a column hit different shared-memory banks.
__host__ __device__ inline int sylv_ld(int n) { return n | 1; }

size_t sylv_smem_bytes(int ra, int m) {
  const size_t lm = sylv_ld(m), la = sylv_ld(ra);
  const size_t dbl = (size_t)ra * ra + (size_t)m * lm + 3 * (size_t)ra * m;
  const size_t cpx = 2 * (size_t)m * lm + (size_t)m * ra * la + (size_t)ra * lm + kSylvMaxRa +
                     (size_t)(kSylvThreads / 32) * kSylvMaxRa;
  return sizeof(double) * dbl + sizeof(cf) * cpx + sizeof(float) * (size_t)ra * ra;
}

__device__ __forceinline__ unsigned long long sylv_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ cf cinv(cf a) {
  const float d = __frcp_rn(cabs2(a));
  return cmk(a.x * d, -a.y * d);
}

// Gauss-Jordan inverses (partial pivoting) of A_i = P_L + (Ts_ii + pi) I for
// i < m, 32 / W matrices per warp, each on W lanes: lane = row (lane =
// column for the pivot-row steps); segment-local maxima by shuffles within
// the W lanes.  A vanishing pivot sets *fail.
template <int W>
__device__ void sylv_invert(cf* Inv, const cf* Ts, const float* PL, double pi, int ra, int la, int lm, int m,
                            cf* prow_w, int warp, int nwarps, int lane, int* fail) {
  constexpr int S = 32 / W;
  const int seg = lane / W, sl = lane % W;
  cf* pr = prow_w + seg * W;
  for (int i0 = warp * S; i0 < m; i0 += nwarps * S) {
    const int i = i0 + seg;
    const bool act = i < m;
    cf* A = Inv + (size_t)(act ? i : 0) * ra * la;
    float amax = 0.f;
    if (act) {
      const cf s = cadd(Ts[i * lm + i], cmk((float)pi, 0.f));
      for (int e = sl; e < ra * ra; e += W) {
        const int p = e / ra, q = e % ra;
        const cf v = cadd(cmk(PL[e], 0.f), p == q ? s : cmk(0.f, 0.f));
        A[p * la + q] = v;
        amax = fmaxf(amax, cabs2(v));
      }
    }
    for (int o = W / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncwarp();
    int perm[kSylvMaxRa];
    bool bad = false;
    for (int p = 0; p < ra; ++p) {
      // pivot: largest |a_qp| over q >= p, ties to the smallest q
      // (non-negative binary32 values order like their bit patterns)
      const bool cand = act && sl >= p && sl < ra;
      const unsigned mine = cand ? __float_as_uint(cabs2(A[sl * la + p])) : 0u;
      unsigned top = mine;
      for (int o = W / 2; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
      const unsigned who = __ballot_sync(0xffffffffu, cand && mine == top);
      unsigned segbits = who;
      if constexpr (W < 32) segbits = (who >> (seg * W)) & ((1u << W) - 1u);
      const int arg = segbits ? __ffs(segbits) - 1 : p;
      perm[p] = arg;
      if (act && !(__uint_as_float(top) > 1e-24f * amax)) bad = true;
      // row arg -> pivot row (scaled by 1 / pivot, the pivot slot set to 1),
      // row p -> row arg
      if (act && sl < ra) {
        const cf piv = A[arg * la + p];
        const cf ip = bad ? cmk(0.f, 0.f) : cinv(piv);
        const cf vp = A[arg * la + sl], vq = A[p * la + sl];
        pr[sl] = cmul(sl == p ? cmk(1.f, 0.f) : vp, ip);
        if (arg != p) A[arg * la + sl] = vq;
      }
      __syncwarp();
      if (act && sl < ra) {
        cf* __restrict__ row = A + sl * la;
        const cf* __restrict__ prr = pr;
        if (sl == p) {
          for (int c = 0; c < ra; ++c) row[c] = prr[c];
        } else {
          const cf f = row[p];
          for (int c = 0; c < ra; ++c) {
            const cf base = (c == p) ? cmk(0.f, 0.f) : row[c];
            row[c] = csub(base, cmul(f, prr[c]));
          }
        }
      }
      __syncwarp();
    }
    // undo the row swaps as column swaps, last first
    for (int p = ra - 1; p >= 0; --p) {
      const int q = perm[p];
      if (act && q != p && sl < ra) {
        const cf u = A[sl * la + p];
        A[sl * la + p] = A[sl * la + q];
        A[sl * la + q] = u;
      }
      __syncwarp();
    }
    if (act && bad && sl == 0) *fail = 1;
  }
}

__global__ void __launch_bounds__(kSylvThreads) sylv_rb1_kernel(SylvProblem P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  const int ra = P.ra, m = P.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int lm = sylv_ld(m), la = sylv_ld(ra);
  double* PL = reinterpret_cast<double*>(smem);  // ra x ra
  double* Bp = PL + ra * ra;                      // m x lm
  double* X = Bp + m * lm;                        // ra x m
  // ra x m: the residual, kept in binary32 (it only feeds the binary32
  // preconditioner, and a binary64 -> binary32 conversion holds the FP64 pipe)
  float* Rf = reinterpret_cast<float*>(X + ra * m);
  double* R = X + ra * m;                         // ra x m slot (holds Rf, then PLf)
  double* F = R + ra * m;                         // ra x m
  cf* Ts = reinterpret_cast<cf*>(F + ra * m);     // m x lm (upper triangle)
  cf* Z = Ts + m * lm;                            // m x lm
  cf* Inv = Z + m * lm;                           // m matrices ra x la
  cf* G = Inv + (size_t)m * ra * la;              // ra x lm: G, then Y in place
  cf* tv = G + ra * lm;                           // kSylvMaxRa: one right-hand side
  cf* prow = tv + kSylvMaxRa;                     // per warp: the pivot row
  float* PLf = reinterpret_cast<float*>(prow + (kSylvThreads / 32) * kSylvMaxRa);  // ra x ra, binary32
  __shared__ double red[kSylvThreads / 32 + 1], red2[kSylvThreads / 32 + 1];
  __shared__ int fail;
  int nst = 0;
  auto stamp = [&]() {
    if (P.tstamp && t == 0 && nst < kSylvStamps) P.tstamp[nst++] = sylv_clock();
  };
  stamp();
  const double pi = P.PR[0];
  const float cop = (float)P.c_op, sh = (float)P.shift;
  for (int e = t; e < ra * ra; e += kSylvThreads) {
    const double v = P.PL[e];
    PL[e] = v;
    PLf[e] = (float)v;
  }
  for (int e = t; e < m * m; e += kSylvThreads) {
    const int i = e / m, j = e % m;
    Bp[i * lm + j] = P.Bp[e];
    Ts[i * lm + j] = cmk(cop * P.Tr[e] + (i == j ? sh : 0.f), cop * P.Ti[e]);
    Z[i * lm + j] = cmk(P.Zr[e], P.Zi[e]);
  }
  for (int e = t; e < ra * m; e += kSylvThreads) {
    X[e] = P.x[e];
    F[e] = P.rhs[e];
  }
  if (t == 0) fail = 0;
  __syncthreads();
  stamp();
  // inverses of A_i = P_L + (Ts_ii + pi) I by Gauss-Jordan: two matrices per
  // warp (16-lane halves) when ra <= 16, else one
  if (ra <= 16)
    sylv_invert<16>(Inv, Ts, PLf, pi, ra, la, lm, m, prow + warp * kSylvMaxRa, warp, kSylvThreads / 32, lane, &fail);
  else
    sylv_invert<32>(Inv, Ts, PLf, pi, ra, la, lm, m, prow + warp * kSylvMaxRa, warp, kSylvThreads / 32, lane, &fail);
  __syncthreads();
  stamp();
  int status = fail ? 1 : 0;
  double rr = 0.0, ff = 0.0, rr_prev = -1.0;
  int its = 0;
  for (int step = 0; status == 0; ++step) {
    // R = F - K X in binary64, ||R||^2 (and ||F||^2 at first)
    double prs = 0.0, pfs = 0.0;
    {
      const double* __restrict__ Xr = X;
      const double* __restrict__ Br = Bp;
      const double* __restrict__ Pr = PL;
      const double* __restrict__ Fr = F;
      float* __restrict__ Rw = Rf;
      for (int e = t; e < ra * m; e += kSylvThreads) {
        const int a = e / m, i = e % m;
        double s0 = pi * Xr[e], s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int p = 0; p < ra; ++p) s0 = fma(Pr[a * ra + p], Xr[p * m + i], s0);
        int j = 0;
        for (; j + 2 < m; j += 3) {
          s1 = fma(Br[i * lm + j], Xr[a * m + j], s1);
          s2 = fma(Br[i * lm + j + 1], Xr[a * m + j + 1], s2);
          s3 = fma(Br[i * lm + j + 2], Xr[a * m + j + 2], s3);
        }
        for (; j < m; ++j) s1 = fma(Br[i * lm + j], Xr[a * m + j], s1);
        const double r = Fr[e] - ((s0 + s1) + (s2 + s3));
        Rw[e] = (float)r;
        prs = fma(r, r, prs);
        if (step == 0) pfs = fma(Fr[e], Fr[e], pfs);
      }
    }
    // binary64 sums: a warp instruction holds an FP64 pipe for ~64 cycles
    // whatever its active lanes, so only warps that hold terms reduce, and
    // one warp combines the per-warp sums
    const int wact = (min(kSylvThreads, ra * m) + 31) >> 5;
    if (warp < wact) {
      for (int o = 16; o > 0; o >>= 1) prs += __shfl_xor_sync(0xffffffffu, prs, o);
      if (step == 0)
        for (int o = 16; o > 0; o >>= 1) pfs += __shfl_xor_sync(0xffffffffu, pfs, o);
      if (lane == 0) {
        red[warp] = prs;
        red2[warp] = pfs;
      }
    }
    __syncthreads();
    if (warp == 0) {
      double v = lane < wact ? red[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      double f = 0.0;
      if (step == 0) {
        f = lane < wact ? red2[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      }
      if (lane == 0) {
        red[kSylvThreads / 32] = v;
        red2[kSylvThreads / 32] = f;
      }
    }
    __syncthreads();
    rr = red[kSylvThreads / 32];
    if (step == 0) ff = red2[kSylvThreads / 32];
    stamp();
    if (rr <= P.tol_rel * P.tol_rel * ff || rr == 0.0) break;  // converged
    if ((rr_prev >= 0.0 && rr > 0.01 * rr_prev) || step == kSylvMaxSteps) {
      status = 1;  // not paying off: the general solver takes over
      break;
    }
    rr_prev = rr;
    // G = R conj(Z)
    {
      const float* __restrict__ Rr = Rf;
      const cf* __restrict__ Zr = Z;
      cf* __restrict__ Gw = G;
      for (int e = t; e < ra * m; e += kSylvThreads) {
        const int a = e / m, i = e % m;
        float gr = 0.f, gi = 0.f, hr = 0.f, hi = 0.f;
        int j = 0;
        for (; j + 1 < m; j += 2) {
          const float rv = Rr[a * m + j], rw = Rr[a * m + j + 1];
          const cf z = Zr[j * lm + i], w = Zr[(j + 1) * lm + i];
          gr = fmaf(rv, z.x, gr);
          gi = fmaf(-rv, z.y, gi);
          hr = fmaf(rw, w.x, hr);
          hi = fmaf(-rw, w.y, hi);
        }
        if (j < m) {
          const float rv = Rr[a * m + j];
          const cf z = Zr[j * lm + i];
          gr = fmaf(rv, z.x, gr);
          gi = fmaf(-rv, z.y, gi);
        }
        Gw[a * lm + i] = cmk(gr + hr, gi + hi);
      }
    }
    __syncthreads();
    stamp();
    // y_i = A_i^{-1} (g_i - sum_{j > i} Ts_ij y_j), i = m-1 .. 0, Y over G in
    // place: blocks of kSylvBlock columns from the last; one warp solves a
    // block step by step with the in-block terms only, then all threads take
    // the block's contribution out of the earlier right-hand sides at once
    for (int hi = m - 1; hi >= 0; hi -= kSylvBlock) {
      const int lo = max(0, hi - kSylvBlock + 1);
      if (warp == 0) {
        const cf* __restrict__ Tr = Ts;
        for (int i = hi; i >= lo; --i) {
          if (lane < ra) {
            cf s = G[lane * lm + i];
            for (int j = i + 1; j <= hi; ++j) s = csub(s, cmul(Tr[i * lm + j], G[lane * lm + j]));
            tv[lane] = s;
          }
          __syncwarp();
          if (lane < ra) {
            const cf* __restrict__ A = Inv + (size_t)i * ra * la + lane * la;
            const cf* __restrict__ v = tv;
            cf y0 = cmk(0.f, 0.f), y1 = cmk(0.f, 0.f);
            int q = 0;
            for (; q + 1 < ra; q += 2) {
              y0 = cadd(y0, cmul(A[q], v[q]));
              y1 = cadd(y1, cmul(A[q + 1], v[q + 1]));
            }
            if (q < ra) y0 = cadd(y0, cmul(A[q], v[q]));
            G[lane * lm + i] = cadd(y0, y1);
          }
          __syncwarp();
        }
      }
      __syncthreads();
      {
        const cf* __restrict__ Tr = Ts;
        for (int e = t; e < ra * lo; e += kSylvThreads) {
          const int a = e / lo, j = e % lo;
          cf s = G[a * lm + j];
          for (int i = lo; i <= hi; ++i) s = csub(s, cmul(Tr[j * lm + i], G[a * lm + i]));
          G[a * lm + j] = s;
        }
      }
      __syncthreads();
    }
    stamp();
    // X += Re(Y Z^T)
    {
      const cf* __restrict__ Yr = G;
      const cf* __restrict__ Zr = Z;
      double* __restrict__ Xw = X;
      for (int e = t; e < ra * m; e += kSylvThreads) {
        const int a = e / m, i = e % m;
        float d0 = 0.f, d1 = 0.f;
        int j = 0;
        for (; j + 1 < m; j += 2) {
          const cf y = Yr[a * lm + j], z = Zr[i * lm + j], y2 = Yr[a * lm + j + 1], z2 = Zr[i * lm + j + 1];
          d0 = fmaf(y.x, z.x, fmaf(-y.y, z.y, d0));
          d1 = fmaf(y2.x, z2.x, fmaf(-y2.y, z2.y, d1));
        }
        if (j < m) {
          const cf y = Yr[a * lm + j], z = Zr[i * lm + j];
          d0 = fmaf(y.x, z.x, fmaf(-y.y, z.y, d0));
        }
        Xw[e] += (double)(d0 + d1);
      }
    }
    ++its;
    __syncthreads();
    stamp();
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
  TraceScope ts(kTrSylv, st, 2.0 * N * (P.ra + P.m) * 3.0, 0.0);
  (void)launch_pdl(sylv_rb1_kernel, 1, kSylvThreads, smem, st, P);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

}  // namespace t2s2
