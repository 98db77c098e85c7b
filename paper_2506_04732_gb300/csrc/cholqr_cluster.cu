// Shifted CholeskyQR (up to four passes) in ONE thread-block cluster.
//
// The same factorisation as cholqr.cu (shifted CholeskyQR3 of Fukaya et al.,
// L D L^T form with L^{-1} built in the same elimination steps, the
// CholeskyQR2 stopping argument, an exact power-of-4 scaling of the Gram),
// for the blocks of the TT sweeps that are small enough to live in the
// shared memory of at most 16 CTAs.  A cooperative grid pays two grid-wide
// barriers per pass (~2 us each on this part) and a launch that cannot
// overlap the previous kernel; a cluster pays one cluster barrier per pass
// (~0.2 us) and is launched with programmatic dependent launch:
//
//   pass p:
//     every CTA:  partial Gram of its own vectors into its shared memory
//                 (double-buffered by pass parity)            (cluster sync)
//     every CTA:  the Gram as the sum of all CTAs' partials, read through
//                 distributed shared memory in a fixed shuffle tree, so that
//                 every CTA holds the same Gram bit for bit; the L D L^T with
//                 L^{-1}; its own vectors v <- D^{-1/2} L^{-1} v; its own
//                 rows of Lacc <- Lacc L D^{1/2}
//
// When the last pass's Gram is I + E with |E| <= 1e-3, that pass needs no
// factorisation: T = (I + E)^(-1/2) and T^-1 = (I + E)^(1/2) are the first
// K terms of their binomial series (K such that |E|^(K+1) <= 2^-56), i.e.
// K - 1 products of c x c matrices that run in parallel instead of c
// dependent pivot steps; Q = V T (Loewdin's symmetric orthogonalisation), and
// R takes T^-1, so that it is then a full c x c matrix with W = Q R.
//
// A CTA reads the partials of pass p only before the barrier of pass p + 1,
// and a partial buffer is rewritten two passes later, after that barrier; a
// last barrier keeps every CTA's shared memory alive until all reads are
// done.  Binary64 issues one warp instruction per ~64 cycles per SM
// sub-partition here, so the pivot chain of the elimination (the next
// pivot's reciprocal, computed one step ahead) runs on a warp of its own
// while the other warps update the trailing block.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "fastmath.cuh"
#include "small.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int kThr = 256;
constexpr int kUpd = kThr - 32;  // threads of the trailing updates (warps 0..6)
constexpr int kMaxCl = 16;
constexpr size_t kClMaxSmem = 200 * 1024;
constexpr float kOrthDev = 0.5f;  // spectral distance of the last pass's Gram from I
constexpr double kUnitRoundoff = 1.1102230246251565e-16;  // 2^-53
// binary64 Gram products per CTA and pass the plan aims at (~0.3 us)
constexpr long kWorkPerCta = 2048;
// blocks above this many Gram products go to the full-grid kernel
constexpr long kMaxWork = 16L * 16384;
constexpr int kStamps = 2 + 6 * kCqrMaxPass + 1;
// the last pass takes the binomial series of (I + E)^(-1/2) instead of a
// Cholesky factorisation when its Gram is this close to I (spectral bound)
constexpr float kPolyDev = 1e-3f;
constexpr int kPolyMaxC = 32;
constexpr int kPolyMaxTerms = 6;
constexpr int kSumBatch = 4;  // remote partial-Gram loads in flight per thread

// binom(-1/2, p) and binom(1/2, p), p = 0..6: dyadic, exact in binary64
__constant__ double kSeriesA[kPolyMaxTerms + 1] = {1.0, -0.5, 0.375, -0.3125, 0.2734375, -0.24609375, 0.2255859375};
__constant__ double kSeriesB[kPolyMaxTerms + 1] = {1.0, 0.5, -0.125, 0.0625, -0.0390625, 0.02734375,
                                                   -0.0205078125};

struct CqrArgs {
  const double* W;
  const double* W2;  // tall only: columns c1 .. c-1 in a second block (null: one block)
  int c1;
  double* Q;
  double* R;
  int* status;
  int nlong, c, per, tall, slices;
  double shift_rel;
  unsigned long long* tstamp;  // diagnostics: phase times of CTA 0 (null: off)
};

__host__ __device__ inline int tri_count(int c) { return c * (c + 1) / 2; }

__host__ __device__ inline size_t cl_smem_bytes(int per, int c, int cl) {
  const int rpc = (c + cl - 1) / cl;
  const size_t T = (size_t)tri_count(c);
  const size_t poly = c <= kPolyMaxC ? 3 * (size_t)c * c : 0;
  return sizeof(double) *
             (2 * (size_t)per * c + 2 * T + 2 * (size_t)c * c + 2 * (size_t)rpc * c + 4 * (size_t)c + poly) +
         sizeof(int) * ((T + 1) & ~(size_t)1);
}

__device__ __forceinline__ long vidx(const CqrArgs& a, int i, int j) {
  return a.tall ? (long)i * a.c + j : (long)j * a.nlong + i;
}

__device__ __forceinline__ double win(const CqrArgs& a, int i, int j) {
  if (a.W2) return j < a.c1 ? a.W[(long)i * a.c1 + j] : a.W2[(long)i * (a.c - a.c1) + (j - a.c1)];
  return a.W[vidx(a, i, j)];
}

// 1/v for a pivot v of the scaled Gram (tau < v < 4, so v's exponent is a
// binary32 one): a binary32 seed from v's bits (truncated, integer
// operations -- a binary64 <-> binary32 conversion holds the FP64 pipe like a
// multiply), its reciprocal widened the same way, one binary64 Newton step:
// about 2^-46.
__device__ __forceinline__ double pivot_rcp(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const float f = __uint_as_float(((hi - ((1023u - 127u) << 20)) << 3) | (lo >> 29));
  const unsigned yb = __float_as_uint(__frcp_rn(f));
  const double y = __hiloint2double((int)((yb >> 3) + ((1023u - 127u) << 20)), (int)(yb << 29));
  return y * fma(-v, y, 2.0);
}

// v > tau for positive tau by the bit patterns (non-negative doubles order
// like their bits, negative ones are negative integers): no FP64 compare
__device__ __forceinline__ bool pivot_kept(double v, long long tau_bits) {
  return __double_as_longlong(v) > tau_bits;
}

__device__ __forceinline__ void stamp(const CqrArgs& a, int k) {
  if (a.tstamp && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long ts;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ts));
    a.tstamp[k] = ts;
  }
}

__global__ void __launch_bounds__(kThr) cqr_cluster_kernel(CqrArgs a) {
  pdl_wait();  // W comes from the previous kernel of the stream
  pdl_trigger();
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks();
  const int b = (int)cl.block_rank();
  extern __shared__ double sm[];
  const int c = a.c, T = tri_count(c);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int i0 = b * a.per, cnt = max(0, min(a.per, a.nlong - i0));
  const int rpc = (c + CL - 1) / CL;
  const int nrow = b < c ? (c - 1 - b) / CL + 1 : 0;  // own rows b, b + CL, ... of Lacc
  double* V = sm;
  double* V2 = V + a.per * c;
  double* P = V2 + a.per * c;  // 2 x T partial Grams
  double* A = P + 2 * T;       // c x c lower: scaled Gram, L D L^T work, then L D^{1/2}
  double* B = A + c * c;       // c x c lower: unit L^{-1}
  double* Lr = B + c * c;      // rpc x c: own rows of Lacc
  double* Lr2 = Lr + rpc * c;
  double* rv = Lr2 + rpc * c;  // 1/d_j (0 for a zeroed pivot), scaled units
  double* dv = rv + c;         // d_j
  double* sdn = dv + c;        // sqrt(d_j)
  double* isdn = sdn + c;      // 1/sqrt(d_j)
  double* PX = isdn + c;       // c <= kPolyMaxC: 3 x (c x c) for the series of the last pass
  int* tri = reinterpret_cast<int*>(PX + (c <= kPolyMaxC ? 3 * c * c : 0));  // (row << 8) | col, lower triangle
  __shared__ unsigned ired[2][kThr / 32];
  __shared__ double shift, sc, isc;
  __shared__ long long taub;  // bits of the pivot threshold (a positive double)
  __shared__ int bad, last, nterm;
  stamp(a, 0);
  for (int e = t; e < cnt * c; e += kThr) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    V[r * c + j] = win(a, i0 + r, j);
  }
  for (int ia = t; ia < c; ia += kThr)
    for (int ib = 0; ib <= ia; ++ib) tri[ia * (ia + 1) / 2 + ib] = (ia << 8) | ib;
  if (t == 0) bad = 0;
  __syncthreads();
  stamp(a, 1);
  const int S = a.slices;  // power of two <= 32: threads per Gram entry
  int pass = 0;
  for (;; ++pass) {
    double* Pw = P + (pass & 1) * T;
    // (1) partial Gram of own vectors: S threads per entry (rows r = s mod
    // S), combined by a fixed xor tree
    // (a binary64 warp instruction holds the FP64 pipe for ~64 cycles whatever
    // its active lanes: warps without terms issue none)
    for (int base = 0; base < T * S; base += kThr) {
      if (base + warp * 32 >= T * S) continue;  // warp-uniform
      const int u = base + t, e = u / S, s = u % S;
      double acc = 0.0;
      if (e < T) {
        const int rc = tri[e], k = rc >> 8, j = rc & 255;
        for (int r = s; r < cnt; r += S) acc = fma(V[r * c + j], V[r * c + k], acc);
      }
      for (int o = S >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (e < T && s == 0) Pw[e] = acc;
    }
    cl.sync();
    stamp(a, 2 + 6 * pass + 0);
    // (2) the Gram: CL lanes per entry read the CTAs' partials, xor tree; the
    // largest diagonal and the distance from the identity as integer maxima of
    // bit patterns (exactly zero columns, left by zeroed pivots, do not count)
    {
      unsigned mxh = 0, devb = 0;
      for (int base = 0; base < T * CL; base += kThr * kSumBatch) {
        double gq[kSumBatch];
#pragma unroll
        for (int q = 0; q < kSumBatch; ++q) {
          const int u = base + q * kThr + t, e = u / CL, r = u % CL;
          gq[q] = e < T ? cl.map_shared_rank(Pw, r)[e] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kSumBatch; ++q) {
        if (base + q * kThr + warp * 32 >= T * CL) continue;  // warp-uniform: no terms
        const int u = base + q * kThr + t, e = u / CL, r = u % CL;
        double g = gq[q];
        for (int o = CL >> 1; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (e < T && r == 0) {
          const int rc = tri[e], k = rc >> 8, j = rc & 255;
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
        }
      }
      mxh = __reduce_max_sync(0xffffffffu, mxh);
      devb = __reduce_max_sync(0xffffffffu, devb);
      if (lane == 0) ired[0][warp] = mxh, ired[1][warp] = devb;
    }
    __syncthreads();
    if (t == 0) {
      unsigned M = 0, D = 0;
      for (int w = 0; w < kThr / 32; ++w) M = max(M, ired[0][w]), D = max(D, ired[1][w]);
      const bool fin = (__uint_as_float(D) * c <= kOrthDev) || c == 1 || pass == kCqrMaxPass - 1;
      const double mx = __hiloint2double((int)M, 0);
      const double sh = (pass < kCqrShiftedPasses && !fin) ? a.shift_rel * c * mx : 0.0;
      shift = sh;
      last = fin;
      // terms of the series: the first K with dev^(K+1) <= 2^-56
      int K = -1;
      const float dev = __uint_as_float(D) * c;
      if (fin && c <= kPolyMaxC && dev <= kPolyDev) {
        double pw = dev;
        K = 1;
        while (pw * dev > 0x1p-56 && K < kPolyMaxTerms) {
          pw *= dev;
          ++K;
        }
      }
      nterm = K;
      const int ex = (int)((M >> 20) & 0x7FF);
      const int k2 = (ex > 0 && ex < 0x7FF) ? ((ex - 1023) >> 1) : 0;
      sc = __longlong_as_double((long long)(1023 + k2) << 52);
      isc = __longlong_as_double((long long)(1023 - k2) << 52);
      const double s2 = __longlong_as_double((long long)(1023 - 2 * k2) << 52);
      taub = __double_as_longlong(64.0 * kUnitRoundoff * (mx + sh) * s2);
    }
    __syncthreads();
    // every read of this pass's partials is done: on the last pass the
    // barrier that keeps shared memory alive is entered now and left at exit
    if (last) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    if (nterm >= 0) {
      // (3') last pass with G = I + E, |E| <= kPolyDev: T = G^(-1/2) and
      // T^-1 = G^(1/2) from their binomial series in E (symmetric, full), so
      // Q = V T is orthonormal to working precision and W = Q (T^-1 Lacc^T)
      double* E = A;
      double* Pk = B;
      double* Pn = PX;
      double* Tm = PX + c * c;
      double* Ti = PX + 2 * c * c;
      for (int e = t; e < T; e += kThr) {
        const int rc = tri[e], k = rc >> 8, j = rc & 255;
        const double g = A[k * c + j];
        // an exactly zero column (a zeroed pivot, or zero input) stays zero and
        // gets a zero row and column in T and T^-1, so that R keeps its rank
        const bool live = (__double_as_longlong(g) << 1) != 0;
        const double ev = (k == j) ? (live ? g - 1.0 : 0.0) : g;
        const double id = (k == j && live) ? 1.0 : 0.0;
        E[k * c + j] = ev;
        E[j * c + k] = ev;
        Pk[k * c + j] = ev;
        Pk[j * c + k] = ev;
        Tm[k * c + j] = Tm[j * c + k] = fma(-0.5, ev, id);
        Ti[k * c + j] = Ti[j * c + k] = fma(0.5, ev, id);
      }
      __syncthreads();
      for (int p = 2; p <= nterm; ++p) {
        const double ca = kSeriesA[p], cb = kSeriesB[p];
        for (int e = t; e < c * c; e += kThr) {
          const int i = e / c, j = e % c;
          double s = 0.0;
          for (int l = 0; l < c; ++l) s = fma(Pk[i * c + l], E[l * c + j], s);
          Pn[e] = s;
          Tm[e] = fma(ca, s, Tm[e]);
          Ti[e] = fma(cb, s, Ti[e]);
        }
        __syncthreads();
        double* sw = Pk;
        Pk = Pn;
        Pn = sw;
      }
      stamp(a, 2 + 6 * pass + 1);
      stamp(a, 2 + 6 * pass + 2);
      for (int e = t; e < cnt * c; e += kThr) {
        const int r = e / c, i = e % c;
        const double* vr = V + r * c;
        double s = 0.0;
        for (int l = 0; l < c; ++l) s = fma(Tm[i * c + l], vr[l], s);
        V2[r * c + i] = s;
      }
      for (int e = t; e < nrow * c; e += kThr) {
        const int q = e / c, k = e % c, i = b + q * CL;
        double s = 0.0;
        if (pass == 0) {
          s = Ti[i * c + k];
        } else {
          for (int l = 0; l < c; ++l) s = fma(Lr[q * c + l], Ti[l * c + k], s);
        }
        Lr2[q * c + k] = s;
      }
      __syncthreads();
      stamp(a, 2 + 6 * pass + 3);
      stamp(a, 2 + 6 * pass + 4);
    } else {
      {
        const double s2 = isc * isc, sh = shift;
        for (int e = t; e < T; e += kThr) {
          const int rc = tri[e], k = rc >> 8, j = rc & 255;
          const double v = (A[k * c + j] + (k == j ? sh : 0.0)) * s2;
          A[k * c + j] = v;
          if (e == 0) {
            const bool z = !pivot_kept(v, taub);
            rv[0] = z ? 0.0 : pivot_rcp(v);
            dv[0] = z ? 0.0 : v;
            if (z) bad = 1;
          }
        }
      }
      __syncthreads();
      stamp(a, 2 + 6 * pass + 1);
      // (3) L D L^T: step j takes column j out of the trailing block and out of
      // the rows of L^{-1} below j.  Lane 0 of the last warp updates the next
      // pivot and takes its reciprocal; warps 0..6 do the rest.
      for (int j = 0; j + 1 < c; ++j) {
        const int rem = c - 1 - j, nt = rem * (rem + 1) / 2, ni = rem * (j + 1);
        const double r = rv[j];
        if (t == kUpd) {
          const int i = j + 1;
          const double l = A[i * c + j];
          const double v = fma(-(l * r), l, A[i * c + i]);
          A[i * c + i] = v;
          const bool z = !pivot_kept(v, taub);
          rv[i] = z ? 0.0 : pivot_rcp(v);
          dv[i] = z ? 0.0 : v;
          if (z) bad = 1;
        } else if (t < kUpd) {
          // e = 0 is the next pivot (the chain's); the others start at 1
          for (int e = t + 1; e < nt + ni; e += kUpd) {
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
      for (int i = t; i < c; i += kThr) {
        const double d = dv[i];
        const double is = d > 0.0 ? drsqrt(d) : 0.0;
        isdn[i] = is;
        sdn[i] = d * is;
      }
      __syncthreads();
      stamp(a, 2 + 6 * pass + 2);
      // (4) v <- D^{-1/2} L^{-1} v for own vectors; rows i and c-1-i together
      {
        const int h = (c + 1) / 2;
        const double sci = isc;
        for (int e = t; e < cnt * h; e += kThr) {
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
      for (int e = t; e < T; e += kThr) {
        const int rc = tri[e], i = rc >> 8, j = rc & 255;
        A[i * c + j] = (i == j) ? sdn[j] * sc : A[i * c + j] * isdn[j] * sc;
      }
      __syncthreads();
      stamp(a, 2 + 6 * pass + 3);
      // (5) own rows of Lacc <- Lacc L D^{1/2}
      for (int e = t; e < nrow * c; e += kThr) {
        const int q = e / c, k = e % c, i = b + q * CL;
        double s = 0.0;
        if (pass == 0) {
          s = (k <= i) ? A[i * c + k] : 0.0;
        } else if (k <= i) {
          for (int l = k; l <= i; ++l) s = fma(Lr[q * c + l], A[l * c + k], s);
        }
        Lr2[q * c + k] = s;
      }
      __syncthreads();
      stamp(a, 2 + 6 * pass + 4);
    }
    double* tmp = Lr;
    Lr = Lr2;
    Lr2 = tmp;
    tmp = V;
    V = V2;
    V2 = tmp;
    if (last) break;  // the same decision in every CTA: same Gram, same code
  }
  for (int e = t; e < cnt * c; e += kThr) {
    const int r = a.tall ? e / c : e % cnt, j = a.tall ? e % c : e / cnt;
    a.Q[vidx(a, i0 + r, j)] = V[r * c + j];
  }
  for (int e = t; e < nrow * c; e += kThr) {
    const int q = e / c, k = e % c, i = b + q * CL;
    if (a.tall) a.R[k * c + i] = Lr[q * c + k];
    else a.R[i * c + k] = Lr[q * c + k];
  }
  if (b == 0 && t == 0 && a.status) *a.status = bad;
  // no CTA leaves while another may still read its partial Grams
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  stamp(a, kStamps - 1);
}

}  // namespace

// Cluster size, vectors per CTA and shared memory for a block of nlong
// vectors of length c; false when the block is too large for one cluster
// (or no cluster of that shape can be resident), in which case the caller
// takes the full-grid kernel.
bool cqr_cluster_plan(int nlong, int c, int* cl_out, int* per_out, size_t* smem_out) {
  if (c < 1 || c > kSmallMax || nlong < c || c > 255) return false;
  const long work = (long)nlong * tri_count(c);
  if (work > kMaxWork) return false;
  int cl = 1;
  while (cl < kMaxCl && (work + cl - 1) / cl > kWorkPerCta && cl < nlong) cl *= 2;
  int per = (nlong + cl - 1) / cl;
  size_t smem = cl_smem_bytes(per, c, cl);
  while (smem > kClMaxSmem && cl < kMaxCl) {
    cl *= 2;
    per = (nlong + cl - 1) / cl;
    smem = cl_smem_bytes(per, c, cl);
  }
  if (smem > kClMaxSmem) return false;
  // one-time function attributes, then whether such a cluster can be resident
  // at all (cached per cluster size and 8 KB of shared memory)
  static std::once_flag attr_once;
  static bool attr_ok = false;
  std::call_once(attr_once, [] {
    attr_ok = cudaFuncSetAttribute(cqr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClMaxSmem) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(cqr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
    if (!attr_ok) cudaGetLastError();
  });
  if (!attr_ok) return false;
  static std::atomic<signed char> fits[5][(kClMaxSmem >> 13) + 1];  // 0 unknown, 1 yes, -1 no
  int lg = 0;
  while ((1 << lg) < cl) ++lg;
  const size_t bucket = (smem + 8191) >> 13;
  signed char f = fits[lg][bucket].load();
  if (f == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kThr);
    cfg.dynamicSmemBytes = bucket << 13;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, cqr_cluster_kernel, &cfg) == cudaSuccess && n > 0;
    if (!ok) cudaGetLastError();
    f = ok ? 1 : -1;
    fits[lg][bucket].store(f);
  }
  if (f < 0) return false;
  *cl_out = cl;
  *per_out = per;
  *smem_out = smem;
  return true;
}

t2s2_status cqr_cluster(const double* W, double* Q, double* R, int nlong, int c, bool tall, double shift_rel,
                        int* status, int cl, int per, size_t smem, cudaStream_t st, const double* W2, int c1) {
  CqrArgs a;
  a.W = W;
  a.W2 = (tall && W2) ? W2 : nullptr;
  a.c1 = c1;
  a.Q = Q;
  a.R = R;
  a.status = status;
  a.nlong = nlong;
  a.c = c;
  a.per = per;
  a.tall = tall ? 1 : 0;
  int slices = 1;
  while (slices < 32 && (long)tri_count(c) * slices * 2 <= kThr) slices *= 2;
  a.slices = slices;
  a.shift_rel = shift_rel;
  a.tstamp = nullptr;
  // T2S2_QR_TIMING=N: the N-th cluster factorisation of the process prints
  // the phase times of its CTA 0 (diagnostics; synchronises that one call)
  static const int stamp_at = [] {
    const char* e = std::getenv("T2S2_QR_TIMING");
    return (e && e[0] >= '0' && e[0] <= '9') ? std::atoi(e) : -1;
  }();
  static std::atomic<int> calls{0};
  static unsigned long long* stamp_buf = nullptr;
  const bool stamp_this = stamp_at >= 0 && calls.fetch_add(1) == stamp_at;
  if (stamp_this) {
    if (!stamp_buf) T2S2_CUDA_TRY(cudaMalloc(&stamp_buf, sizeof(unsigned long long) * kStamps));
    T2S2_CUDA_TRY(cudaMemsetAsync(stamp_buf, 0, sizeof(unsigned long long) * kStamps, st));
    a.tstamp = stamp_buf;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  // work of two passes (the common case): Gram and triangular product
  // 2 n c^2 each, the L D L^T with its inverse 2 c^3 / 3
  const double fl = 2.0 * (4.0 * nlong * (double)c * c) + 2.0 * (2.0 * (double)c * c * c / 3.0);
  {
    TraceScope ts(kTrCholQR, st, fl, 16.0 * nlong * c);
    T2S2_CUDA_TRY(cudaLaunchKernelEx(&cfg, cqr_cluster_kernel, a));
  }
  if (stamp_this) {
    unsigned long long h[kStamps];
    T2S2_CUDA_TRY(cudaMemcpyAsync(h, stamp_buf, sizeof(h), cudaMemcpyDeviceToHost, st));
    T2S2_CUDA_TRY(cudaStreamSynchronize(st));
    fprintf(stderr, "[t2s2] cluster cholqr phase times (ns) nlong=%d c=%d cluster=%d: load %lld", nlong, c, cl,
            (long long)(h[1] - h[0]));
    unsigned long long prev = h[1];
    for (int p = 0; p < kCqrMaxPass && h[2 + 6 * p]; ++p) {
      fprintf(stderr, " | pass %d:", p);
      for (int k = 0; k < 5; ++k) {
        fprintf(stderr, " %lld", (long long)(h[2 + 6 * p + k] - prev));
        prev = h[2 + 6 * p + k];
      }
    }
    fprintf(stderr, " | store %lld total %lld\n", (long long)(h[kStamps - 1] - prev),
            (long long)(h[kStamps - 1] - h[0]));
  }
  return T2S2_OK;
}

}  // namespace t2s2
