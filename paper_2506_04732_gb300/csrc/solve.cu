// Alternating TT solver (AMEn) and the Crank-Nicolson / backward-Euler steps.
//
// The paper solves its collocation systems with AMEn (Results,
// "Superconsistent Stabilization", Fig. 6), sweeping over the cores and solving
// a local problem at each.  This implementation works on the equivalent
// Kronecker-sum system: with M = Rt_1 x ... x Rt_d,
//     M^{-1} (c_mass M + c_op A) = sum_k I x ... x B'_k x ... x I,
//     B'_k = c_op Rt_k^{-1} Lt_k + (c_mass / d) I,      rhs f = M^{-1} b,
// so that, with orthonormal left/right frames, each local operator is the
// three-term Kronecker sum P_L (+) B'_k (+) P_R (local.cu).  Per core and sweep:
// local right-hand side, local GMRES solve, SVD truncation at tol/sqrt(d),
// enrichment of the new core with the residual projected onto a rank-4 TT z
// (Dolgov & Savostyanov's AMEn, cited by the paper), orthogonalisation, and
// the interface updates -- all as GEMM chains on the device.  After each sweep
// the true residual ||b - (c_mass M + c_op A) x|| / ||b|| of the ORIGINAL
// collocation system is evaluated in FP64 and decides convergence.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <random>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "local.h"
#include "trace.h"

void t2s2_op_s::free_solver_buffers() {}

namespace t2s2 {

namespace {

Gemm<double> gdesc(int M, int N, int K, bool tA, bool tB, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc, int batch = 1, long sA = 0,
                   long sB = 0, long sC = 0) {
  Gemm<double> g;
  g.M = M; g.N = N; g.K = K; g.tA = tA; g.tB = tB; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.sA = sA; g.B = B; g.ldb = ldb; g.sB = sB;
  g.C = C; g.ldc = ldc; g.sC = sC; g.batch = batch;
  return g;
}
// Mode products of a core X (ra x m x rb) and the interface contractions, in
// the context's contraction arithmetic: descriptors (for grouped launches)
// and single calls.
// Y[c,i,b] = sum_a P[c,a] X[a,i,b]
Gemm<double> g_mode1(const double* P, int rn, int ro, const double* X, int m, int rb, double* Y,
                     double alpha = 1.0, double beta = 0.0) {
  return gdesc(rn, m * rb, ro, false, false, alpha, P, ro, X, (long)m * rb, beta, Y, (long)m * rb);
}
// Y[a,i,b] = sum_j B[i,j] X[a,j,b]
Gemm<double> g_mode2(const double* B, int m, const double* X, int ra, int rb, double* Y, double alpha = 1.0,
                     double beta = 0.0) {
  return gdesc(m, rb, m, false, false, alpha, B, m, X, rb, beta, Y, rb, ra, 0, (long)m * rb, (long)m * rb);
}
// Y[a,i,c] = sum_b X[a,i,b] Q[c,b]
Gemm<double> g_mode3(const double* X, int ra, int m, int ro, const double* Q, int rn, double* Y,
                     double alpha = 1.0, double beta = 0.0) {
  return gdesc(ra * m, rn, ro, false, true, alpha, X, ro, Q, ro, beta, Y, rn);
}
// out[b][c] = sum_{a,i} U[a,i,b] T[a,i,c]
Gemm<double> g_cleft(const double* U, int ra, int m, int rb, const double* T, int rc, double* out) {
  return gdesc(rb, rc, ra * m, true, false, 1.0, U, rb, T, rc, 0.0, out, rc);
}
// out[a][c] = sum_{i,b} U[a,i,b] T[c,i,b]
Gemm<double> g_cright(const double* U, int ra, int m, int rb, const double* T, int rc, double* out) {
  return gdesc(ra, rc, m * rb, false, true, 1.0, U, (long)m * rb, T, (long)m * rb, 0.0, out, rc);
}
t2s2_status mode1(Ctx& cx, const double* P, int rn, int ro, const double* X, int m, int rb, double* Y,
                  double alpha = 1.0, double beta = 0.0) {
  return contract_gemm(cx, g_mode1(P, rn, ro, X, m, rb, Y, alpha, beta));
}
t2s2_status mode3(Ctx& cx, const double* X, int ra, int m, int ro, const double* Q, int rn, double* Y,
                  double alpha = 1.0, double beta = 0.0) {
  return contract_gemm(cx, g_mode3(X, ra, m, ro, Q, rn, Y, alpha, beta));
}
template <int N>
t2s2_status group(Ctx& cx, const Gemm<double> (&gs)[N]) {
  return contract_group(cx, gs, N);
}
t2s2_status d2d(Ctx& cx, double* dst, const double* src, size_t n) {
  if (n == 0) return T2S2_OK;
  T2S2_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, cx.st));
  return T2S2_OK;
}
t2s2_status set_scalars(Ctx& cx, double* p0, double v0, double* p1, double v1, double* p2, double v2, double* p3,
                        double v3, double* p4, double v4);

// The next core of the sweep, (Q^T U S V^T) x_1 X1, in one CTA when X1 fits
// in shared memory: C = Q^T U (one warp per entry, lanes over the rows, fixed
// shuffle tree), CS = C S V^T, then X1 <- CS x_1 X1 in place (X1 is staged
// in shared memory first).
constexpr size_t kNextCoreSmem = 40 * 1024;

// The enrichment and z-update residuals of one core, slice by slice.  With
// Xt = U S V^T the local solution (ra x m x rb) and BX = B' x_2 Xt, every
// remaining product of
//   res  = (FL F) x_3 ZFR - (BX + PL x_1 Xt) x_3 ZIR - Xt x_3 ZBR,
//   zres = (ZFL F) x_3 ZFR - (ZBL x_1 Xt + ZIL x_1 BX) x_3 ZIR - (ZIL x_1 Xt) x_3 ZBR
// acts on one slice i of the cores, so CTA i computes slice i of res and zres
// in shared memory, in binary64 with sums in a fixed order: one launch instead
// of four grouped ones.  When the whole of Xt fits shared memory (the first
// sweep, rb = 1), every CTA also forms its slice of BX from row i of B';
// otherwise BX comes from a product launched before.
struct EnrichArgs {
  int ra, rb, fa, fb, za, zb, m;
  const double *Xt, *BX, *T1, *F, *Bp;            // cores (a, i, b) row-major; B' m x m
  const double *PL, *ZBL, *ZIL, *ZFL;             // left interfaces: (rows) x (ra | fa)
  const double *ZFR, *ZIR, *ZBR;                  // right interfaces: zb x (fb | rb)
  double *res, *zres;                             // ra x m x zb, za x m x zb
  int bx_here;                                    // 1: BX from Xt and B' in this kernel
};

constexpr int kEnrichThreads = 256;
constexpr size_t kEnrichMaxSmem = 96 * 1024;

__host__ __device__ inline size_t enrich_smem_doubles(const EnrichArgs& a) {
  const size_t ra = a.ra, rb = a.rb, fa = a.fa, fb = a.fb, za = a.za, zb = a.zb;
  size_t n = 3 * ra * rb + ra * fb + fa * fb + ra * ra + 2 * za * ra + za * fa + zb * fb + 2 * zb * rb +
             2 * za * rb + za * fb;
  if (a.bx_here) n += ra * (size_t)a.m * rb + a.m;
  return n;
}

__global__ void __launch_bounds__(kEnrichThreads) k_enrich(EnrichArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double es[];
  const int i = blockIdx.x, t = threadIdx.x, m = a.m;
  const int ra = a.ra, rb = a.rb, fa = a.fa, fb = a.fb, za = a.za, zb = a.zb;
  double* xs = es;               // ra x rb: Xt[:, i, :]
  double* bs = xs + ra * rb;     // ra x rb: BX[:, i, :]
  double* y1 = bs + ra * rb;     // ra x rb
  double* ts = y1 + ra * rb;     // ra x fb: T1[:, i, :]
  double* fs = ts + ra * fb;     // fa x fb: F[:, i, :]
  double* pl = fs + fa * fb;     // ra x ra
  double* zbl = pl + ra * ra;    // za x ra
  double* zil = zbl + za * ra;   // za x ra
  double* zfl = zil + za * ra;   // za x fa
  double* zfr = zfl + za * fa;   // zb x fb
  double* zir = zfr + zb * fb;   // zb x rb
  double* zbr = zir + zb * rb;   // zb x rb
  double* t2 = zbr + zb * rb;    // za x rb
  double* t2b = t2 + za * rb;    // za x rb
  double* tz = t2b + za * rb;    // za x fb
  double* xall = tz + za * fb;   // bx_here: ra x m x rb, then row i of B'
  double* brow = xall + (a.bx_here ? ra * m * rb : 0);
  for (int e = t; e < ra * rb; e += kEnrichThreads) {
    const int p = e / rb, q = e % rb;
    xs[e] = a.Xt[((long)p * m + i) * rb + q];
    if (!a.bx_here) bs[e] = a.BX[((long)p * m + i) * rb + q];
  }
  for (int e = t; e < ra * fb; e += kEnrichThreads) ts[e] = a.T1[((long)(e / fb) * m + i) * fb + e % fb];
  for (int e = t; e < fa * fb; e += kEnrichThreads) fs[e] = a.F[((long)(e / fb) * m + i) * fb + e % fb];
  for (int e = t; e < ra * ra; e += kEnrichThreads) pl[e] = a.PL[e];
  for (int e = t; e < za * ra; e += kEnrichThreads) {
    zbl[e] = a.ZBL[e];
    zil[e] = a.ZIL[e];
  }
  for (int e = t; e < za * fa; e += kEnrichThreads) zfl[e] = a.ZFL[e];
  for (int e = t; e < zb * fb; e += kEnrichThreads) zfr[e] = a.ZFR[e];
  for (int e = t; e < zb * rb; e += kEnrichThreads) {
    zir[e] = a.ZIR[e];
    zbr[e] = a.ZBR[e];
  }
  if (a.bx_here) {
    for (int e = t; e < ra * m * rb; e += kEnrichThreads) xall[e] = a.Xt[e];
    for (int j = t; j < m; j += kEnrichThreads) brow[j] = a.Bp[(long)i * m + j];
  }
  __syncthreads();
  if (a.bx_here) {
    // BX[:, i, :] = sum_j B'[i, j] Xt[:, j, :]
    for (int e = t; e < ra * rb; e += kEnrichThreads) {
      const int p = e / rb, q = e % rb;
      double s0 = 0.0, s1 = 0.0;
      int j = 0;
      for (; j + 1 < m; j += 2) {
        s0 = fma(brow[j], xall[((long)p * m + j) * rb + q], s0);
        s1 = fma(brow[j + 1], xall[((long)p * m + j + 1) * rb + q], s1);
      }
      if (j < m) s0 = fma(brow[j], xall[((long)p * m + j) * rb + q], s0);
      bs[e] = s0 + s1;
    }
    __syncthreads();
  }
  // Y1 = BX + PL Xt,  T2 = ZBL Xt + ZIL BX,  T2b = ZIL Xt,  Tz = ZFL F (slice i)
  for (int e = t; e < ra * rb; e += kEnrichThreads) {
    const int p = e / rb, q = e % rb;
    double s = bs[e];
    for (int c = 0; c < ra; ++c) s = fma(pl[p * ra + c], xs[c * rb + q], s);
    y1[e] = s;
  }
  for (int e = t; e < za * rb; e += kEnrichThreads) {
    const int p = e / rb, q = e % rb;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < ra; ++c) {
      s0 = fma(zbl[p * ra + c], xs[c * rb + q], s0);
      s1 = fma(zil[p * ra + c], bs[c * rb + q], s1);
      s2 = fma(zil[p * ra + c], xs[c * rb + q], s2);
    }
    t2[e] = s0 + s1;
    t2b[e] = s2;
  }
  for (int e = t; e < za * fb; e += kEnrichThreads) {
    const int p = e / fb, q = e % fb;
    double s = 0.0;
    for (int c = 0; c < fa; ++c) s = fma(zfl[p * fa + c], fs[c * fb + q], s);
    tz[e] = s;
  }
  __syncthreads();
  // res[:, i, :] = T1 ZFR^T - Y1 ZIR^T - Xt ZBR^T;  zres[:, i, :] = Tz ZFR^T - T2 ZIR^T - T2b ZBR^T
  for (int e = t; e < (ra + za) * zb; e += kEnrichThreads) {
    const int row = e / zb, q = e % zb;
    const bool top = row < ra;
    const int p = top ? row : row - ra;
    const double* u = top ? ts + p * fb : tz + p * fb;
    const double* v = top ? y1 + p * rb : t2 + p * rb;
    const double* w = top ? xs + p * rb : t2b + p * rb;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < fb; ++c) s0 = fma(u[c], zfr[q * fb + c], s0);
    for (int c = 0; c < rb; ++c) {
      s1 = fma(v[c], zir[q * rb + c], s1);
      s2 = fma(w[c], zbr[q * rb + c], s2);
    }
    const double r = s0 - s1 - s2;
    if (top) a.res[((long)p * m + i) * zb + q] = r;
    else a.zres[((long)p * m + i) * zb + q] = r;
  }
}

// The local right-hand side of core k, slice by slice: T1 = FL x_1 F (kept
// for the enrichment) and rhs = T1 x_3 FR, CTA i forming slice i of both in
// shared memory (binary64, fixed-order sums): one launch instead of two.
struct RhsArgs {
  int ra, rb, fa, fb, m;
  const double *FL, *F, *FR;  // ra x fa, fa x m x fb, rb x fb
  double *T1, *rhs;           // ra x m x fb, ra x m x rb
};

__global__ void __launch_bounds__(kEnrichThreads) k_local_rhs(RhsArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double rs[];
  const int i = blockIdx.x, t = threadIdx.x, m = a.m;
  const int ra = a.ra, rb = a.rb, fa = a.fa, fb = a.fb;
  double* fl = rs;             // ra x fa
  double* fs = fl + ra * fa;   // fa x fb
  double* fr = fs + fa * fb;   // rb x fb
  double* t1 = fr + rb * fb;   // ra x fb
  for (int e = t; e < ra * fa; e += kEnrichThreads) fl[e] = a.FL[e];
  for (int e = t; e < fa * fb; e += kEnrichThreads) fs[e] = a.F[((long)(e / fb) * m + i) * fb + e % fb];
  for (int e = t; e < rb * fb; e += kEnrichThreads) fr[e] = a.FR[e];
  __syncthreads();
  for (int e = t; e < ra * fb; e += kEnrichThreads) {
    const int p = e / fb, q = e % fb;
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
    for (; c + 1 < fa; c += 2) {
      s0 = fma(fl[p * fa + c], fs[c * fb + q], s0);
      s1 = fma(fl[p * fa + c + 1], fs[(c + 1) * fb + q], s1);
    }
    if (c < fa) s0 = fma(fl[p * fa + c], fs[c * fb + q], s0);
    const double v = s0 + s1;
    t1[e] = v;
    a.T1[((long)p * m + i) * fb + q] = v;
  }
  __syncthreads();
  for (int e = t; e < ra * rb; e += kEnrichThreads) {
    const int p = e / rb, q = e % rb;
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
    for (; c + 1 < fb; c += 2) {
      s0 = fma(t1[p * fb + c], fr[q * fb + c], s0);
      s1 = fma(t1[p * fb + c + 1], fr[q * fb + c + 1], s1);
    }
    if (c < fb) s0 = fma(t1[p * fb + c], fr[q * fb + c], s0);
    a.rhs[((long)p * m + i) * rb + q] = s0 + s1;
  }
}

// Five interface boundary values (the 1 x 1 interfaces at bond 0 or d) in
// one launch.
struct ScalarSet {
  double* p[5];
  double v[5];
};
__global__ void k_set_scalars(ScalarSet s) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x < 5) *s.p[threadIdx.x] = s.v[threadIdx.x];
}

// B'_k = c_op B_k + shift I for every dimension in one launch.
struct BprimeArgs {
  int d;
  double* out[T2S2_MAX_D];
  const double* B[T2S2_MAX_D];
  const double* I[T2S2_MAX_D];
  int mm[T2S2_MAX_D];  // m_k^2
  double c_op, shift;
};
__global__ void k_bprime(BprimeArgs a) {
  pdl_wait();
  pdl_trigger();
  const int stride = gridDim.x * blockDim.x;
  for (int k = 0; k < a.d; ++k)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.mm[k]; e += stride)
      a.out[k][e] = fma(a.shift, a.I[k][e], a.c_op * a.B[k][e]);
}

t2s2_status set_scalars(Ctx& cx, double* p0, double v0, double* p1, double v1, double* p2, double v2, double* p3,
                        double v3, double* p4, double v4) {
  ScalarSet s;
  s.p[0] = p0, s.p[1] = p1, s.p[2] = p2, s.p[3] = p3, s.p[4] = p4;
  s.v[0] = v0, s.v[1] = v1, s.v[2] = v2, s.v[3] = v3, s.v[4] = v4;
  {
    TraceScope ts_(kTrElem, cx.st, 0.0, 40.0);
    (void)launch_pdl(k_set_scalars, 1, 32, 0, cx.st, s);
  }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

__global__ void k_next_core(const double* Q, const double* U, const double* SV, int rows, int rn, int rk, int rb,
                            double* X1, int mn, int rnn) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double nsm[];
  double* xs = nsm;                     // rb x mn x rnn
  double* C = xs + (size_t)rb * mn * rnn;  // rn x rk
  double* CS = C + rn * rk;             // rn x rb
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int nx = rb * mn * rnn;
  for (int e = t; e < nx; e += blockDim.x) xs[e] = X1[e];
  for (int q = warp; q < rn * rk; q += nw) {
    const int cc = q / rk, a = q % rk;
    double s0 = 0.0, s1 = 0.0;
    int r = lane;
    for (; r + 32 < rows; r += 64) {
      s0 = fma(Q[(long)r * rn + cc], U[(long)r * rk + a], s0);
      s1 = fma(Q[(long)(r + 32) * rn + cc], U[(long)(r + 32) * rk + a], s1);
    }
    if (r < rows) s0 = fma(Q[(long)r * rn + cc], U[(long)r * rk + a], s0);
    double s = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[q] = s;
  }
  __syncthreads();
  for (int e = t; e < rn * rb; e += blockDim.x) {
    const int cc = e / rb, b = e % rb;
    double s = 0.0;
    for (int a = 0; a < rk; ++a) s = fma(C[cc * rk + a], SV[a * rb + b], s);
    CS[e] = s;
  }
  __syncthreads();
  const int inner = mn * rnn;
  for (int e = t; e < rn * inner; e += blockDim.x) {
    const int cc = e / inner, ie = e % inner;
    double s = 0.0;
    for (int b = 0; b < rb; ++b) s = fma(CS[cc * rb + b], xs[b * inner + ie], s);
    X1[e] = s;
  }
}

// SVD of one column x (n entries): u = x / |x| (0 for x = 0), s v^T = |x|,
// and the truncated product u s v^T = x.  One CTA, fixed-order sum.
__global__ void k_col_split(const double* x, int n, double* u, double* sv, double* xt) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[32];
  double p = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) p = fma(x[i], x[i], p);
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[0] = sqrt(t);
    sv[0] = red[0];
  }
  __syncthreads();
  const double nrm = red[0];
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    u[i] = x[i] * inv;
    xt[i] = x[i];
  }
}

// Optional per-phase timing of the solver (T2S2_PHASES=1): CUDA events at the
// phase boundaries on the solver's stream, summed and printed per solve.
struct PhaseTimer {
  static constexpr int kPhases = 11;
  bool on = false;
  cudaStream_t st = 0;
  int cur = -1;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  void start(cudaStream_t s) {
    const char* e = std::getenv("T2S2_PHASES");
    on = e && e[0] == '1';
    st = s;
  }
  void phase(int p) {
    if (!on) return;
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    cudaEventRecord(ev, st);
    marks.push_back({p, ev});
  }
  void report() {
    if (!on || marks.empty()) return;
    static const char* names[kPhases] = {"init", "right_ifaces", "local_rhs", "local_solve", "truncate",
                                         "enrich", "z_update", "new_core", "left_ifaces", "residual", "orth_x"};
    double tot[kPhases] = {0};
    cudaEventSynchronize(marks.back().second);
    for (size_t i = 0; i + 1 < marks.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, marks[i].second, marks[i + 1].second);
      tot[marks[i].first] += ms;
    }
    fprintf(stderr, "[t2s2] phases (ms):");
    for (int i = 0; i < kPhases; ++i) fprintf(stderr, " %s %.2f", names[i], tot[i]);
    fprintf(stderr, "\n");
    for (auto& m : marks) cudaEventDestroy(m.second);
    marks.clear();
  }
};

// Rank of the enrichment (residual) directions added per core and sweep.
// The paper names AMEn without parameters.  On the d = 6, n = 32 problem a
// kick of 4 needs 7 sweeps (ranks grow 1, 5, 9, 13, ...), a kick of 8 one
// sweep: the solution's rank at 1e-8 is about 9-13, and a first sweep whose
// bases span it converges at once.  T2S2_KICK overrides it (1 .. 16).
// Enrichment rank of the time steps (their solves start from the previous
// step): on the d = 7, n = 64 Crank-Nicolson step a kick of 4 keeps ranks at
// 7 and takes 10.3 ms, a kick of 8 raises them to 11 and takes 15 ms.
constexpr int kStepKick = 4;

// Sweeps without a halving of the residual, at the rank cap, after which a
// solve stops early (T2S2_STALL overrides it; 0 turns the stop off).
int stall_sweeps() {
  static const int v = [] {
    const char* e = std::getenv("T2S2_STALL");
    const int k = e ? std::atoi(e) : 8;
    return k < 0 ? 8 : k;
  }();
  return v;
}

int amen_kick() {
  static const int k = [] {
    const char* e = std::getenv("T2S2_KICK");
    const int v = e ? std::atoi(e) : T2S2_RANK_KICK;
    return (v >= 1 && v <= 16) ? v : T2S2_RANK_KICK;
  }();
  return k;
}

struct Amen {
  PhaseTimer* pt = nullptr;
  void ph(int p) {
    if (pt) pt->phase(p);
  }
  t2s2_op op = nullptr;
  Ctx* cx = nullptr;
  int d = 0, kick = amen_kick(), rcap = 0, rmax = 0, mmax = 0, R = 0;
  double ltol = 0.0;
  DevTT x, f, z;
  double* Bp[T2S2_MAX_D] = {nullptr};
  double *PL[T2S2_MAX_D + 1], *FL[T2S2_MAX_D + 1], *ZIL[T2S2_MAX_D + 1], *ZBL[T2S2_MAX_D + 1],
      *ZFL[T2S2_MAX_D + 1];
  double *PR[T2S2_MAX_D + 1], *FR[T2S2_MAX_D + 1], *ZIR[T2S2_MAX_D + 1], *ZBR[T2S2_MAX_D + 1],
      *ZFR[T2S2_MAX_D + 1];
  double* tmp[12] = {nullptr};
  size_t tmp_elems = 0;
  double* gm_work = nullptr;
  double* gm_part = nullptr;
  int* gm_iters = nullptr;
  double* gm_res = nullptr;
  double* svals = nullptr;
  double* eig_buf = nullptr;  // complex binary32 eigen data of both interfaces
  double* ybuf = nullptr;     // complex binary32 intermediate of the exact preconditioner
  int* sylv_status = nullptr; // status word of the rb = 1 local solver
  int* eig_status = nullptr;
  bool use_fls = true;
  float* fbuf = nullptr;     // FP32 rhs / x / GMRES basis for the mixed-precision local solves
  bool fp32_local = false;
  long long local_iters = 0;
  // GMRES counts of local solves that no synchronisation followed, copied
  // without a wait into pinned slots and read at the next collect_iters()
  static constexpr int kIterSlot = kSmallMax + 16;
  static constexpr int kMaxPending = 2 * T2S2_MAX_D;
  int npending = 0;
  int pend_shape[kMaxPending][3];
  t2s2_status defer_iters(int ra, int m, int rb) {
    if (npending == kMaxPending) T2S2_TRY(collect_iters());
    T2S2_CUDA_TRY(cudaMemcpyAsync(cx->hbuf + kIterSlot + npending, gm_iters, sizeof(int), cudaMemcpyDeviceToHost,
                                  cx->st));
    pend_shape[npending][0] = ra, pend_shape[npending][1] = m, pend_shape[npending][2] = rb;
    ++npending;
    return T2S2_OK;
  }
  // the operator's side stream (created on first use; false if that fails)
  bool side_ready() {
    if (op->side && op->ev_fork && op->ev_join) return true;
    if (!op->side && cudaStreamCreateWithFlags(&op->side, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      op->side = nullptr;
      return false;
    }
    if (!op->ev_fork && cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (!op->ev_join && cudaEventCreateWithFlags(&op->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }
  t2s2_status collect_iters() {
    if (npending == 0) return T2S2_OK;
    T2S2_CUDA_TRY(cudaStreamSynchronize(cx->st));
    for (int j = 0; j < npending; ++j) {
      int it;
      std::memcpy(&it, cx->hbuf + kIterSlot + j, sizeof(int));
      local_iters += it;
      trace_add_work(kTrLocal, local_flops(pend_shape[j][0], pend_shape[j][1], pend_shape[j][2], it, gm_restart),
                     0.0);
    }
    npending = 0;
    return T2S2_OK;
  }
  double c_op = 1.0, c_mass = 0.0;
  int gm_restart = 40, gm_maxit = 600;
  bool tstamp_req = false, tstamp_done = false;
  // first sweep of a solve: a rank-1-right local solve runs the Sylvester
  // solver alone, without the general solver queued behind it (see local_solve)
  bool sylv_no_fallback = false;
  int tstamp_target = 0, local_count = 0;
  unsigned long long* tstamp_dev = nullptr;

  static size_t bytes_needed(int d, const int* m, int rcap, int rfmax, int kick, int mr) {
    int mm = 0;
    for (int k = 0; k < d; ++k) mm = std::max(mm, m[k]);
    size_t R = std::max(std::max(rcap, rfmax), kick);
    size_t core = R * mm * R;
    size_t s = 0;
    s += 3 * (size_t)d * core;                  // x, f, z
    s += 10 * (size_t)(d + 1) * R * R;          // interfaces
    s += 12 * core;                             // temporaries
    s += (size_t)(2 * mr + 2) * rcap * mm * rcap;  // flexible GMRES bases
    s += (size_t)rcap * mm * rcap + 2 * (R + 2 * R * R) + 8;  // exact preconditioner buffers
    s += kLocalPartElems + 64;
    s += (size_t)d * mm * mm;                   // B'
    // residual evaluation: apply output, sum, orthogonalisation temporaries
    size_t rr = (size_t)rfmax + 2 * rcap;
    s += 4 * (size_t)d * rr * mm * rr + 16 * rr * rr;
    // SVD / QR temporaries inside orth / qr_tall
    s += 8 * core + 16 * (size_t)kSmallMax * kSmallMax;
    return s * sizeof(double) + ((size_t)16 << 20);
  }

  t2s2_status init(t2s2_op o, Ctx& c, const DevTT& b, const DevTT& x0, double cm, double co, double tol,
                   int rmax_) {
    op = o;
    cx = &c;
    d = op->d;
    c_mass = cm;
    c_op = co;
    rmax = rmax_;
    kick = c.kick > 0 ? c.kick : amen_kick();
    rcap = rmax + kick;
    if (rcap > kSmallMax) return T2S2_EINVAL;
    ltol = tol / std::sqrt((double)d);
    int rfmax = 1;
    for (int k = 0; k <= d; ++k) rfmax = std::max(rfmax, b.r[k]);
    if (rfmax > kSmallMax) return T2S2_EINVAL;
    for (int k = 0; k < d; ++k) mmax = std::max(mmax, op->m[k]);
    if (mmax > kLocalMaxM) return T2S2_EINVAL;
    R = std::max(std::max(rcap, rfmax), kick);
    const size_t core = (size_t)R * mmax * R;
    // B'_k = c_op B_k + (c_mass / d) I, every dimension in one launch
    {
      BprimeArgs ba;
      ba.d = d;
      ba.c_op = c_op;
      ba.shift = c_mass / d;
      int mmx = 1;
      for (int k = 0; k < d; ++k) {
        const int m = op->m[k];
        Bp[k] = aget<double>(c, (size_t)m * m);
        if (!Bp[k]) return T2S2_ENOMEM;
        ba.out[k] = Bp[k];
        ba.B[k] = op->dB[k];
        ba.I[k] = op->dI[k];
        ba.mm[k] = m * m;
        mmx = std::max(mmx, m * m);
      }
      {
        TraceScope ts_(kTrElem, c.st, 2.0 * d * mmx, 24.0 * d * mmx);
        (void)launch_pdl(k_bprime, (unsigned)std::min(64, (mmx + 255) / 256), 256, 0, c.st, ba);
      }
      T2S2_CUDA_TRY(cudaGetLastError());
    }
    // transformed right-hand side f = M^{-1} b (mode-k products with Rt_k^{-1})
    // (always FP64: the right-hand side fixes what the inner solve converges to)
    T2S2_TRY(tt_alloc(c, f, d, op->m, b.r, 0));
    {
      Ctx c64 = c;
      c64.contract_prec = T2S2_FP64;
      Gemm<double> gs[T2S2_MAX_D];
      for (int k = 0; k < d; ++k) gs[k] = g_mode2(op->dRinv[k], op->m[k], b.c[k], b.r[k], b.r[k + 1], f.c[k]);
      for (int k0 = 0; k0 < d; k0 += kMaxGroup) T2S2_TRY(contract_group(c64, gs + k0, std::min(kMaxGroup, d - k0)));
    }
    // x: copy of the initial guess with capacity rcap
    int rx[T2S2_MAX_D + 1];
    for (int k = 0; k <= d; ++k) rx[k] = x0.r[k];
    T2S2_TRY(tt_alloc(c, x, d, op->m, rx, R));
    T2S2_TRY(tt_copy(c, x0, x));
    int rx0 = 1;
    for (int k = 0; k <= d; ++k) rx0 = std::max(rx0, x0.r[k]);
    if (rx0 > rcap) T2S2_TRY(tt_round(c, x, 1e-15, rcap));
    // z: random rank-kick TT (bounded by the mode-size products)
    int rz[T2S2_MAX_D + 1];
    rz[0] = rz[d] = 1;
    for (int k = 1; k < d; ++k) {
      double left = 1, right = 1;
      for (int j = 0; j < k; ++j) left *= op->m[j];
      for (int j = k; j < d; ++j) right *= op->m[j];
      rz[k] = (int)std::min<double>(kick, std::min(left, right));
    }
    T2S2_TRY(tt_alloc(c, z, d, op->m, rz, kick));
    size_t zel = 0;
    for (int k = 0; k < d; ++k) zel += z.core_elems(k);
    if (op->zcache && op->zcache_kick == kick && op->zcache_elems == zel) {
      // the right-orthogonalised start of z depends only on the mode sizes
      // and the kick: kept with the operator after its first use
      size_t o = 0;
      for (int k = 0; k < d; ++k) {
        T2S2_TRY(d2d(c, z.c[k], op->zcache + o, z.core_elems(k)));
        o += z.core_elems(k);
      }
    } else {
      std::mt19937_64 gen(0x5eedULL + d);
      std::normal_distribution<double> nd(0.0, 1.0);
      std::vector<double> h(zel);
      for (auto& v : h) v = nd(gen);
      size_t o = 0;
      for (int k = 0; k < d; ++k) {
        T2S2_CUDA_TRY(cudaMemcpyAsync(z.c[k], h.data() + o, z.core_elems(k) * sizeof(double),
                                      cudaMemcpyHostToDevice, c.st));
        o += z.core_elems(k);
      }
      T2S2_CUDA_TRY(cudaStreamSynchronize(c.st));
      T2S2_TRY(tt_orth_right(c, z));
      if (op->zcache_elems < zel) {
        if (op->zcache) cudaFree(op->zcache);
        op->zcache = nullptr;
        op->zcache_elems = 0;
        T2S2_CUDA_TRY(cudaMalloc(&op->zcache, zel * sizeof(double)));
      }
      o = 0;
      for (int k = 0; k < d; ++k) {
        T2S2_TRY(d2d(c, op->zcache + o, z.c[k], z.core_elems(k)));
        o += z.core_elems(k);
      }
      op->zcache_elems = zel;
      op->zcache_kick = kick;
    }
    for (int k = 0; k <= d; ++k) {
      double** arrs[10] = {PL, FL, ZIL, ZBL, ZFL, PR, FR, ZIR, ZBR, ZFR};
      for (auto a : arrs) {
        a[k] = aget<double>(c, (size_t)R * R);
        if (!a[k]) return T2S2_ENOMEM;
      }
    }
    tmp_elems = core;
    for (auto& t : tmp) {
      t = aget<double>(c, core);
      if (!t) return T2S2_ENOMEM;
    }
    gm_work = aget<double>(c, local_work_elems<double>((long)rcap * mmax * rcap, gm_restart));
    if (fp32_local) {
      fbuf = aget<float>(c, 2 * core + local_work_elems<float>((long)rcap * mmax * rcap, gm_restart));
      if (!fbuf) return T2S2_ENOMEM;
    }
    gm_part = aget<double>(c, kLocalPartElems);
    gm_iters = reinterpret_cast<int*>(aget<double>(c, 2));
    gm_res = aget<double>(c, 4);
    svals = aget<double>(c, kSmallMax);
    {
      const char* e = std::getenv("T2S2_LOCAL_PRECOND");
      use_fls = !(e && e[0] == 'd');  // "diag": per-fibre diagonal shifts only
      const size_t side = (size_t)R + 2 * (size_t)R * R;  // complex values per side
      eig_buf = aget<double>(c, 2 * side);                 // 8 bytes per complex binary32
      ybuf = aget<double>(c, (size_t)rcap * mmax * rcap);
      eig_status = reinterpret_cast<int*>(aget<double>(c, 1));
      sylv_status = reinterpret_cast<int*>(aget<double>(c, 1));
      if (!sylv_status) return T2S2_ENOMEM;
      if (!eig_buf || !ybuf || !eig_status) return T2S2_ENOMEM;
    }
    {
      const char* e = std::getenv("T2S2_LOCAL_TIMING");
      tstamp_req = e && e[0] >= '0' && e[0] <= '9';
      tstamp_target = tstamp_req ? std::atoi(e) : 0;
      if (tstamp_req) {
        tstamp_dev = reinterpret_cast<unsigned long long*>(aget<double>(c, 2 + 8 * kLocalTimingIts));
        if (!tstamp_dev) return T2S2_ENOMEM;
        T2S2_CUDA_TRY(cudaMemsetAsync(tstamp_dev, 0, sizeof(unsigned long long) * (2 + 8 * kLocalTimingIts), c.st));
      }
    }
    if (!gm_work || !gm_part || !gm_iters || !gm_res || !svals) return T2S2_ENOMEM;
    return T2S2_OK;
  }

  // Right interfaces for bonds d-1 .. 1 from right-orthonormal x (and z).
  t2s2_status right_interfaces() {
    Ctx& c = *cx;
    T2S2_TRY(set_scalars(c, PR[d], 0.0, FR[d], 1.0, ZIR[d], 1.0, ZBR[d], 0.0, ZFR[d], 1.0));
    for (int k = d - 1; k >= 1; --k) {
      const int m = op->m[k];
      const int ra = x.r[k], rb = x.r[k + 1], fa = f.r[k], fb = f.r[k + 1], za = z.r[k], zb = z.r[k + 1];
      const double *X = x.c[k], *F = f.c[k], *Z = z.c[k];
      double *BX = tmp[0], *A1 = tmp[1], *A2 = tmp[2], *A3 = tmp[3], *A4 = tmp[4], *A5 = tmp[5];
      // PR[k] = X (X x_3 PR[k+1] + B' x_2 X),  FR[k] = X (F x_3 FR[k+1]),
      // ZIR[k] = Z (X x_3 ZIR[k+1]),  ZBR[k] = Z (X x_3 ZBR[k+1] + (B' X) x_3 ZIR[k+1]),
      // ZFR[k] = Z (F x_3 ZFR[k+1]): three launches of independent products
      const Gemm<double> s1[] = {g_mode2(Bp[k], m, X, ra, rb, BX),
                                 g_mode2(Bp[k], m, X, ra, rb, A1),
                                 g_mode3(F, fa, m, fb, FR[k + 1], rb, A2),
                                 g_mode3(X, ra, m, rb, ZIR[k + 1], zb, A3),
                                 g_mode3(X, ra, m, rb, ZBR[k + 1], zb, A4),
                                 g_mode3(F, fa, m, fb, ZFR[k + 1], zb, A5)};
      T2S2_TRY(group(c, s1));
      const Gemm<double> s2[] = {g_mode3(X, ra, m, rb, PR[k + 1], rb, A1, 1.0, 1.0),
                                 g_mode3(BX, ra, m, rb, ZIR[k + 1], zb, A4, 1.0, 1.0)};
      T2S2_TRY(group(c, s2));
      const Gemm<double> s3[] = {g_cright(X, ra, m, rb, A1, ra, PR[k]),
                                 g_cright(X, ra, m, rb, A2, fa, FR[k]),
                                 g_cright(Z, za, m, zb, A3, ra, ZIR[k]),
                                 g_cright(Z, za, m, zb, A4, ra, ZBR[k]),
                                 g_cright(Z, za, m, zb, A5, fa, ZFR[k])};
      T2S2_TRY(group(c, s3));
    }
    return T2S2_OK;
  }

  t2s2_status left_boundary() {
    Ctx& c = *cx;
    T2S2_TRY(set_scalars(c, PL[0], 0.0, FL[0], 1.0, ZIL[0], 1.0, ZBL[0], 0.0, ZFL[0], 1.0));
    return T2S2_OK;
  }

  t2s2_status local_solve(int k, double* rhs, double* X) {
    if (fp32_local) return local_solve_f32(k, rhs, X);
    Ctx& c = *cx;
    LocalProblem<double> P;
    P.ra = x.r[k];
    P.m = op->m[k];
    P.rb = x.r[k + 1];
    P.PL = PL[k];
    P.PR = PR[k + 1];
    P.Bp = Bp[k];
    P.Tr = op->fptr[5][k];
    P.Ti = op->fptr[6][k];
    P.Zr = op->fptr[7][k];
    P.Zi = op->fptr[8][k];
    P.c_op = c_op;
    P.shift = c_mass / d;
    P.rhs = rhs;
    P.x = X;
    P.work = gm_work;
    P.part = gm_part;
    P.tol_rel = ltol;
    P.maxit = gm_maxit;
    P.mr = gm_restart;
    P.iters_out = gm_iters;
    P.res_out = gm_res;
    P.fls = use_fls ? 1 : 0;
    P.team = op->team;
    P.eigL = eig_buf;
    P.eigR = eig_buf + (size_t)R + 2 * (size_t)R * R;
    P.eig_status = eig_status;
    P.ybuf = ybuf;
    const bool stamp_this = tstamp_req && !tstamp_done && local_count == tstamp_target;
    ++local_count;
    if (stamp_this) P.tstamp = tstamp_dev;
    if (P.rb == 1 && use_fls && sylv_rb1_fits(P.ra, P.m)) {
      // rb = 1: the Schur-basis Sylvester solver first; the general solver
      // below runs only if it leaves status 1
      SylvProblem S;
      S.ra = P.ra;
      S.m = P.m;
      S.PL = P.PL;
      S.PR = P.PR;
      S.Bp = P.Bp;
      S.Tr = P.Tr;
      S.Ti = P.Ti;
      S.Zr = P.Zr;
      S.Zi = P.Zi;
      S.c_op = P.c_op;
      S.shift = P.shift;
      S.rhs = P.rhs;
      S.x = P.x;
      S.tol_rel = P.tol_rel;
      S.status = sylv_status;
      S.iters_out = P.iters_out;
      S.res_out = P.res_out;
      if (stamp_this) {
        T2S2_CUDA_TRY(cudaMemsetAsync(tstamp_dev, 0, sizeof(unsigned long long) * kSylvStamps, c.st));
        S.tstamp = tstamp_dev;
      }
      T2S2_TRY(sylv_rb1(S, c.st));
      P.skip = sylv_status;
      if (stamp_this) {
        unsigned long long h[kSylvStamps];
        T2S2_CUDA_TRY(cudaMemcpyAsync(h, tstamp_dev, sizeof(h), cudaMemcpyDeviceToHost, c.st));
        T2S2_CUDA_TRY(cudaStreamSynchronize(c.st));
        fprintf(stderr, "[t2s2] rb=1 local solve phase times (ns) ra=%d m=%d:", P.ra, P.m);
        for (int i = 1; i < kSylvStamps && h[i]; ++i) fprintf(stderr, " %lld", (long long)(h[i] - h[i - 1]));
        fprintf(stderr, "\n");
        P.tstamp = nullptr;
      }
      // In the first sweep the general solver (an eigendecomposition launch
      // and a cooperative GMRES launch that return at once when the Sylvester
      // solver succeeded) is not queued: when the Sylvester solver stops short
      // of the local tolerance its iterate (the guess, or its last refinement)
      // stays in X, the global residual after the sweep decides, and every
      // later sweep queues the general solver again.
      if (sylv_no_fallback) {
        if (stamp_this) tstamp_done = true;
        return T2S2_OK;
      }
    }
    T2S2_TRY(local_gmres<double>(P, c.st));
    if (stamp_this) {
      tstamp_done = true;
      unsigned long long h[2 + 8 * kLocalTimingIts];
      T2S2_CUDA_TRY(cudaMemcpyAsync(h, tstamp_dev, sizeof(h), cudaMemcpyDeviceToHost, c.st));
      T2S2_CUDA_TRY(cudaStreamSynchronize(c.st));
      fprintf(stderr, "[t2s2] local solve phase times (ns) ra=%d m=%d rb=%d:", P.ra, P.m, P.rb);
      for (int i = 1; i < 2 + 8 * kLocalTimingIts; ++i) fprintf(stderr, " %lld", (long long)(h[i] - h[i - 1]));
      fprintf(stderr, "\n");
    }
    return T2S2_OK;
  }

  // FP32 local solve (mixed precision): the caller's FP64 rhs / guess are
  // rounded to binary32, solved, and the result widened back.
  t2s2_status local_solve_f32(int k, double* rhs, double* X) {
    Ctx& c = *cx;
    const size_t N = (size_t)x.r[k] * op->m[k] * x.r[k + 1];
    float* frhs = fbuf;
    float* fx = fbuf + tmp_elems;
    float* fwork = fbuf + 2 * tmp_elems;
    T2S2_TRY(dev_d2f(c, frhs, rhs, N));
    T2S2_TRY(dev_d2f(c, fx, X, N));
    LocalProblem<float> P;
    P.ra = x.r[k];
    P.m = op->m[k];
    P.rb = x.r[k + 1];
    P.PL = PL[k];
    P.PR = PR[k + 1];
    P.Bp = Bp[k];
    P.Tr = op->fptr[5][k];
    P.Ti = op->fptr[6][k];
    P.Zr = op->fptr[7][k];
    P.Zi = op->fptr[8][k];
    P.c_op = c_op;
    P.shift = c_mass / d;
    P.rhs = frhs;
    P.x = fx;
    P.work = fwork;
    P.part = gm_part;
    P.tol_rel = std::max(ltol, 2e-6);
    P.maxit = gm_maxit;
    P.mr = gm_restart;
    P.iters_out = gm_iters;
    P.res_out = gm_res;
    P.fls = use_fls ? 1 : 0;
    P.team = op->team;
    P.eigL = eig_buf;
    P.eigR = eig_buf + (size_t)R + 2 * (size_t)R * R;
    P.eig_status = eig_status;
    P.ybuf = ybuf;
    T2S2_TRY(local_gmres<float>(P, c.st));
    return dev_f2d(c, X, fx, N);
  }

  // One forward sweep k = 0 .. d-1.
  t2s2_status sweep() {
    Ctx& c = *cx;
    ph(1);
    T2S2_TRY(right_interfaces());
    T2S2_TRY(left_boundary());
    for (int k = 0; k < d; ++k) {
      ph(2);
      const int m = op->m[k];
      const int ra = x.r[k], rb = x.r[k + 1], fa = f.r[k], fb = f.r[k + 1], za = z.r[k], zb = z.r[k + 1];
      const double* F = f.c[k];
      double *rhs = tmp[3], *X = tmp[4], *T1 = tmp[0], *T2 = tmp[1];
      // local rhs = FL[k] x_1 F x_3 FR[k+1] (one launch slice by slice where
      // the matrices fit shared memory)
      {
        const size_t sm = sizeof(double) * ((size_t)ra * fa + (size_t)fa * fb + (size_t)rb * fb + (size_t)ra * fb);
        if (c.contract_prec != T2S2_BF16_REFINE && c.contract_prec != T2S2_TF32_REFINE && sm <= kEnrichMaxSmem) {
          static std::once_flag attr;
          std::call_once(attr, [] {
            if (cudaFuncSetAttribute(k_local_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEnrichMaxSmem) !=
                cudaSuccess)
              cudaGetLastError();
          });
          RhsArgs ar;
          ar.ra = ra, ar.rb = rb, ar.fa = fa, ar.fb = fb, ar.m = m;
          ar.FL = FL[k], ar.F = F, ar.FR = FR[k + 1], ar.T1 = T1, ar.rhs = rhs;
          {
            TraceScope ts_(kTrGemm, c.st, 2.0 * m * (double)ra * fb * (fa + rb),
                           8.0 * m * ((double)fa * fb + ra * fb + ra * rb));
            (void)launch_pdl(k_local_rhs, (unsigned)m, kEnrichThreads, sm, c.st, ar);
          }
          T2S2_CUDA_TRY(cudaGetLastError());
        } else {
          T2S2_TRY(mode1(c, FL[k], ra, fa, F, m, fb, T1));
          T2S2_TRY(mode3(c, T1, ra, m, fb, FR[k + 1], rb, rhs));
        }
      }
      T2S2_TRY(d2d(c, X, x.c[k], (size_t)ra * m * rb));
      ph(3);
      T2S2_TRY(local_solve(k, rhs, X));
      ph(4);
      if (k == d - 1) {
        T2S2_TRY(d2d(c, x.c[k], X, (size_t)ra * m * rb));
        // the count is read after the solver's next synchronisation
        T2S2_TRY(defer_iters(ra, m, rb));
        break;
      }
      // --- truncation: X (rows x rb) = U S V^T
      const int rows = ra * m;
      double *Qx = tmp[5], *Ux = tmp[6], *Vx = tmp[7], *Rx = tmp[8];
      double *U = tmp[9], *SV = tmp[10], *Xt = tmp[11];
      int kk, rk;
      if (rb == 1) {
        // a single column: U = X / |X|, S V^T = |X|, rank 1 -- no
        // factorisation and no read-back
        {
          TraceScope ts(kTrSmall, c.st, 3.0 * rows, 24.0 * rows);
          (void)launch_pdl(k_col_split, 1, 256, 0, c.st, X, rows, U, SV, Xt);
        }
        T2S2_CUDA_TRY(cudaGetLastError());
        T2S2_TRY(defer_iters(ra, m, rb));
        rk = 1;
      } else {
      if (rows >= rb) {
        T2S2_TRY(qr_tall(c, X, rows, rb, Qx, Rx));
        T2S2_TRY(jacobi_svd(Rx, rb, rb, Ux, svals, Vx, nullptr, c.st));
        kk = rb;
      } else {
        T2S2_TRY(jacobi_svd(X, rows, rb, Ux, svals, Vx, nullptr, c.st));
        kk = rows;
      }
      T2S2_CUDA_TRY(cudaMemcpyAsync(c.hbuf, svals, sizeof(double) * kk, cudaMemcpyDeviceToHost, c.st));
      T2S2_CUDA_TRY(cudaMemcpyAsync(c.hbuf + kSmallMax, gm_iters, sizeof(int), cudaMemcpyDeviceToHost, c.st));
      T2S2_CUDA_TRY(cudaStreamSynchronize(c.st));
      {
        int it;
        std::memcpy(&it, c.hbuf + kSmallMax, sizeof(int));
        local_iters += it;
        trace_add_work(kTrLocal, local_flops(ra, m, rb, it, gm_restart), 0.0);
      }
      double snorm = 0.0;
      for (int j = 0; j < kk; ++j) snorm += c.hbuf[j] * c.hbuf[j];
      snorm = std::sqrt(snorm);
      rk = trunc_rank(c.hbuf, kk, ltol * snorm, rmax);
      if (rows >= rb) {
        T2S2_TRY(gemm_ex<double>(c, rows, rk, rb, false, false, 1.0, Qx, rb, Ux, kk, 0.0, U, rk));
      } else {
        T2S2_CUDA_TRY(cudaMemcpy2DAsync(U, sizeof(double) * rk, Ux, sizeof(double) * kk,
                                        sizeof(double) * rk, rows, cudaMemcpyDeviceToDevice, c.st));
      }
      T2S2_TRY(dev_sv_t(c, SV, svals, Vx, rk, rb, kk));
      T2S2_TRY(gemm_ex<double>(c, rows, rb, rk, false, false, 1.0, U, rk, SV, rb, 0.0, Xt, rb));
      }
      ph(5);
      // --- enrichment directions: residual on (x-left) x m x (z-right),
      //   res  = (FL F) x_3 ZFR - (B' Xt + PL Xt) x_3 ZIR - Xt x_3 ZBR,
      // --- z update: residual on (z-left) x m x (z-right),
      //   zres = (ZFL F) x_3 ZFR - (ZBL Xt + ZIL B' Xt) x_3 ZIR - (ZIL Xt) x_3 ZBR;
      // one launch slice by slice (k_enrich) where the cores fit shared
      // memory, else four launches of independent products.  tmp[0] still
      // holds FL[k] x_1 F from the local right-hand side.
      double *Tz = tmp[2], *T2b = tmp[3];  // T1 = tmp[0], T2 = tmp[1]
      double *BX = tmp[5], *Y1 = tmp[6], *res = tmp[7], *zres = tmp[8];
      bool fused = false;
      if (c.contract_prec != T2S2_BF16_REFINE && c.contract_prec != T2S2_TF32_REFINE) {
        EnrichArgs ea;
        ea.ra = ra, ea.rb = rb, ea.fa = fa, ea.fb = fb, ea.za = za, ea.zb = zb, ea.m = m;
        ea.Xt = Xt, ea.BX = BX, ea.T1 = T1, ea.F = F, ea.Bp = Bp[k];
        ea.PL = PL[k], ea.ZBL = ZBL[k], ea.ZIL = ZIL[k], ea.ZFL = ZFL[k];
        ea.ZFR = ZFR[k + 1], ea.ZIR = ZIR[k + 1], ea.ZBR = ZBR[k + 1];
        ea.res = res, ea.zres = zres;
        ea.bx_here = 1;
        size_t sm = enrich_smem_doubles(ea) * sizeof(double);
        if (sm > kEnrichMaxSmem) {
          ea.bx_here = 0;
          sm = enrich_smem_doubles(ea) * sizeof(double);
        }
        if (sm <= kEnrichMaxSmem) {
          static std::once_flag attr;
          std::call_once(attr, [] {
            if (cudaFuncSetAttribute(k_enrich, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEnrichMaxSmem) !=
                cudaSuccess)
              cudaGetLastError();
          });
          if (!ea.bx_here) T2S2_TRY(contract_gemm(c, g_mode2(Bp[k], m, Xt, ra, rb, BX)));
          {
            const double fl = 2.0 * m * ((double)ra * rb * (ra + 2.0 * za) + (double)za * fa * fb +
                                         (double)(ra + za) * zb * (fb + 2.0 * rb)) +
                              (ea.bx_here ? 2.0 * ra * m * (double)m * rb : 0.0);
            TraceScope ts_(kTrGemm, c.st, fl, 8.0 * m * ((double)ra * rb + ra * fb + fa * fb + (ra + za) * zb));
            (void)launch_pdl(k_enrich, (unsigned)m, kEnrichThreads, sm, c.st, ea);
          }
          T2S2_CUDA_TRY(cudaGetLastError());
          fused = true;
        }
      }
      if (!fused) {
        const Gemm<double> s1[] = {g_mode2(Bp[k], m, Xt, ra, rb, BX),
                                   g_mode2(Bp[k], m, Xt, ra, rb, Y1),
                                   g_mode1(ZFL[k], za, fa, F, m, fb, Tz),
                                   g_mode1(ZBL[k], za, ra, Xt, m, rb, T2),
                                   g_mode1(ZIL[k], za, ra, Xt, m, rb, T2b)};
        T2S2_TRY(group(c, s1));
        const Gemm<double> s2[] = {g_mode1(PL[k], ra, ra, Xt, m, rb, Y1, 1.0, 1.0),
                                   g_mode1(ZIL[k], za, ra, BX, m, rb, T2, 1.0, 1.0),
                                   g_mode3(T1, ra, m, fb, ZFR[k + 1], zb, res),
                                   g_mode3(Tz, za, m, fb, ZFR[k + 1], zb, zres)};
        T2S2_TRY(group(c, s2));
        const Gemm<double> s3[] = {g_mode3(Y1, ra, m, rb, ZIR[k + 1], zb, res, -1.0, 1.0),
                                   g_mode3(T2, za, m, rb, ZIR[k + 1], zb, zres, -1.0, 1.0)};
        T2S2_TRY(group(c, s3));
        const Gemm<double> s4[] = {g_mode3(Xt, ra, m, rb, ZBR[k + 1], zb, res, -1.0, 1.0),
                                   g_mode3(T2b, za, m, rb, ZBR[k + 1], zb, zres, -1.0, 1.0)};
        T2S2_TRY(group(c, s4));
      }
      ph(6);
      // the orthonormal factor goes straight into z's core k (same shape); on
      // the operator's side stream it overlaps the new core's QR below and
      // joins before the left interfaces read z's core k
      const size_t zmark = c.ar->mark();
      bool zside = false;
      {
        double* Rz = tmp[3];
        t2s2_status zs = T2S2_OK;
        if (side_ready()) {
          T2S2_CUDA_TRY(cudaEventRecord(op->ev_fork, c.st));
          T2S2_CUDA_TRY(cudaStreamWaitEvent(op->side, op->ev_fork, 0));
          zside = qr_tall_async(c, zres, za * m, zb, z.c[k], Rz, op->side, &zs);
          T2S2_TRY(zs);
          if (zside) T2S2_CUDA_TRY(cudaEventRecord(op->ev_join, op->side));
        }
        if (!zside) T2S2_TRY(qr_tall(c, zres, za * m, zb, z.c[k], Rz));
      }
      ph(7);
      // --- new core: orthonormal basis of [U | res], written over core k
      // (whose old content the local solve has consumed)
      const int cols = rk + zb;
      const int mn = op->m[k + 1], rnn = x.r[k + 2];
      const int rn = (rows >= cols) ? cols : rows;
      if ((size_t)rn * mn * rnn > x.cap[k + 1] || (size_t)rows * rn > x.cap[k]) return T2S2_ENOMEM;
      double* Q = x.c[k];
      if (rows >= cols) {
        double* Rq = tmp[5];  // tmp[8] holds zres, which the side stream may still read
        T2S2_TRY(qr_tall2(c, U, rk, res, zb, rows, Q, Rq, tmp[1]));
      } else {
        T2S2_TRY(dev_identity(c, Q, rows));
      }
      // next core: (Q^T U SV) x_1 x[k+1], carried in FP64 whatever the
      // contraction arithmetic
      {
        const size_t nx = (size_t)rb * mn * rnn;
        const size_t sm = sizeof(double) * (nx + (size_t)rn * (rk + rb));
        if (sm <= kNextCoreSmem) {
          TraceScope ts(kTrGemm, c.st, 2.0 * rows * rn * rk + 2.0 * rn * rk * rb + 2.0 * rn * (double)nx, 0.0);
          (void)launch_pdl(k_next_core, 1, 256, sm, c.st, Q, U, SV, rows, rn, rk, rb, x.c[k + 1], mn, rnn);
          T2S2_CUDA_TRY(cudaGetLastError());
        } else {
          double* C = tmp[6];
          double* CS = tmp[7];
          double* P = tmp[0];
          T2S2_TRY(gemm_ex<double>(c, rn, rk, rows, true, false, 1.0, Q, rn, U, rk, 0.0, C, rk));
          T2S2_TRY(gemm_ex<double>(c, rn, rb, rk, false, false, 1.0, C, rk, SV, rb, 0.0, CS, rb));
          Ctx c64 = c;
          c64.contract_prec = T2S2_FP64;
          T2S2_TRY(mode1(c64, CS, rn, rb, x.c[k + 1], mn, rnn, P));
          T2S2_TRY(d2d(c, x.c[k + 1], P, nx / rb * rn));
        }
        x.r[k + 1] = rn;
      }
      ph(8);
      if (zside) T2S2_CUDA_TRY(cudaStreamWaitEvent(c.st, op->ev_join, 0));
      c.ar->release(zmark);
      // --- left interfaces for bond k+1:
      //   PL' = Qc^T (PL Qc + B' Qc),  FL' = Qc^T (FL F),  ZIL' = Z^T (ZIL Qc),
      //   ZBL' = Z^T (ZBL Qc + ZIL B' Qc),  ZFL' = Z^T (ZFL F)
      // in three launches of independent products
      {
        const double* Qc = x.c[k];
        const double* Z = z.c[k];
        double *BQ = tmp[3], *A1 = tmp[4], *A2 = tmp[5], *A3 = tmp[6], *A4 = tmp[7], *A5 = tmp[8];
        const Gemm<double> s1[] = {g_mode2(Bp[k], m, Qc, ra, rn, BQ),
                                   g_mode2(Bp[k], m, Qc, ra, rn, A1),
                                   g_mode1(FL[k], ra, fa, F, m, fb, A2),
                                   g_mode1(ZIL[k], za, ra, Qc, m, rn, A3),
                                   g_mode1(ZBL[k], za, ra, Qc, m, rn, A4),
                                   g_mode1(ZFL[k], za, fa, F, m, fb, A5)};
        T2S2_TRY(group(c, s1));
        const Gemm<double> s2[] = {g_mode1(PL[k], ra, ra, Qc, m, rn, A1, 1.0, 1.0),
                                   g_mode1(ZIL[k], za, ra, BQ, m, rn, A4, 1.0, 1.0)};
        T2S2_TRY(group(c, s2));
        const Gemm<double> s3[] = {g_cleft(Qc, ra, m, rn, A1, rn, PL[k + 1]),
                                   g_cleft(Qc, ra, m, rn, A2, fb, FL[k + 1]),
                                   g_cleft(Z, za, m, zb, A3, rn, ZIL[k + 1]),
                                   g_cleft(Z, za, m, zb, A4, rn, ZBL[k + 1]),
                                   g_cleft(Z, za, m, zb, A5, fb, ZFL[k + 1])};
        T2S2_TRY(group(c, s3));
      }
    }
    return T2S2_OK;
  }
};

t2s2_status refine_impl(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                        double tol, int rmax, int max_sweeps, t2s2_precision prec, t2s2_solve_info* info);

t2s2_status solve_impl(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                       double tol, int rmax, int max_sweeps, t2s2_precision prec, t2s2_solve_info* info) {
  if (prec != T2S2_FP64) return refine_impl(op, cx, b, xio, c_mass, c_op, tol, rmax, max_sweeps, prec, info);
  Amen am;
  PhaseTimer pt;
  pt.start(cx.st);
  am.pt = &pt;
  am.ph(0);
  T2S2_TRY(am.init(op, cx, b, xio, c_mass, c_op, tol, rmax));
  T2S2_TRY(tt_orth_right(cx, am.x));
  // the residual of the original system, before and after every sweep
  ResidualCache rcache;
  double res = 0.0;
  T2S2_TRY(residual_fast(op, cx, b, am.x, c_mass, c_op, &res, &rcache, true));
  int sweeps = 0;
  const char* ev = std::getenv("T2S2_VERBOSE");
  const bool verbose = ev && ev[0] == '1';
  if (verbose) fprintf(stderr, "[t2s2] solve d=%d c_mass=%g c_op=%g tol=%g rmax=%d initial residual %.3e\n",
                       op->d, c_mass, c_op, tol, rmax, res);
  // stagnation under the rank cap: once some bond carries rmax + kick and the
  // residual has not halved in stall_sweeps() sweeps, more sweeps at that cap
  // do not reach tol (the cap, not the sweep count, limits the solution)
  const int kStallSweeps = stall_sweeps();
  double mark = res;
  int mark_sweep = 0;
  while (res > tol && sweeps < max_sweeps) {
    am.sylv_no_fallback = sweeps == 0;
    T2S2_TRY(am.sweep());
    ++sweeps;
    am.ph(9);
    T2S2_TRY(residual_fast(op, cx, b, am.x, c_mass, c_op, &res, &rcache, false));
    if (res < 0.5 * mark) {
      mark = res;
      mark_sweep = sweeps;
    }
    int rx = 1;
    for (int k = 0; k <= op->d; ++k) rx = std::max(rx, am.x.r[k]);
    const bool stalled =
        kStallSweeps > 0 && res > tol && rx >= am.rcap && sweeps - mark_sweep >= kStallSweeps;
    T2S2_TRY(am.collect_iters());
    if (verbose) {
      double rt = 0.0;
      T2S2_TRY(residual_impl(op, cx, am.f, am.x, c_mass, c_op, true, &rt, nullptr));
      fprintf(stderr, "[t2s2] sweep %d residual %.3e (transformed %.3e) ranks", sweeps, res, rt);
      for (int k = 0; k <= op->d; ++k) fprintf(stderr, " %d", am.x.r[k]);
      fprintf(stderr, " local_iters %lld%s\n", am.local_iters, stalled ? " (stalled at the rank cap)" : "");
    }
    if (res <= tol || stalled) break;
    am.ph(10);
    T2S2_TRY(tt_orth_right(cx, am.x));
  }
  am.ph(0);
  pt.report();
  // copy out
  for (int k = 0; k < op->d; ++k)
    if (am.x.core_elems(k) > xio.cap[k]) return T2S2_ENOMEM;
  T2S2_TRY(tt_copy(cx, am.x, xio));
  if (info) {
    info->residual = res;
    info->sweeps = sweeps;
    int mr = 1;
    for (int k = 0; k <= op->d; ++k) mr = std::max(mr, am.x.r[k]);
    info->max_rank = mr;
    info->refinements = 0;
    info->local_iters = am.local_iters;
  }
  return res <= tol ? T2S2_OK : T2S2_ENOCONV;
}

// Mixed precision with iterative refinement.  The outer loop is FP64:
//     r = b - (c_mass M + c_op A) x                (FP64 apply and TT sum),
//     r <- rndg(r) at a tenth of the inner tolerance,
//     delta ~ (c_mass M + c_op A)^{-1} r           (inner AMEn, loose tolerance),
//     x <- rndg(x + delta) at tol / 10, rank cap rmax,
// until the FP64 residual ||b - A x|| / ||b|| <= tol.  The inner AMEn runs
// its local solves in binary32 and, for TF32 / BF16, its core contractions
// (mode products and interface updates) on the tensor cores; its QR / SVD,
// the residual and every rounding stay FP64.
//
// The contraction arithmetic puts a floor under what one inner solve can
// reach (about 2u: near 1e-3 for TF32, 1e-2 for BF16), so the inner target is
// set above it per precision, and an inner solve that stops improving ends
// early.  A correction computed with rounded contractions also carries
// rounding noise of relative size ~u ||delta||, spread over many TT ranks;
// once ||delta|| is small that noise can no longer be represented under the
// rank cap and refinement stalls (near 5e-6 for TF32 on the d = 6, n = 32
// problem).  So the tensor-core contractions serve a first stage only: an
// inner solve of the whole system down to their floor, whose result is not
// added to x but becomes the initial guess of the next inner solve of the
// whole system, with FP64 contractions and binary32 local solves (the
// alternating sweeps re-solve every core and so discard the noise); then the
// corrections proceed as usual.  When the caller's x0 is worse than zero
// (residual above 1) the loop starts from x = 0, so that the first inner
// solve is the original system and takes x0 as its initial guess (a warm
// start acts there); each later correction starts from the previous one,
// whose ranks already fit the error's.
double inner_tol_for(t2s2_precision prec) {
  switch (prec) {
    case T2S2_BF16_REFINE: return 3e-2;
    case T2S2_TF32_REFINE: return 3e-3;
    default: return 1e-4;
  }
}

t2s2_status refine_impl(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                        double tol, int rmax, int max_sweeps, t2s2_precision prec, t2s2_solve_info* info) {
  const double kInnerTol = inner_tol_for(prec);
  constexpr int kMaxRefinements = 40;
  const int d = op->d;
  const int kick = cx.kick > 0 ? cx.kick : amen_kick(), rcap = rmax + kick;
  const char* ev = std::getenv("T2S2_VERBOSE");
  const bool verbose = ev && ev[0] == '1';
  // persistent state: the iterate x, the caller's guess g and the previous
  // correction dprev (capacity rcap each)
  DevTT x, g, ones, dprev;
  int rx[T2S2_MAX_D + 1];
  for (int k = 0; k <= d; ++k) rx[k] = std::min(xio.r[k], rcap);
  rx[0] = rx[d] = 1;
  T2S2_TRY(tt_alloc(cx, x, d, op->m, rx, rcap));
  T2S2_TRY(tt_alloc(cx, g, d, op->m, rx, rcap));
  {
    int r1[T2S2_MAX_D + 1];
    for (int k = 0; k <= d; ++k) r1[k] = 1;
    T2S2_TRY(tt_alloc(cx, ones, d, op->m, r1, 1));
    for (int k = 0; k < d; ++k) T2S2_TRY(dev_fill(cx, ones.c[k], op->m[k], 1.0));
    T2S2_TRY(tt_alloc(cx, dprev, d, op->m, r1, rcap));
    T2S2_TRY(tt_copy(cx, ones, dprev));
  }
  {
    const size_t mk = cx.ar->mark();
    DevTT t;
    T2S2_TRY(tt_alloc(cx, t, d, op->m, xio.r, 0));
    T2S2_TRY(tt_copy(cx, xio, t));
    T2S2_TRY(tt_round(cx, t, 0.0, rcap));
    for (int k = 0; k <= d; ++k) x.r[k] = g.r[k] = t.r[k];
    T2S2_TRY(tt_copy(cx, t, x));
    T2S2_TRY(tt_copy(cx, t, g));
    cx.ar->release(mk);
  }
  ResidualCache rcache;
  double res = 0.0;
  T2S2_TRY(residual_fast(op, cx, b, x, c_mass, c_op, &res, &rcache, true));
  bool x_zero = false;
  if (res >= 1.0) {  // x0 is worse than x = 0
    x_zero = true;
    res = 1.0;
  }
  if (verbose)
    fprintf(stderr, "[t2s2] refine d=%d prec=%d tol=%g initial residual %.3e%s\n", d, (int)prec, tol, res,
            x_zero ? " (starting from x = 0)" : "");
  const bool tc = prec == T2S2_BF16_REFINE || prec == T2S2_TF32_REFINE;
  if (tc) T2S2_CUDA_TRY(cudaMemsetAsync(cx.dstat + kStatTensorCore, 0, sizeof(int), cx.st));
  bool tc_stage = tc;  // the tensor-core stage: a guess for the whole system
  if (tc_stage && !x_zero) {
    // start that stage from the caller's iterate: solve the whole system
    x_zero = true;
    res = 1.0;
  }
  int sweeps = 0, refinements = 0, stall = 0;
  long long local_iters = 0;
  while (res > tol && sweeps < max_sweeps && refinements < kMaxRefinements) {
    const size_t mk = cx.ar->mark();
    // the inner target follows the stage's contraction arithmetic
    const double tin = std::max(tc_stage ? kInnerTol : inner_tol_for(T2S2_FP32_REFINE), 0.5 * tol / res);
    // r = b - A x in FP64, rounded (r = b while x = 0)
    DevTT r;
    const DevTT* rhs = &b;
    if (!x_zero) {
      DevTT y;
      int r2[T2S2_MAX_D + 1];
      for (int k = 0; k <= d; ++k) r2[k] = (k == 0 || k == d) ? 1 : 2 * x.r[k];
      T2S2_TRY(tt_alloc(cx, y, d, op->m, r2, 0));
      T2S2_TRY(apply_op(op, cx, x, y, c_mass, c_op, false));
      T2S2_TRY(tt_axpby(cx, 1.0, b, -1.0, y, r));
      T2S2_TRY(tt_round(cx, r, 0.1 * tin, std::min(kSmallMax, 2 * rcap)));
      rhs = &r;
    }
    // inner solve: tensor-core contractions in the first stage only
    Ctx cl = cx;
    cl.contract_prec = tc_stage ? (int)prec : (int)T2S2_FP64;
    Amen am;
    am.fp32_local = true;
    T2S2_TRY(am.init(op, cl, *rhs, x_zero ? g : dprev, c_mass, c_op, tin, rmax));
    T2S2_TRY(tt_orth_right(cl, am.x));
    double rnorm = -1.0;
    T2S2_TRY(tt_norm(cx, *rhs, &rnorm));
    double est = 1.0, est_prev2 = 1e300, est_prev = 1e300;
    int inner = 0;
    while (sweeps < max_sweeps) {
      T2S2_TRY(am.sweep());
      ++sweeps;
      ++inner;
      double rr = rnorm * rnorm;
      T2S2_TRY(residual_estimate(op, cx, *rhs, am.x, c_mass, c_op, &rr, &est));
      T2S2_TRY(am.collect_iters());
      if (verbose) {
        fprintf(stderr, "[t2s2]   inner sweep %d est %.3e ranks", inner, est);
        for (int k = 0; k <= d; ++k) fprintf(stderr, " %d", am.x.r[k]);
        fprintf(stderr, " local_iters %lld\n", am.local_iters);
      }
      if (est <= tin) break;
      if (inner >= 3 && est > 0.7 * est_prev2) break;  // at the precision floor
      est_prev2 = est_prev;
      est_prev = est;
      T2S2_TRY(tt_orth_right(cl, am.x));
    }
    local_iters += am.local_iters;
    if (tc_stage) {
      // its result seeds the next solve of the whole system (x stays 0)
      for (int k = 0; k < d; ++k)
        if (am.x.core_elems(k) > g.cap[k]) return T2S2_ENOMEM;
      T2S2_TRY(tt_copy(cx, am.x, g));
      cx.ar->release(mk);
      tc_stage = false;
      ++refinements;
      if (verbose) {
        double rg = 0.0;
        T2S2_TRY(residual_fast(op, cx, b, g, c_mass, c_op, &rg, &rcache, true));
        fprintf(stderr, "[t2s2] tensor-core stage: inner sweeps %d est %.2e residual %.3e\n", inner, est, rg);
      }
      continue;
    }
    if (am.x.core_elems(0) > 0) {
      bool fits = true;
      for (int k = 0; k < d; ++k) fits = fits && am.x.core_elems(k) <= dprev.cap[k];
      if (fits) T2S2_TRY(tt_copy(cx, am.x, dprev));
    }
    // x <- rndg(x + delta)  (x <- delta while x = 0)
    DevTT z;
    if (x_zero) {
      int rz[T2S2_MAX_D + 1];
      for (int k = 0; k <= d; ++k) rz[k] = am.x.r[k];
      T2S2_TRY(tt_alloc(cx, z, d, op->m, rz, 0));
      T2S2_TRY(tt_copy(cx, am.x, z));
    } else {
      T2S2_TRY(tt_axpby(cx, 1.0, x, 1.0, am.x, z));
    }
    T2S2_TRY(tt_round(cx, z, 0.1 * tol, rmax));
    for (int k = 0; k < d; ++k)
      if (z.core_elems(k) > x.cap[k]) return T2S2_ENOMEM;
    for (int k = 0; k <= d; ++k) x.r[k] = z.r[k];
    T2S2_TRY(tt_copy(cx, z, x));
    cx.ar->release(mk);
    x_zero = false;
    ++refinements;
    const double prev = res;
    T2S2_TRY(residual_fast(op, cx, b, x, c_mass, c_op, &res, &rcache, true));
    if (verbose) {
      fprintf(stderr, "[t2s2] refinement %d: inner sweeps %d est %.2e (target %.1e) residual %.3e ranks", refinements,
              inner, est, tin, res);
      for (int k = 0; k <= d; ++k) fprintf(stderr, " %d", x.r[k]);
      fprintf(stderr, "\n");
    }
    stall = (res > 0.5 * prev) ? stall + 1 : 0;
    if (stall >= 3) break;  // no longer contracting (rank cap or precision floor)
  }
  if (tc) T2S2_TRY(tensor_core_status(cx));
  for (int k = 0; k < d; ++k)
    if (x.core_elems(k) > xio.cap[k]) return T2S2_ENOMEM;
  for (int k = 0; k <= d; ++k) xio.r[k] = x.r[k];
  T2S2_TRY(tt_copy(cx, x, xio));
  if (info) {
    info->residual = res;
    info->sweeps = sweeps;
    int mr = 1;
    for (int k = 0; k <= d; ++k) mr = std::max(mr, x.r[k]);
    info->max_rank = mr;
    info->refinements = refinements;
    info->local_iters = local_iters;
  }
  return res <= tol ? T2S2_OK : T2S2_ENOCONV;
}

}  // namespace

// The public apply: FP64 and FP32_REFINE take the FP64 kernel; BF16 / TF32
// take the tcgen05 kernel when every core has m <= 64 (else the FP64 one).
t2s2_status apply_dispatch(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass,
                           double c_op, t2s2_precision prec) {
  ApplyBatch b;
  T2S2_TRY(apply_batch(op, x, y, c_mass, c_op, false, b));
  if ((prec == T2S2_BF16_REFINE || prec == T2S2_TF32_REFINE) && apply_tc_supported(b)) {
    int* err = cx.dstat + kStatTensorCore;
    T2S2_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), cx.st));
    T2S2_TRY(apply_tc(b, prec, err, cx.st));
    return tensor_core_status(cx);
  }
  return apply_fp64(b, cx.st);
}

// Arena bytes the refinement loop needs beyond one FP64 solve: the iterate,
// A x, the residual train and x + delta (all at most rank rf + 2 rcap), and
// the inner solver's workspace for a right-hand side of rank 2 rcap.
static size_t refine_extra_bytes(t2s2_op op, int rcap, int rf) {
  size_t mm = 0;
  for (int k = 0; k < op->d; ++k) mm = std::max<size_t>(mm, op->m[k]);
  const size_t R = (size_t)rf + 2 * rcap;
  const size_t train = (size_t)op->d * R * mm * R * sizeof(double);
  return 6 * train + Amen::bytes_needed(op->d, op->m, rcap, std::min(kSmallMax, 2 * rcap), amen_kick(), 40);
}

t2s2_status solve_run(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                      double tol, int rmax, int max_sweeps, t2s2_precision prec, t2s2_solve_info* info) {
  return solve_impl(op, cx, b, xio, c_mass, c_op, tol, rmax, max_sweeps, prec, info);
}

// Operators with a product reaction P: the reaction-free operator shifted by
// the product's mean, K = c_mass M + c_op A + c_op rho_bar M, is solved by the
// alternating solver with the rest of the reaction lagged,
//     K x_{j+1} = b - c_op (P - rho_bar M) x_j,
// each solve starting from x_j (its right-hand side is as smooth as b and
// x_j, unlike a residual) at a tolerance that follows the full residual
// ||b - (c_mass M + c_op A + c_op P) x_j|| / ||b||, until that is at most tol.
// The steps contract by ||K^-1 c_op (P - rho_bar M)||.
static t2s2_status prod_solve(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                              double tol, int rmax, int max_sweeps, t2s2_solve_info* info) {
  constexpr int kMaxOuter = 60;
  const int d = op->d;
  const int rcap = rmax + amen_kick();
  const double shift = c_op * op->rho_bar;
  DevTT x;
  int rx[T2S2_MAX_D + 1];
  for (int k = 0; k <= d; ++k) rx[k] = std::min(xio.r[k], rcap);
  rx[0] = rx[d] = 1;
  T2S2_TRY(tt_alloc(cx, x, d, op->m, rx, rcap));
  {
    const size_t mk = cx.ar->mark();
    DevTT t;
    T2S2_TRY(tt_alloc(cx, t, d, op->m, xio.r, 0));
    T2S2_TRY(tt_copy(cx, xio, t));
    T2S2_TRY(tt_round(cx, t, 0.0, rcap));
    T2S2_TRY(tt_copy(cx, t, x));
    cx.ar->release(mk);
  }
  const char* ev = std::getenv("T2S2_VERBOSE");
  const bool verbose = ev && ev[0] == '1';
  double bn = 0.0;
  T2S2_TRY(tt_norm(cx, b, &bn));
  double res = 0.0;
  int sweeps = 0, outer = 0;
  for (;;) {
    const size_t mk = cx.ar->mark();
    T2S2_TRY(residual_full(op, cx, b, x, c_mass, c_op, &res));
    if (verbose) {
      fprintf(stderr, "[t2s2] lagged-reaction step %d: full residual %.3e, sweeps %d, ranks", outer, res, sweeps);
      for (int k = 0; k <= d; ++k) fprintf(stderr, " %d", x.r[k]);
      fprintf(stderr, "\n");
    }
    if (res <= tol || outer >= kMaxOuter || sweeps >= max_sweeps) {
      cx.ar->release(mk);
      break;
    }
    // rhs = b - c_op (P x - rho_bar M x)
    DevTT px, mx, lag, rhs;
    T2S2_TRY(apply_kron(cx, x, op->dP, px));
    T2S2_TRY(apply_kron(cx, x, op->dRt, mx));
    T2S2_TRY(tt_axpby(cx, c_op, px, -shift, mx, lag));
    const double tin = std::max(0.3 * tol, 0.05 * res);
    int rsum = 1, rbmax = 1;
    for (int k = 0; k <= d; ++k) {
      rsum = std::max(rsum, b.r[k] + lag.r[k]);
      rbmax = std::max(rbmax, b.r[k]);
    }
    if (rsum > kSmallMax) {
      // the sum would exceed the orthogonalisation's rank limit: compress the
      // lagged term first, its error measured against |b|
      double ln = 0.0;
      T2S2_TRY(tt_norm(cx, lag, &ln));
      T2S2_TRY(tt_round(cx, lag, ln > 0.0 ? 1e-3 * tin * bn / ln : 0.0, kSmallMax - rbmax));
    }
    T2S2_TRY(tt_axpby(cx, 1.0, b, -1.0, lag, rhs));
    T2S2_TRY(tt_round(cx, rhs, 0.01 * tin, kSmallMax));
    t2s2_solve_info ii{};
    const t2s2_status st = solve_impl(op, cx, rhs, x, c_mass + shift, c_op, tin, rmax, max_sweeps - sweeps,
                                      T2S2_FP64, &ii);
    if (st != T2S2_OK && st != T2S2_ENOCONV) return st;
    sweeps += std::max(1, ii.sweeps);
    cx.ar->release(mk);
    ++outer;
  }
  for (int k = 0; k < d; ++k)
    if (x.core_elems(k) > xio.cap[k]) return T2S2_ENOMEM;
  T2S2_TRY(tt_copy(cx, x, xio));
  if (info) {
    info->residual = res;
    info->sweeps = sweeps;
    int mr = 1;
    for (int k = 0; k <= d; ++k) mr = std::max(mr, x.r[k]);
    info->max_rank = mr;
    info->refinements = outer;
    info->local_iters = 0;
  }
  return res <= tol ? T2S2_OK : T2S2_ENOCONV;
}

size_t solve_bytes(t2s2_op op, int rmax, int rfmax, t2s2_precision prec) {
  size_t need = Amen::bytes_needed(op->d, op->m, rmax + amen_kick(), rfmax, amen_kick(), 40);
  if (prec != T2S2_FP64) need += refine_extra_bytes(op, rmax + amen_kick(), rfmax);
  return need;
}

static t2s2_status solve_entry(t2s2_op op, const t2s2_tt* b, t2s2_tt* x, double c_mass, double c_op,
                               double tol, int rmax, int max_sweeps, t2s2_precision prec, void* stream,
                               t2s2_solve_info* info) {
  if (!op || !b || !x) return T2S2_EINVAL;
  if (!(tol > 0.0) || rmax < 1 || max_sweeps < 0) return T2S2_EINVAL;
  if (prec < T2S2_FP64 || prec > T2S2_BF16_REFINE) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, b));
  T2S2_TRY(check_tt(op, x));
  int rfmax = 1;
  for (int k = 0; k <= op->d; ++k) rfmax = std::max(rfmax, b->r[k]);
  size_t need = Amen::bytes_needed(op->d, op->m, rmax + amen_kick(), rfmax, amen_kick(), 40) + 2 * (tt_bytes(b) + tt_bytes(x));
  if (prec != T2S2_FP64) need += refine_extra_bytes(op, rmax + amen_kick(), rfmax);
  if (op->has_prod) {
    if (prec != T2S2_FP64) return T2S2_ENOTIMPL;
    // the lagged term P x - rho_bar M x (ranks 2 rcap) is rounded as one train
    if (2 * (rmax + amen_kick()) > kSmallMax) return T2S2_EINVAL;
    // the full operator's product and residual trains (ranks up to
    // r_b + 3 rcap), their rounding temporaries, the correction and x + d
    size_t mm = 1;
    for (int k = 0; k < op->d; ++k) mm = std::max<size_t>(mm, op->m[k]);
    const size_t r3 = (size_t)rfmax + 3 * (size_t)(rmax + amen_kick());
    need += 12 * (size_t)op->d * r3 * r3 * mm * sizeof(double);
  }
  T2S2_TRY(ensure_arena(op, need));
  Ctx cx = make_ctx(op, stream);
  DevTT db, dx;
  T2S2_TRY(bind_tt(cx, b, db, true));
  T2S2_TRY(bind_tt(cx, x, dx, true));
  t2s2_status st = op->has_prod ? prod_solve(op, cx, db, dx, c_mass, c_op, tol, rmax, max_sweeps, info)
                                : solve_impl(op, cx, db, dx, c_mass, c_op, tol, rmax, max_sweeps, prec, info);
  if (st != T2S2_OK && st != T2S2_ENOCONV) return st;
  t2s2_status st2 = unbind_tt(cx, dx, x);
  return st2 != T2S2_OK ? st2 : st;
}

static t2s2_status step_entry(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax, bool cn,
                              t2s2_precision prec, void* stream, t2s2_solve_info* info) {
  if (!op || !u || !(dt > 0.0) || !(tol > 0.0) || rmax < 1) return T2S2_EINVAL;
  if (op->has_prod) return T2S2_ENOTIMPL;
  T2S2_TRY(check_tt(op, u));
  const int d = op->d;
  size_t need = Amen::bytes_needed(d, op->m, rmax + amen_kick(), 2 * (rmax + amen_kick()), amen_kick(), 40) + 8 * tt_bytes(u);
  if (prec != T2S2_FP64) need += refine_extra_bytes(op, rmax + amen_kick(), 2 * (rmax + amen_kick()));
  T2S2_TRY(ensure_arena(op, need));
  Ctx cx = make_ctx(op, stream);
  DevTT du;
  T2S2_TRY(bind_tt(cx, u, du, true));
  // rhs = rndg((M - dt/2 A) u)  (CN)  or  rndg(M u)  (BE)
  int r2[T2S2_MAX_D + 1];
  for (int k = 0; k <= d; ++k) r2[k] = (k == 0 || k == d) ? 1 : 2 * du.r[k];
  DevTT rhs;
  T2S2_TRY(tt_alloc(cx, rhs, d, du.m, r2, 0));
  T2S2_TRY(apply_op(op, cx, du, rhs, 1.0, cn ? -0.5 * dt : 0.0, false));
  T2S2_TRY(tt_round(cx, rhs, tol, rmax));
  const double co = cn ? 0.5 * dt : dt;
  // a time step starts from the previous step, already close: a small kick
  // keeps the ranks (and the cost of every later step) down
  cx.kick = std::min(kStepKick, amen_kick());
  t2s2_status st = solve_impl(op, cx, rhs, du, 1.0, co, tol, rmax, 20, prec, info);
  if (st != T2S2_OK && st != T2S2_ENOCONV) return st;
  t2s2_status st2 = unbind_tt(cx, du, u);
  return st2 != T2S2_OK ? st2 : st;
}

// Batched steady solves: `count` independent instances, each with its own
// operator (and so its own workspace).  Worker threads take instances from a
// shared counter; each worker owns a CUDA stream, and every instance's
// cooperative local solves are limited to kNumSMs / workers CTAs so that the
// workers' teams fit on the GPU side by side.
static t2s2_status solve_batched_entry(const t2s2_op* ops, const t2s2_tt* b, t2s2_tt* x, int count,
                                       double tol, int rmax, int max_sweeps, t2s2_precision prec,
                                       int workers, t2s2_solve_info* infos, t2s2_status* statuses) {
  if (!ops || !b || !x || count < 0 || !statuses) return T2S2_EINVAL;
  if (count == 0) return T2S2_OK;
  for (int i = 0; i < count; ++i) {
    if (!ops[i]) return T2S2_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return T2S2_EINVAL;  // instances may not share a workspace
  }
  if (workers <= 0) workers = 8;
  workers = std::min(workers, count);
  int dev = 0;
  T2S2_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<cudaStream_t> streams(workers);
  for (auto& s : streams) T2S2_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const int team = std::max(1, kNumSMs / workers);
  std::atomic<int> next{0};
  auto work = [&](int w) {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      const int saved = ops[i]->team;
      ops[i]->team = team;
      statuses[i] = solve_entry(ops[i], &b[i], &x[i], 0.0, 1.0, tol, rmax, max_sweeps, prec, streams[w],
                                infos ? &infos[i] : nullptr);
      ops[i]->team = saved;
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < workers; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  for (auto& s : streams) cudaStreamDestroy(s);
  for (int i = 0; i < count; ++i)
    if (statuses[i] != T2S2_OK && statuses[i] != T2S2_ENOCONV) return statuses[i];
  for (int i = 0; i < count; ++i)
    if (statuses[i] == T2S2_ENOCONV) return T2S2_ENOCONV;
  return T2S2_OK;
}

}  // namespace t2s2

using namespace t2s2;

extern "C" {
t2s2_status t2s2_solve_batched(const t2s2_op* ops, const t2s2_tt* b, t2s2_tt* x, int count, double tol,
                               int rmax, int max_sweeps, t2s2_precision prec, int workers,
                               t2s2_solve_info* infos, t2s2_status* statuses) {
  return solve_batched_entry(ops, b, x, count, tol, rmax, max_sweeps, prec, workers, infos, statuses);
}

t2s2_status t2s2_solve(t2s2_op op, const t2s2_tt* b, t2s2_tt* x, double c_mass, double c_op,
                       double tol, int rmax, int max_sweeps, t2s2_precision prec, void* stream,
                       t2s2_solve_info* info) {
  return solve_entry(op, b, x, c_mass, c_op, tol, rmax, max_sweeps, prec, stream, info);
}
t2s2_status t2s2_cn_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info) {
  return step_entry(op, u, dt, tol, rmax, true, prec, stream, info);
}
t2s2_status t2s2_be_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info) {
  return step_entry(op, u, dt, tol, rmax, false, prec, stream, info);
}
}
