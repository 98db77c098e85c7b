// Local solves of the alternating TT solver, one kernel launch per solve.
//
// The local system at core k (Results, Fig. 6: "local problems at each TT
// core") is, for the operator written as a Kronecker sum K = sum_k I x B'_k x I
// and left/right interfaces taken in orthonormal frames,
//     (P_L (+) B'_k (+) P_R) X = F,   X of shape ra x m x rb,
//     [K X](a,i,b) = sum_p P_L(a,p) X(p,i,b) + sum_j B'(i,j) X(a,j,b) + sum_q P_R(b,q) X(a,i,q).
// It is solved by restarted GMRES with right preconditioning.  The
// preconditioner inverts, for every fibre (a,b), the 1D operator
// B' + (P_L(a,a) + P_R(b,b)) I exactly through the complex Schur form
// B = Z T Z^H computed once per operator (B' = c_op B + s I shares Z):
//     y = Z (c_op T + (s + sigma) I)^{-1} Z^H v,
// one warp per fibre with a column-oriented back substitution.
//
// All CTAs of the grid form one team (cooperative launch); phases are
// separated by grid-wide barriers; dot products reduce per CTA into a
// double-buffered partial array that every CTA then sums in the same order,
// so all CTAs hold identical Hessenberg / Givens data without a broadcast.
#include <cooperative_groups.h>

#include "eig.cuh"
#include "local.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int kRichardsonSteps = 3;  // before GMRES, with the exact preconditioner

// Vectors written during the kernel (basis, preconditioned vector, iterate)
// are read with coherent loads; only launch-constant data may use __ldg.
template <typename T>
struct Ops {
  static __device__ T ld(const T* p) { return *p; }
};

// Each CTA owns a contiguous range of fibres (a, b) and all m elements of
// each: the preconditioner then touches only the CTA's own data, and only the
// matrix-vector product needs the whole vector.
template <typename T>
struct Team {
  LocalProblem<T> P;
  long N, nf;
  int G, g;
  long f0, f1;   // owned fibres
  long nown;     // owned elements = (f1 - f0) * m
  cg::grid_group grid;
  __device__ Team(const LocalProblem<T>& p) : P(p), grid(cg::this_grid()) {
    N = (long)P.ra * P.m * P.rb;
    nf = (long)P.ra * P.rb;
    G = gridDim.x;
    g = blockIdx.x;
    long chunk = (nf + G - 1) / G;
    f0 = min(nf, (long)g * chunk);
    f1 = min(nf, f0 + chunk);
    nown = (f1 - f0) * P.m;
  }
  __device__ void sync() { grid.sync(); }
  // global element index of the k-th owned element (fibre fastest: coalesced in b)
  __device__ long elem(long k) const {
    const long nfl = f1 - f0;
    const long f = f0 + k % nfl;
    const int i = (int)(k / nfl);
    const long a = f / P.rb, b = f % P.rb;
    return (a * P.m + i) * P.rb + b;
  }

  // y = K x on this CTA's elements (x complete in global memory)
  __device__ void matvec(const T* __restrict__ x, T* __restrict__ y) {
    const int ra = P.ra, m = P.m, rb = P.rb;
    for (long k = threadIdx.x; k < nown; k += NT) {
      const long e = elem(k);
      int b = (int)(e % rb);
      long t = e / rb;
      int i = (int)(t % m);
      int a = (int)(t / m);
      // three independent accumulation chains (FP64 latency is long on this part)
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      const double* pl = P.PL + (long)a * ra;
      for (int p = 0; p < ra; ++p) s0 = fma(pl[p], (double)Ops<T>::ld(x + ((long)p * m + i) * rb + b), s0);
      const double* bp = P.Bp + (long)i * m;
      const T* xa = x + (long)a * m * rb + b;
      for (int j = 0; j < m; ++j) s1 = fma(bp[j], (double)Ops<T>::ld(xa + (long)j * rb), s1);
      const double* pr = P.PR + (long)b * rb;
      const T* xi = x + ((long)a * m + i) * rb;
      for (int q = 0; q < rb; ++q) s2 = fma(pr[q], (double)Ops<T>::ld(xi + q), s2);
      y[e] = (T)(s0 + s1 + s2);
    }
  }

  // z = M^{-1} v over the CTA's own fibres (warp per fibre), arithmetic in
  // binary32: the preconditioner only steers the Krylov space (flexible GMRES
  // keeps every z_j), so its precision does not limit the solution's accuracy,
  // while binary32 runs the m-step triangular recurrences at full SIMT speed.
  // Ttr/Tti: (c_op T)^T, Zr/Zi: Z, row stride ld.  scratch: per-warp 5 * kLocalMaxM floats.
  __device__ void precond(const T* __restrict__ v, T* __restrict__ z, const float* Ttr,
                          const float* Tti, const float* Zr, const float* Zi, int ld, float* scratch) {
    const int ra = P.ra, m = P.m, rb = P.rb;
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    float* sv = scratch + w * 5 * kLocalMaxM;  // fibre input
    float* yr = sv + kLocalMaxM;               // solution of the triangular system
    float* yi = yr + kLocalMaxM;
    float* idr = yi + kLocalMaxM;              // reciprocal diagonal
    float* idi = idr + kLocalMaxM;
    for (long f = f0 + w; f < f1; f += NW) {
      const int a = (int)(f / rb), b = (int)(f % rb);
      const float sig = (float)(P.PL[(long)a * ra + a] + P.PR[(long)b * rb + b] + P.shift);
      const T* vf = v + (long)a * m * rb + b;
      for (int i = lane; i < m; i += 32) {
        sv[i] = (float)vf[(long)i * rb];
        float dr = Ttr[(long)i * ld + i] + sig, di = Tti[(long)i * ld + i];
        float den = __frcp_rn(dr * dr + di * di);
        idr[i] = dr * den;
        idi[i] = -di * den;
      }
      __syncwarp();
      // vt = Z^H v, lane-owned entries i = lane + 32 s
      float vr[4], vi[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        float sr = 0.f, si = 0.f;
        if (i < m) {
          for (int j = 0; j < m; ++j) {
            const float vj = sv[j];
            sr = fmaf(Zr[(long)j * ld + i], vj, sr);
            si = fmaf(-Zi[(long)j * ld + i], vj, si);
          }
        }
        vr[s] = sr;
        vi[s] = si;
      }
      // column-oriented back substitution with (c_op T + sig I)
      for (int i = m - 1; i >= 0; --i) {
        const int owner = i & 31, si_ = i >> 5;
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (s == si_) { ar = vr[s]; ai = vi[s]; }
        float cr = ar * idr[i] - ai * idi[i];
        float ci = ar * idi[i] + ai * idr[i];
        cr = __shfl_sync(0xffffffffu, cr, owner);
        ci = __shfl_sync(0xffffffffu, ci, owner);
        const float* tcr = Ttr + (long)i * ld;  // column i of c_op T = row i of its transpose
        const float* tci = Tti + (long)i * ld;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int j = lane + 32 * s;
          if (s == si_ && lane == owner) {
            vr[s] = cr;
            vi[s] = ci;
          } else if (j < i) {
            const float tr = tcr[j], ti = tci[j];
            vr[s] -= tr * cr - ti * ci;
            vi[s] -= tr * ci + ti * cr;
          }
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        if (i < m) {
          yr[i] = vr[s];
          yi[i] = vi[s];
        }
      }
      __syncwarp();
      // z = Re(Z y)
      T* zf = z + (long)a * m * rb + b;
      for (int i = lane; i < m; i += 32) {
        float acc0 = 0.f, acc1 = 0.f;
        const float* zr = Zr + (long)i * ld;
        const float* zi = Zi + (long)i * ld;
        for (int j = 0; j < m; ++j) {
          acc0 = fmaf(zr[j], yr[j], acc0);
          acc1 = fmaf(-zi[j], yi[j], acc1);
        }
        zf[(long)i * rb] = (T)(acc0 + acc1);
      }
      __syncwarp();
    }
  }
};

// Exact Kronecker-sum preconditioner (used when the interface eigendecompositions
// P_L = V_L diag(lL) V_L^{-1}, P_R = V_R diag(lR) V_R^{-1} are available):
//   K^{-1} = (V_L x Z x V_R) (lL (+) (c_op T + s I) (+) lR)^{-1} (V_L^{-1} x Z^H x V_R^{-1}),
// whose middle factor is, fibre by fibre, an upper-triangular solve with the
// complex shift lL[a'] + lR[b'].  Complex binary32.
struct FlsSmem {
  cf *VL, *VLi, *VR, *VRi, *lamL, *lamR, *Wst;  // eigen data and the m x max(ra,rb) staging slab
  float* fib;                                  // per-warp fibre scratch, 8 * kLocalMaxM floats
};

// Phase A: Y[a',i,b'] over the CTA's own fibres, reading the whole vector v.
template <typename T>
__device__ void fls_phase_a(const Team<T>& tm, const T* __restrict__ v, cf* __restrict__ Y, const FlsSmem& F,
                            const float* Ttr, const float* Tti, const float* Zr, const float* Zi, int ld) {
  const int ra = tm.P.ra, m = tm.P.m, rb = tm.P.rb;
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const float shift = (float)tm.P.shift;
  if (tm.f1 <= tm.f0) return;
  const int a_lo = (int)(tm.f0 / rb), a_hi = (int)((tm.f1 - 1) / rb);
  float* sr = F.fib + w * 8 * kLocalMaxM;
  float* si = sr + kLocalMaxM;
  float* yr = si + kLocalMaxM;
  float* yi = yr + kLocalMaxM;
  for (int ap = a_lo; ap <= a_hi; ++ap) {
    // W[i][b] = sum_a VLi[ap][a] v[a,i,b]
    for (int idx = threadIdx.x; idx < m * rb; idx += NT) {
      const int i = idx / rb, b = idx % rb;
      float xr = 0.f, xi = 0.f;
      for (int a = 0; a < ra; ++a) {
        const cf c = F.VLi[ap * ra + a];
        const float vv = (float)v[((long)a * m + i) * rb + b];
        xr = fmaf(c.x, vv, xr);
        xi = fmaf(c.y, vv, xi);
      }
      F.Wst[idx] = cmk(xr, xi);
    }
    __syncthreads();
    const long fb0 = max(tm.f0, (long)ap * rb), fb1 = min(tm.f1, (long)(ap + 1) * rb);
    for (long f = fb0 + w; f < fb1; f += NW) {
      const int bp = (int)(f - (long)ap * rb);
      // vt_i = sum_b VRi[bp][b] W[i][b]
      for (int i = lane; i < m; i += 32) {
        cf acc = cmk(0.f, 0.f);
        for (int b = 0; b < rb; ++b) acc = cadd(acc, cmul(F.VRi[bp * rb + b], F.Wst[i * rb + b]));
        sr[i] = acc.x;
        si[i] = acc.y;
      }
      __syncwarp();
      // Z^H vt
      float vr[4], vi[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        float ar = 0.f, ai = 0.f;
        if (i < m) {
          for (int j = 0; j < m; ++j) {
            const float zr = Zr[(long)j * ld + i], zi = Zi[(long)j * ld + i];  // conj(Z_ji)
            ar = fmaf(zr, sr[j], fmaf(zi, si[j], ar));
            ai = fmaf(zr, si[j], fmaf(-zi, sr[j], ai));
          }
        }
        vr[s] = ar;
        vi[s] = ai;
      }
      const cf sh = cadd(cadd(F.lamL[ap], F.lamR[bp]), cmk(shift, 0.f));
      // back substitution with (c_op T + shift I + lL + lR), column oriented
      for (int i = m - 1; i >= 0; --i) {
        const int owner = i & 31, si_ = i >> 5;
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (s == si_) { ar = vr[s]; ai = vi[s]; }
        const cf dg = cadd(cmk(Ttr[(long)i * ld + i], Tti[(long)i * ld + i]), sh);
        const cf q = cdiv(cmk(ar, ai), dg);
        const float cr = __shfl_sync(0xffffffffu, q.x, owner);
        const float ci = __shfl_sync(0xffffffffu, q.y, owner);
        const float* tcr = Ttr + (long)i * ld;
        const float* tci = Tti + (long)i * ld;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int j = lane + 32 * s;
          if (s == si_ && lane == owner) {
            vr[s] = cr;
            vi[s] = ci;
          } else if (j < i) {
            const float tr = tcr[j], ti = tci[j];
            vr[s] -= tr * cr - ti * ci;
            vi[s] -= tr * ci + ti * cr;
          }
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        if (i < m) {
          yr[i] = vr[s];
          yi[i] = vi[s];
        }
      }
      __syncwarp();
      // Y = Z y
      for (int i = lane; i < m; i += 32) {
        float ar = 0.f, ai = 0.f;
        const float* zr = Zr + (long)i * ld;
        const float* zi = Zi + (long)i * ld;
        for (int j = 0; j < m; ++j) {
          ar = fmaf(zr[j], yr[j], fmaf(-zi[j], yi[j], ar));
          ai = fmaf(zr[j], yi[j], fmaf(zi[j], yr[j], ai));
        }
        Y[((long)ap * m + i) * rb + bp] = cmk(ar, ai);
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

// Phase B: z[a,i,b] = Re sum_{a',b'} VL[a][a'] VR[b][b'] Y[a',i,b'] on own fibres (Y complete).
template <typename T>
__device__ void fls_phase_b(const Team<T>& tm, const cf* __restrict__ Y, T* __restrict__ z, const FlsSmem& F) {
  const int ra = tm.P.ra, m = tm.P.m, rb = tm.P.rb;
  if (tm.f1 <= tm.f0) return;
  const int a_lo = (int)(tm.f0 / rb), a_hi = (int)((tm.f1 - 1) / rb);
  for (int a = a_lo; a <= a_hi; ++a) {
    for (int idx = threadIdx.x; idx < m * rb; idx += NT) {
      const int i = idx / rb, bp = idx % rb;
      cf acc = cmk(0.f, 0.f);
      for (int ap = 0; ap < ra; ++ap) acc = cadd(acc, cmul(F.VL[a * ra + ap], Y[((long)ap * m + i) * rb + bp]));
      F.Wst[idx] = acc;
    }
    __syncthreads();
    const long fb0 = max(tm.f0, (long)a * rb), fb1 = min(tm.f1, (long)(a + 1) * rb);
    const int nb = (int)(fb1 - fb0);
    for (int idx = threadIdx.x; idx < nb * m; idx += NT) {
      const int b = (int)(fb0 - (long)a * rb) + idx % nb, i = idx / nb;
      float acc = 0.f;
      for (int bp = 0; bp < rb; ++bp) {
        const cf c = F.VR[b * rb + bp], wv = F.Wst[i * rb + bp];
        acc = fmaf(c.x, wv.x, fmaf(-c.y, wv.y, acc));
      }
      z[((long)a * m + i) * rb + b] = (T)acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__global__ void __launch_bounds__(NT) gmres_team_kernel(LocalProblem<T> P) {
  pdl_trigger();
  if (P.skip && *P.skip == 0) return;  // solved already (every CTA reads the same word)
  Team<T> tm(P);
  // optional phase timestamps (CTA 0, thread 0): slot 0 start, then 8 per
  // iteration for the first kLocalTimingIts iterations
  unsigned long long* tsb = (P.tstamp && blockIdx.x == 0 && threadIdx.x == 0) ? P.tstamp : nullptr;
  int tsi = 0;
  auto stamp = [&]() {
    if (tsb && tsi < 2 + 8 * kLocalTimingIts) tsb[tsi++] = gtimer();
  };
  stamp();
  const int mr = P.mr;
  __shared__ double H[(kLocalMaxRestart + 1) * kLocalMaxRestart];
  __shared__ double cs[kLocalMaxRestart], sn[kLocalMaxRestart], gv[kLocalMaxRestart + 1],
      yv[kLocalMaxRestart];
  __shared__ double hcol[kLocalMaxRestart + 2];
  __shared__ double dots[kLocalMaxRestart + 2];
  __shared__ double red2[(kLocalMaxRestart + 2) * 8];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* scratch = reinterpret_cast<float*>(dyn_smem);  // NW * 8 * kLocalMaxM, either preconditioner
  int* eidx = reinterpret_cast<int*>(scratch + NW * 8 * kLocalMaxM);  // own element indices
  const float *Ttr, *Tti, *Zr, *Zi;
  int ld;
  const bool own_in_smem = tm.nown <= P.own_cap;
  {
    const int m = P.m;
    float* after_idx = reinterpret_cast<float*>(eidx + P.own_cap);
    if (own_in_smem)
      for (long k = threadIdx.x; k < tm.nown; k += NT) eidx[k] = (int)tm.elem(k);
    if (P.smem_mats) {
      ld = m + 1;
      float* ttr = after_idx;
      float* tti = ttr + (long)m * ld;
      float* zr = tti + (long)m * ld;
      float* zi = zr + (long)m * ld;
      const float cop = (float)P.c_op;
      for (int e = threadIdx.x; e < m * m; e += NT) {
        const int i = e / m, j = e % m;
        ttr[(long)j * ld + i] = cop * P.Tr[e];  // transpose of c_op T
        tti[(long)j * ld + i] = cop * P.Ti[e];
        zr[(long)i * ld + j] = P.Zr[e];
        zi[(long)i * ld + j] = P.Zi[e];
      }
      Ttr = ttr; Tti = tti; Zr = zr; Zi = zi;
    } else {
      ld = m;
      Ttr = P.Ttc_r; Tti = P.Ttc_i; Zr = P.Zr; Zi = P.Zi;
    }
    __syncthreads();
  }
  // exact (FLS) preconditioner data, when both eigendecompositions succeeded
  FlsSmem F;
  const bool fls_on = P.fls && P.eig_status[0] == 0 && P.eig_status[1] == 0;
  if (fls_on) {
    const int ra = P.ra, rb = P.rb, m = P.m;
    float* base = reinterpret_cast<float*>(eidx + P.own_cap) + (P.smem_mats ? 4 * m * (m + 1) : 0);
    cf* c = reinterpret_cast<cf*>((reinterpret_cast<uintptr_t>(base) + 15) & ~(uintptr_t)15);
    F.lamL = c;
    F.VL = F.lamL + ra;
    F.VLi = F.VL + ra * ra;
    F.lamR = F.VLi + ra * ra;
    F.VR = F.lamR + rb;
    F.VRi = F.VR + rb * rb;
    F.Wst = F.VRi + rb * rb;
    F.fib = scratch;
    const cf* gl = reinterpret_cast<const cf*>(P.eigL);
    const cf* gr = reinterpret_cast<const cf*>(P.eigR);
    for (int e = threadIdx.x; e < ra + 2 * ra * ra; e += NT) F.lamL[e] = gl[e];
    for (int e = threadIdx.x; e < rb + 2 * rb * rb; e += NT) F.lamR[e] = gr[e];
    __syncthreads();
  }
  cf* Ybuf = reinterpret_cast<cf*>(P.ybuf);
  auto E = [&](long k) -> long { return own_in_smem ? (long)eidx[k] : tm.elem(k); };
  const long N = tm.N;
  T* V = P.work;                       // (mr+1) x N   Arnoldi basis
  T* Zs = V + (long)(mr + 1) * N;      // mr x N      preconditioned basis (flexible GMRES)
  T* Wv = Zs + (long)mr * N;           // N
  double* part = P.part;               // 2 x G x (kLocalMaxRestart + 2)
  const int G = tm.G, g = tm.g;
  const int stride = kLocalMaxRestart + 2;
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  int pbuf = 0;
  auto partial = [&](int buf, int gi, int v) -> double& { return part[((long)buf * G + gi) * stride + v]; };
  // CTA-local dot products over the own elements: dots[i] = <a, V_i> for i < nvec,
  // and dots[nvec] = <a, a> if with_norm; one warp per product, then published.
  auto own_dots = [&](const T* a, int nvec, bool with_norm) {
    const int nv = nvec + (with_norm ? 1 : 0);
    for (int v = wid; v < nv; v += NW) {
      const T* b = (v < nvec) ? V + (long)v * N : a;
      double s0 = 0.0, s1 = 0.0;
      long k = lane;
      for (; k + 32 < tm.nown; k += 64) {
        const long e0 = E(k), e1 = E(k + 32);
        s0 = fma((double)a[e0], (double)b[e0], s0);
        s1 = fma((double)a[e1], (double)b[e1], s1);
      }
      if (k < tm.nown) {
        const long e0 = E(k);
        s0 = fma((double)a[e0], (double)b[e0], s0);
      }
      double s = s0 + s1;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) partial(pbuf, g, v) = s;
    }
  };
  // After a grid barrier: hcol[v] = sum over CTAs of the published partials,
  // in a fixed order (bitwise identical in every CTA).
  auto gather = [&](int nv) {
    for (int idx = threadIdx.x; idx < nv * 8; idx += NT) {
      const int v = idx >> 3, sub = idx & 7;
      double s = 0.0;
      for (int gi = sub; gi < G; gi += 8) s += partial(pbuf, gi, v);
      red2[v * 8 + sub] = s;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
      const double* r = red2 + threadIdx.x * 8;
      hcol[threadIdx.x] = ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
    }
    __syncthreads();
    pbuf ^= 1;
  };

  // ||rhs||
  double rhs_norm = 0.0, tol_abs = 0.0;
  int its = 0;
  double resid = 0.0;
  bool done = false;
  if (fls_on) {
    // Preconditioned Richardson steps x <- x + M^{-1} r while each one cuts
    // the residual at least tenfold.  With the exact Kronecker-sum
    // preconditioner ||I - K M^{-1}|| is of the order of the binary32
    // eigendecompositions' accuracy, so one or two steps usually reach the
    // tolerance with no Arnoldi basis; otherwise GMRES continues from x.
    T* zr = Zs;  // scratch: the first preconditioned-basis slot
    double beta = -1.0;
    for (int step = 0; step <= kRichardsonSteps; ++step) {
      // r = rhs - K x -> Wv (own elements), ||r|| (and ||rhs|| at first)
      tm.matvec(P.x, Wv);
      for (long k = threadIdx.x; k < tm.nown; k += NT) {
        const long e = E(k);
        Wv[e] = (T)((double)P.rhs[e] - (double)Wv[e]);
      }
      __syncthreads();
      const int nv = (step == 0) ? 2 : 1;
      for (int v = wid; v < nv; v += NW) {
        const T* a = (v == 0) ? Wv : P.rhs;
        double s0 = 0.0, s1 = 0.0;
        long k = lane;
        for (; k + 32 < tm.nown; k += 64) {
          const long e0 = E(k), e1 = E(k + 32);
          s0 = fma((double)a[e0], (double)a[e0], s0);
          s1 = fma((double)a[e1], (double)a[e1], s1);
        }
        if (k < tm.nown) {
          const long e0 = E(k);
          s0 = fma((double)a[e0], (double)a[e0], s0);
        }
        double sv = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (lane == 0) partial(pbuf, g, v) = sv;
      }
      tm.sync();
      gather(nv);
      if (step == 0) {
        rhs_norm = sqrt(hcol[1]);
        tol_abs = P.tol_rel * rhs_norm;
      }
      const double bn = sqrt(hcol[0]);
      resid = bn;
      if (bn <= tol_abs || bn == 0.0) {
        done = true;
        break;
      }
      // the last step did not pay: hand the current x to GMRES
      if ((beta >= 0.0 && bn > 0.1 * beta) || step == kRichardsonSteps || its >= P.maxit) break;
      beta = bn;
      tm.sync();  // Wv complete for the preconditioner
      fls_phase_a(tm, Wv, Ybuf, F, Ttr, Tti, Zr, Zi, ld);
      tm.sync();  // Y complete
      fls_phase_b(tm, Ybuf, zr, F);
      for (long k = threadIdx.x; k < tm.nown; k += NT) {
        const long e = E(k);
        P.x[e] = (T)((double)P.x[e] + (double)zr[e]);
      }
      ++its;
      tm.sync();  // x complete before the next residual
    }
  }
  for (int cycle = 0; !done; ++cycle) {
    // r = rhs - K x -> Wv (own elements) ; beta = ||r||   (x complete); the
    // first cycle also takes ||rhs|| in the same reduction
    tm.matvec(P.x, Wv);
    for (long k = threadIdx.x; k < tm.nown; k += NT) {
      const long e = E(k);
      Wv[e] = (T)((double)P.rhs[e] - (double)Wv[e]);
    }
    __syncthreads();
    if (cycle == 0 && !fls_on) {
      for (int v = wid; v < 2; v += NW) {
        const T* a = (v == 0) ? Wv : P.rhs;
        double s0 = 0.0, s1 = 0.0;
        long k = lane;
        for (; k + 32 < tm.nown; k += 64) {
          const long e0 = E(k), e1 = E(k + 32);
          s0 = fma((double)a[e0], (double)a[e0], s0);
          s1 = fma((double)a[e1], (double)a[e1], s1);
        }
        if (k < tm.nown) {
          const long e0 = E(k);
          s0 = fma((double)a[e0], (double)a[e0], s0);
        }
        double sv = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (lane == 0) partial(pbuf, g, v) = sv;
      }
      tm.sync();
      gather(2);
      rhs_norm = sqrt(hcol[1]);
      tol_abs = P.tol_rel * rhs_norm;
    } else {
      own_dots(Wv, 0, true);
      tm.sync();
      gather(1);
    }
    const double beta = sqrt(hcol[0]);
    resid = beta;
    if (beta <= tol_abs || its >= P.maxit || beta == 0.0) break;
    const double binv = 1.0 / beta;
    for (long k = threadIdx.x; k < tm.nown; k += NT) {
      const long e = E(k);
      V[e] = (T)((double)Wv[e] * binv);
    }
    if (threadIdx.x == 0) {
      gv[0] = beta;
      for (int i = 1; i <= mr; ++i) gv[i] = 0.0;
    }
    __syncthreads();
    int jend = 0;
    for (int j = 0; j < mr; ++j) {
      const T* vj = V + (long)j * N;
      T* zj = Zs + (long)j * N;
      stamp();
      if (fls_on) {
        tm.sync();                                          // v_j complete
        fls_phase_a(tm, vj, Ybuf, F, Ttr, Tti, Zr, Zi, ld);
        tm.sync();                                          // Y complete
        fls_phase_b(tm, Ybuf, zj, F);
      } else {
        tm.precond(vj, zj, Ttr, Tti, Zr, Zi, ld, scratch);  // own fibres only
      }
      stamp();
      tm.sync();                                            // barrier 1: z_j complete
      stamp();
      tm.matvec(zj, Wv);
      __syncthreads();
      own_dots(Wv, j + 1, true);                            // h_i = <w, v_i>, and ||w||^2
      stamp();
      tm.sync();                                            // barrier 2
      gather(j + 2);
      stamp();
      double hsq = 0.0;
      for (int i = 0; i <= j; ++i) hsq += hcol[i] * hcol[i];
      const double ww = hcol[j + 1];
      if (threadIdx.x <= j) H[threadIdx.x * mr + j] = hcol[threadIdx.x];
      __syncthreads();
      double hn2 = ww - hsq;
      // w <- w - V h   (own elements)
      for (long k = threadIdx.x; k < tm.nown; k += NT) {
        const long e = E(k);
        double w0 = (double)Wv[e], w1 = 0.0;
        int i = 0;
        for (; i + 1 <= j; i += 2) {
          w0 = fma(-H[i * mr + j], (double)V[(long)i * N + e], w0);
          w1 = fma(-H[(i + 1) * mr + j], (double)V[(long)(i + 1) * N + e], w1);
        }
        if (i <= j) w0 = fma(-H[i * mr + j], (double)V[(long)i * N + e], w0);
        Wv[e] = (T)(w0 + w1);
      }
      __syncthreads();
      stamp();
      if (!(hn2 > 0.5 * ww)) {
        // severe cancellation: a second Gram-Schmidt pass (DGKS criterion)
        own_dots(Wv, j + 1, true);
        tm.sync();                                          // barrier 3 (rare)
        gather(j + 2);
        double h2 = 0.0;
        for (int i = 0; i <= j; ++i) h2 += hcol[i] * hcol[i];
        hn2 = hcol[j + 1] - h2;
        for (long k = threadIdx.x; k < tm.nown; k += NT) {
          const long e = E(k);
          double w0 = (double)Wv[e];
          for (int i = 0; i <= j; ++i) w0 = fma(-hcol[i], (double)V[(long)i * N + e], w0);
          Wv[e] = (T)w0;
        }
        __syncthreads();
        if (threadIdx.x <= j) H[threadIdx.x * mr + j] += hcol[threadIdx.x];
        __syncthreads();
      }
      stamp();
      const double hn = sqrt(fmax(hn2, 0.0));
      const double hinv = hn > 0 ? 1.0 / hn : 0.0;
      for (long k = threadIdx.x; k < tm.nown; k += NT) {
        const long e = E(k);
        V[(long)(j + 1) * N + e] = (T)((double)Wv[e] * hinv);
      }
      if (threadIdx.x == 0) {
        // apply previous rotations to column j, then a new one
        for (int i = 0; i < j; ++i) {
          double a = H[i * mr + j], b = H[(i + 1) * mr + j];
          H[i * mr + j] = cs[i] * a + sn[i] * b;
          H[(i + 1) * mr + j] = -sn[i] * a + cs[i] * b;
        }
        double a = H[j * mr + j], b = hn;
        double r = hypot(a, b);
        double c = (r > 0) ? a / r : 1.0, s = (r > 0) ? b / r : 0.0;
        cs[j] = c;
        sn[j] = s;
        H[j * mr + j] = r;
        gv[j + 1] = -s * gv[j];
        gv[j] = c * gv[j];
      }
      __syncthreads();
      stamp();
      stamp();
      ++its;
      jend = j + 1;
      resid = fabs(gv[j + 1]);
      if (resid <= tol_abs || its >= P.maxit || hn == 0.0) break;
    }
    // y = H^{-1} g ; x += Z y (own elements)
    if (threadIdx.x == 0) {
      for (int i = jend - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < jend; ++l) s -= H[i * mr + l] * yv[l];
        yv[i] = (H[i * mr + i] != 0.0) ? s / H[i * mr + i] : 0.0;
      }
    }
    __syncthreads();
    for (long k = threadIdx.x; k < tm.nown; k += NT) {
      const long e = E(k);
      double s0 = 0.0, s1 = 0.0;
      int i = 0;
      for (; i + 1 < jend; i += 2) {
        s0 = fma(yv[i], (double)Zs[(long)i * N + e], s0);
        s1 = fma(yv[i + 1], (double)Zs[(long)(i + 1) * N + e], s1);
      }
      if (i < jend) s0 = fma(yv[i], (double)Zs[(long)i * N + e], s0);
      P.x[e] = (T)((double)P.x[e] + s0 + s1);
    }
    tm.sync();  // x complete before the residual of the next cycle
  }
  if (g == 0 && threadIdx.x == 0) {
    if (P.iters_out) *P.iters_out = its;
    if (P.res_out) {
      P.res_out[0] = resid;
      P.res_out[1] = rhs_norm;
    }
  }
}

}  // namespace

// Eigendecompositions of the two interface matrices, one warp each; output
// layout per side: lam[r], V[r*r], Vinv[r*r] (complex binary32).
__global__ void local_eig_kernel(const double* PL, int ra, const double* PR, int rb, cf* outL, cf* outR,
                                 int* status, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (skip && *skip == 0) return;  // the local system is solved already
  extern __shared__ __align__(16) unsigned char esm[];
  const int w = threadIdx.x / 32;
  const int r = (w == 0) ? ra : rb;
  const double* A = (w == 0) ? PL : PR;
  cf* out = (w == 0) ? outL : outR;
  const size_t off = (w == 0) ? 0 : ((eig_smem_bytes(ra) + 15) & ~(size_t)15);
  EigSmem es = eig_smem(esm + off, r);
  const bool ok = warp_eig(A, r, r, es, out, out + r, r, out + r + (long)r * r, r);
  if ((threadIdx.x & 31) == 0) status[w] = ok ? 0 : 1;
}

template <typename T>
size_t local_work_elems(long N, int mr) {
  return (size_t)(2 * mr + 2) * N;
}

size_t local_smem_bytes(int m, bool mats, int own_cap, int ra = 0, int rb = 0, bool fls = false) {
  size_t s = (size_t)NW * 8 * kLocalMaxM * sizeof(float) + (size_t)own_cap * sizeof(int);
  if (mats) s += (size_t)4 * m * (m + 1) * sizeof(float);
  if (fls)
    s += sizeof(cf) * ((size_t)2 * ra * ra + (size_t)2 * rb * rb + ra + rb + (size_t)m * std::max(ra, rb)) + 64;
  return s;
}

template <typename T>
t2s2_status local_gmres(const LocalProblem<T>& P, cudaStream_t st) {
  if (P.m > kLocalMaxM || P.mr > kLocalMaxRestart || P.mr < 1) return T2S2_EINVAL;
  const long N = (long)P.ra * P.m * P.rb;
  const int ti = sizeof(T) == 8 ? 0 : 1;
  LocalProblem<T> Q = P;
  int dev0 = 0, sms0 = 0;
  T2S2_CUDA_TRY(cudaGetDevice(&dev0));
  T2S2_CUDA_TRY(cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0));
  // Team size: one CTA per fibre (the preconditioner gives each fibre a
  // warp, and fibres of one CTA that differ in a are done one after another)
  // and at least one element per thread, at most the GPU (or the caller's
  // share of it).  Every grid barrier and reduction costs more with more
  // CTAs, so a small local system gets a small team.
  const long nf = (long)P.ra * P.rb;
  int G_target = sms0;
  if (sizeof(T) == 8) G_target = (int)std::min<long>(sms0, std::max(nf, (N + NT - 1) / NT));
  else G_target = (int)std::min<long>(sms0, std::max((N + NT * 4 - 1) / (NT * 4), (nf + NW - 1) / NW));
  if (P.team > 0) G_target = std::min(G_target, P.team);
  G_target = std::max(1, G_target);
  {
    // own-element list sized for that team (a smaller, occupancy-limited
    // grid recomputes indices instead)
    const long per = ((nf + G_target - 1) / G_target) * P.m;
    Q.own_cap = (int)std::min<long>(per, kLocalOwnMax);
  }
  Q.smem_mats = local_smem_bytes(P.m, true, Q.own_cap) <= kLocalSmemCap;
  if (!Q.smem_mats && (!Q.Ttc_r || !Q.Ttc_i)) return T2S2_EINVAL;
  Q.fls = P.fls && Q.smem_mats && P.eigL && P.eigR && P.ybuf && P.eig_status && P.ra <= kEigMax &&
          P.rb <= kEigMax && local_smem_bytes(P.m, true, Q.own_cap, P.ra, P.rb, true) <= kLocalSmemCap;
  const size_t smem = local_smem_bytes(P.m, Q.smem_mats, Q.own_cap, P.ra, P.rb, Q.fls);
  if (Q.fls) {
    static bool eattr = false;
    const size_t esm = ((eig_smem_bytes(P.ra) + 15) & ~(size_t)15) + eig_smem_bytes(P.rb);
    if (!eattr) {
      T2S2_CUDA_TRY(cudaFuncSetAttribute(local_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * eig_smem_bytes(kEigMax) + 16)));
      eattr = true;
    }
    TraceScope ts(kTrSmall, st, 40.0 * ((double)P.ra * P.ra * P.ra + (double)P.rb * P.rb * P.rb), 0.0);
    (void)launch_pdl(local_eig_kernel, 1, 64, esm, st, P.PL, P.ra, P.PR, P.rb, reinterpret_cast<cf*>(P.eigL),
                                          reinterpret_cast<cf*>(P.eigR), P.eig_status, P.skip);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  static int attr_done[2] = {0, 0};
  if (!attr_done[ti]) {
    T2S2_CUDA_TRY(cudaFuncSetAttribute(gmres_team_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kLocalSmemCap));
    attr_done[ti] = 1;
  }
  int per_sm = 0;
  T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gmres_team_kernel<T>, NT, smem));
  int dev = 0, sms = 0;
  T2S2_CUDA_TRY(cudaGetDevice(&dev));
  T2S2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long resident = (long)std::max(1, per_sm) * sms;
  int G = (int)std::max(1L, std::min<long>(G_target, std::min<long>(resident, sms)));
  void* args[] = {&Q};
  {
    TraceScope ts(kTrLocal, st, 0.0, 0.0);
    T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((void*)gmres_team_kernel<T>, dim3(G), dim3(NT), args, smem, st));
  }
  return T2S2_OK;
}

double local_flops(int ra, int m, int rb, int its, int mr) {
  const double N = (double)ra * m * rb;
  const double jbar = 0.5 * std::min(its, mr) + 1.0;
  const double per_it = 2.0 * N * (ra + m + rb) + 12.0 * m * m * (double)ra * rb + 8.0 * N * jbar + 3.0 * N;
  const int restarts = its / std::max(1, mr) + 1;
  return per_it * its + restarts * (2.0 * N * (ra + m + rb) + 12.0 * m * m * (double)ra * rb + 4.0 * N);
}

template size_t local_work_elems<double>(long, int);
template size_t local_work_elems<float>(long, int);
template t2s2_status local_gmres<double>(const LocalProblem<double>&, cudaStream_t);
template t2s2_status local_gmres<float>(const LocalProblem<float>&, cudaStream_t);

}  // namespace t2s2
