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

#include "local.h"
#include "trace.h"

namespace cg = cooperative_groups;

namespace t2s2 {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;

template <typename T>
struct Ops;
template <>
struct Ops<double> {
  static __device__ double ld(const double* p) { return __ldg(p); }
};
template <>
struct Ops<float> {
  static __device__ float ld(const float* p) { return __ldg(p); }
};

// block-wide sum of nv values per thread (vals[0..nv-1]) into smem red[nv][NW]
__device__ void block_sum(double* vals, int nv, double* red) {
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  for (int v = 0; v < nv; ++v) {
    double s = vals[v];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[v * NW + w] = s;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0;
    for (int i = 0; i < NW; ++i) s += red[threadIdx.x * NW + i];
    vals[threadIdx.x] = s;  // only valid in thread v for value v
    red[threadIdx.x * NW] = s;
  }
  __syncthreads();
}

template <typename T>
struct Team {
  LocalProblem<T> P;
  long N;
  int G, g;
  long e0, e1;
  cg::grid_group grid;
  __device__ Team(const LocalProblem<T>& p) : P(p), grid(cg::this_grid()) {
    N = (long)P.ra * P.m * P.rb;
    G = gridDim.x;
    g = blockIdx.x;
    long chunk = (N + G - 1) / G;
    e0 = min(N, (long)g * chunk);
    e1 = min(N, e0 + chunk);
  }
  __device__ void sync() { grid.sync(); }

  // y = K x on this CTA's elements (x complete in global memory)
  __device__ void matvec(const T* __restrict__ x, T* __restrict__ y) {
    const int ra = P.ra, m = P.m, rb = P.rb;
    for (long e = e0 + threadIdx.x; e < e1; e += NT) {
      int b = (int)(e % rb);
      long t = e / rb;
      int i = (int)(t % m);
      int a = (int)(t / m);
      double s = 0.0;
      const double* pl = P.PL + (long)a * ra;
      for (int p = 0; p < ra; ++p) s += pl[p] * (double)Ops<T>::ld(x + ((long)p * m + i) * rb + b);
      const double* bp = P.Bp + (long)i * m;
      const T* xa = x + (long)a * m * rb + b;
      for (int j = 0; j < m; ++j) s += bp[j] * (double)Ops<T>::ld(xa + (long)j * rb);
      const double* pr = P.PR + (long)b * rb;
      const T* xi = x + ((long)a * m + i) * rb;
      for (int q = 0; q < rb; ++q) s += pr[q] * (double)Ops<T>::ld(xi + q);
      y[e] = (T)s;
    }
  }

  // z = M^{-1} v over fibres (warp per fibre); v complete in global memory
  __device__ void precond(const T* __restrict__ v, T* __restrict__ z, T* sm_re, T* sm_im) {
    const int ra = P.ra, m = P.m, rb = P.rb;
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const long nf = (long)ra * rb;
    T* vr = sm_re + w * kLocalMaxM;  // per-warp scratch (length m)
    T* vi = sm_im + w * kLocalMaxM;
    const T* Zr = P.Zr;
    const T* Zi = P.Zi;
    const T* Tr = P.Tr;
    const T* Ti = P.Ti;
    const T cop = (T)P.c_op;
    for (long f = (long)g * NW + w; f < nf; f += (long)G * NW) {
      const int a = (int)(f / rb), b = (int)(f % rb);
      const T sig = (T)(P.PL[(long)a * ra + a] + P.PR[(long)b * rb + b] + P.shift);
      const T* vf = v + (long)a * m * rb + b;
      // vt = Z^H v : vt_i = sum_j conj(Z_ji) v_j
      for (int i = lane; i < m; i += 32) {
        T sr = 0, si = 0;
        for (int j = 0; j < m; ++j) {
          T vj = Ops<T>::ld(vf + (long)j * rb);
          sr += Ops<T>::ld(Zr + (long)j * m + i) * vj;
          si -= Ops<T>::ld(Zi + (long)j * m + i) * vj;
        }
        vr[i] = sr;
        vi[i] = si;
      }
      __syncwarp();
      // back substitution with (c_op T + sig I), column oriented
      for (int i = m - 1; i >= 0; --i) {
        T yr = 0, yi = 0;
        if (lane == 0) {
          T dr = cop * Ops<T>::ld(Tr + (long)i * m + i) + sig;
          T di = cop * Ops<T>::ld(Ti + (long)i * m + i);
          T den = dr * dr + di * di;
          T nr = vr[i], ni = vi[i];
          yr = (nr * dr + ni * di) / den;
          yi = (ni * dr - nr * di) / den;
          vr[i] = yr;
          vi[i] = yi;
        }
        yr = __shfl_sync(0xffffffffu, yr, 0);
        yi = __shfl_sync(0xffffffffu, yi, 0);
        for (int j = lane; j < i; j += 32) {
          T tr = cop * Ops<T>::ld(Tr + (long)j * m + i), ti = cop * Ops<T>::ld(Ti + (long)j * m + i);
          vr[j] -= tr * yr - ti * yi;
          vi[j] -= tr * yi + ti * yr;
        }
        __syncwarp();
      }
      // z = Re(Z y)
      T* zf = z + (long)a * m * rb + b;
      for (int i = lane; i < m; i += 32) {
        T s = 0;
        for (int j = 0; j < m; ++j)
          s += Ops<T>::ld(Zr + (long)i * m + j) * vr[j] - Ops<T>::ld(Zi + (long)i * m + j) * vi[j];
        zf[(long)i * rb] = s;
      }
      __syncwarp();
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(NT) gmres_team_kernel(LocalProblem<T> P) {
  Team<T> tm(P);
  const int mr = P.mr;
  __shared__ double H[(kLocalMaxRestart + 1) * kLocalMaxRestart];
  __shared__ double cs[kLocalMaxRestart], sn[kLocalMaxRestart], gv[kLocalMaxRestart + 1],
      yv[kLocalMaxRestart];
  __shared__ double red[(kLocalMaxRestart + 2) * NW];
  __shared__ double hcol[kLocalMaxRestart + 2];
  __shared__ T pre_re[NW * kLocalMaxM], pre_im[NW * kLocalMaxM];
  const long N = tm.N;
  T* V = P.work;                       // (mr+1) x N
  T* Zv = V + (long)(mr + 1) * N;      // N
  T* Wv = Zv + N;                      // N
  double* part = P.part;               // 2 x G x (mr+2)
  const int G = tm.G, g = tm.g;
  const int stride = kLocalMaxRestart + 2;
  int pbuf = 0;
  auto partial = [&](int buf, int gi, int v) -> double& { return part[((long)buf * G + gi) * stride + v]; };
  auto team_sum = [&](int buf, int nv) {  // sums partials into hcol[0..nv-1]
    if (threadIdx.x < nv) {
      double s = 0;
      for (int gi = 0; gi < G; ++gi) s += partial(buf, gi, threadIdx.x);
      hcol[threadIdx.x] = s;
    }
    __syncthreads();
  };

  // ||rhs||
  {
    double v[1] = {0.0};
    for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
      double r = (double)P.rhs[e];
      v[0] += r * r;
    }
    block_sum(v, 1, red);
    if (threadIdx.x == 0) partial(pbuf, g, 0) = red[0];
  }
  tm.sync();
  team_sum(pbuf, 1);
  pbuf ^= 1;
  const double rhs_norm = sqrt(hcol[0]);
  const double tol_abs = P.tol_rel * rhs_norm;
  int its = 0;
  double resid = 0.0;
  bool done = false;
  for (int cycle = 0; !done; ++cycle) {
    // r = rhs - K x  -> Wv ; beta = ||r||
    tm.matvec(P.x, Wv);
    {
      double v[1] = {0.0};
      for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
        double r = (double)P.rhs[e] - (double)Wv[e];
        Wv[e] = (T)r;
        v[0] += r * r;
      }
      block_sum(v, 1, red);
      if (threadIdx.x == 0) partial(pbuf, g, 0) = red[0];
    }
    tm.sync();
    team_sum(pbuf, 1);
    pbuf ^= 1;
    const double beta = sqrt(hcol[0]);
    resid = beta;
    if (beta <= tol_abs || its >= P.maxit || beta == 0.0) break;
    for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) V[e] = (T)((double)Wv[e] / beta);
    if (threadIdx.x == 0) {
      gv[0] = beta;
      for (int i = 1; i <= mr; ++i) gv[i] = 0.0;
    }
    __syncthreads();
    tm.sync();
    int jend = 0;
    for (int j = 0; j < mr; ++j) {
      const T* vj = V + (long)j * N;
      tm.precond(vj, Zv, pre_re, pre_im);
      tm.sync();
      tm.matvec(Zv, Wv);
      // CGS pass 1: h_i = <w, v_i>, i <= j
      {
        double v[kLocalMaxRestart + 1];
        for (int i = 0; i <= j; ++i) v[i] = 0.0;
        for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
          double we = (double)Wv[e];
          for (int i = 0; i <= j; ++i) v[i] += we * (double)V[(long)i * N + e];
        }
        block_sum(v, j + 1, red);
        if (threadIdx.x <= j) partial(pbuf, g, threadIdx.x) = red[threadIdx.x * NW];
      }
      tm.sync();
      team_sum(pbuf, j + 1);
      pbuf ^= 1;
      if (threadIdx.x <= j) H[threadIdx.x * mr + j] = hcol[threadIdx.x];
      __syncthreads();
      // w -= V h ; CGS pass 2 dots
      {
        double v[kLocalMaxRestart + 1];
        for (int i = 0; i <= j; ++i) v[i] = 0.0;
        for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
          double we = (double)Wv[e];
          for (int i = 0; i <= j; ++i) we -= H[i * mr + j] * (double)V[(long)i * N + e];
          for (int i = 0; i <= j; ++i) v[i] += we * (double)V[(long)i * N + e];
          Wv[e] = (T)we;
        }
        block_sum(v, j + 1, red);
        if (threadIdx.x <= j) partial(pbuf, g, threadIdx.x) = red[threadIdx.x * NW];
      }
      tm.sync();
      team_sum(pbuf, j + 1);
      pbuf ^= 1;
      // w -= V h2 ; h += h2 ; ||w||^2
      {
        double v[1] = {0.0};
        for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
          double we = (double)Wv[e];
          for (int i = 0; i <= j; ++i) we -= hcol[i] * (double)V[(long)i * N + e];
          Wv[e] = (T)we;
          v[0] += we * we;
        }
        __syncthreads();
        if (threadIdx.x <= j) H[threadIdx.x * mr + j] += hcol[threadIdx.x];
        block_sum(v, 1, red);
        if (threadIdx.x == 0) partial(pbuf, g, 0) = red[0];
      }
      tm.sync();
      team_sum(pbuf, 1);
      pbuf ^= 1;
      const double hn = sqrt(hcol[0]);
      for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT)
        V[(long)(j + 1) * N + e] = (T)(hn > 0 ? (double)Wv[e] / hn : 0.0);
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
      ++its;
      jend = j + 1;
      resid = fabs(gv[j + 1]);
      if (resid <= tol_abs || its >= P.maxit || hn == 0.0) break;
      tm.sync();
    }
    // y = H^{-1} g ; u = V y -> Wv ; x += M^{-1} u
    if (threadIdx.x == 0) {
      for (int i = jend - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < jend; ++l) s -= H[i * mr + l] * yv[l];
        yv[i] = (H[i * mr + i] != 0.0) ? s / H[i * mr + i] : 0.0;
      }
    }
    __syncthreads();
    for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
      double s = 0.0;
      for (int i = 0; i < jend; ++i) s += yv[i] * (double)V[(long)i * N + e];
      Wv[e] = (T)s;
    }
    tm.sync();
    tm.precond(Wv, Zv, pre_re, pre_im);
    tm.sync();
    for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) P.x[e] = (T)((double)P.x[e] + (double)Zv[e]);
    tm.sync();
    if (its >= P.maxit) {
      // recompute the true residual once more for the report
      tm.matvec(P.x, Wv);
      double v[1] = {0.0};
      for (long e = tm.e0 + threadIdx.x; e < tm.e1; e += NT) {
        double r = (double)P.rhs[e] - (double)Wv[e];
        v[0] += r * r;
      }
      block_sum(v, 1, red);
      if (threadIdx.x == 0) partial(pbuf, g, 0) = red[0];
      tm.sync();
      team_sum(pbuf, 1);
      pbuf ^= 1;
      resid = sqrt(hcol[0]);
      done = true;
    }
  }
  if (g == 0 && threadIdx.x == 0) {
    if (P.iters_out) *P.iters_out = its;
    if (P.res_out) {
      P.res_out[0] = resid;
      P.res_out[1] = rhs_norm;
    }
  }
}

int g_team_blocks[2] = {0, 0};
}  // namespace

template <typename T>
size_t local_work_elems(long N, int mr) {
  return (size_t)(mr + 3) * N;
}

template <typename T>
t2s2_status local_gmres(const LocalProblem<T>& P, cudaStream_t st) {
  if (P.m > kLocalMaxM || P.mr > kLocalMaxRestart || P.mr < 1) return T2S2_EINVAL;
  const long N = (long)P.ra * P.m * P.rb;
  const int ti = sizeof(T) == 8 ? 0 : 1;
  if (g_team_blocks[ti] == 0) {
    int per_sm = 0;
    T2S2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gmres_team_kernel<T>, NT, 0));
    int dev = 0, sms = 0;
    T2S2_CUDA_TRY(cudaGetDevice(&dev));
    T2S2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g_team_blocks[ti] = std::max(1, per_sm) * sms;
  }
  long want = std::max((N + NT * 2 - 1) / (NT * 2), ((long)P.ra * P.rb + NW - 1) / NW);
  int G = (int)std::max(1L, std::min<long>(want, std::min(g_team_blocks[ti], kNumSMs)));
  if (P.team > 0) G = std::min(G, P.team);
  LocalProblem<T> Q = P;
  void* args[] = {&Q};
  {
    TraceScope ts(kTrLocal, st, 0.0, 0.0);
    T2S2_CUDA_TRY(cudaLaunchCooperativeKernel((void*)gmres_team_kernel<T>, dim3(G), dim3(NT), args, 0, st));
  }
  return T2S2_OK;
}

template size_t local_work_elems<double>(long, int);
template size_t local_work_elems<float>(long, int);
template t2s2_status local_gmres<double>(const LocalProblem<double>&, cudaStream_t);
template t2s2_status local_gmres<float>(const LocalProblem<float>&, cudaStream_t);

}  // namespace t2s2
