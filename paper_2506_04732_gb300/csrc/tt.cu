// FP64 tensor-train arithmetic on the device.
//
// Orthogonalisation uses shifted CholeskyQR (Fukaya et al. 2020, with a
// second shifted pass for nearly rank-deficient blocks): two to four
// Gram / Cholesky / triangular-multiply passes whose heavy parts are GEMMs
// spread over all SMs, instead of a Householder QR that would serialise on
// one SM's FP64 pipe.  Truncation takes a one-sided Jacobi SVD of the small
// triangular factor.  Rounding follows the TT paper's rndg (Methods): right-to-
// left orthogonalisation, then left-to-right truncated SVDs with threshold
// tol ||x|| / sqrt(d-1) per unfolding.
#include "tt.h"
#include "trace.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace t2s2 {

namespace {

__global__ void k_scale_copy(double* dst, const double* src, size_t n, double alpha) {
  pdl_wait();
  pdl_trigger();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = alpha * src[e];
}
__global__ void k_axpy(double* dst, const double* src, size_t n, double beta) {
  pdl_wait();
  pdl_trigger();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] += beta * src[e];
}
__global__ void k_fill(double* dst, size_t n, double v) {
  pdl_wait();
  pdl_trigger();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = v;
}
__global__ void k_identity(double* dst, int n) {
  pdl_wait();
  pdl_trigger();
  size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (e / n == e % n) ? 1.0 : 0.0;
}
__global__ void k_sv_t(double* M, const double* s, const double* V, int r, int q, int ldv) {
  pdl_wait();
  pdl_trigger();
  int n = r * q;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int i = e / q, j = e % q;
    M[e] = s[i] * V[(size_t)j * ldv + i];
  }
}
__global__ void k_d2f(float* dst, const double* src, size_t n) {
  pdl_wait();
  pdl_trigger();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}
__global__ void k_f2d(double* dst, const float* src, size_t n) {
  pdl_wait();
  pdl_trigger();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}
// sum of squares, one block, fixed order per thread then tree (deterministic)
__global__ void k_sumsq(const double* v, size_t n, double* out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[1024];
  double s = 0.0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) s += v[e] * v[e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

inline int blocks_for(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 8 * kNumSMs)); }

}  // namespace

t2s2_status dev_scale_copy(Ctx& cx, double* dst, const double* src, size_t n, double alpha) {
  if (n == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 16.0 * n); (void)launch_pdl(k_scale_copy, blocks_for(n), 256, 0, cx.st, dst, src, n, alpha); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}
t2s2_status dev_axpy(Ctx& cx, double* dst, const double* src, size_t n, double beta) {
  if (n == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 24.0 * n); (void)launch_pdl(k_axpy, blocks_for(n), 256, 0, cx.st, dst, src, n, beta); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}
t2s2_status dev_fill(Ctx& cx, double* dst, size_t n, double v) {
  if (n == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 8.0 * n); (void)launch_pdl(k_fill, blocks_for(n), 256, 0, cx.st, dst, n, v); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}
t2s2_status dev_identity(Ctx& cx, double* dst, int n) {
  { TraceScope ts_(kTrElem, cx.st, 0.0, 8.0 * n * n); (void)launch_pdl(k_identity, blocks_for((size_t)n * n), 256, 0, cx.st, dst, n); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}
t2s2_status dev_sv_t(Ctx& cx, double* M, const double* s, const double* V, int r, int q, int ldv) {
  if (r * q == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 16.0 * r * q); (void)launch_pdl(k_sv_t, blocks_for((size_t)r * q), 256, 0, cx.st, M, s, V, r, q, ldv); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

t2s2_status dev_d2f(Ctx& cx, float* dst, const double* src, size_t n) {
  if (n == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 12.0 * n); (void)launch_pdl(k_d2f, blocks_for(n), 256, 0, cx.st, dst, src, n); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}
t2s2_status dev_f2d(Ctx& cx, double* dst, const float* src, size_t n) {
  if (n == 0) return T2S2_OK;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 12.0 * n); (void)launch_pdl(k_f2d, blocks_for(n), 256, 0, cx.st, dst, src, n); }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

t2s2_status core_norm(Ctx& cx, const double* v, size_t n, double* out) {
  size_t mk = cx.ar->mark();
  double* d = aget<double>(cx, 1);
  if (!d) return T2S2_ENOMEM;
  { TraceScope ts_(kTrElem, cx.st, 0.0, 8.0 * n); (void)launch_pdl(k_sumsq, 1, 1024, 0, cx.st, v, n, d); }
  T2S2_CUDA_TRY(cudaGetLastError());
  T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, d, sizeof(double), cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  *out = std::sqrt(cx.hbuf[0]);
  cx.ar->release(mk);
  return T2S2_OK;
}

int trunc_rank(const double* s, int n, double delta, int rmax) {
  // tail[j] = ||s[j:]||; smallest j >= 1 with tail[j] < delta (ties keep the larger rank)
  std::vector<double> tail(n + 1, 0.0);
  for (int j = n - 1; j >= 0; --j) tail[j] = std::sqrt(tail[j + 1] * tail[j + 1] + s[j] * s[j]);
  int r = n;
  for (int j = 1; j < n; ++j)
    if (tail[j] < delta * (1.0 - 1e-14)) { r = j; break; }
  if (rmax > 0) r = std::min(r, rmax);
  return std::max(r, 1);
}

static constexpr double kUnit = 1.1102230246251565e-16;

namespace {
__global__ void k_transpose(double* dst, const double* src, int r, int c) {
  pdl_wait();
  pdl_trigger();
  int n = r * c;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int i = e / c, j = e % c;
    dst[(size_t)j * r + i] = src[e];
  }
}
}  // namespace

// Fused single-launch CholeskyQR3 when its grid fits (cholqr.cu), else the
// pass-by-pass sequence below.
static bool qr_fused(Ctx& cx, const double* W, int nlong, int c, bool tall, double* Q, double* R,
                     t2s2_status* st, const double* W2 = nullptr, int c1 = 0) {
  int grid = 0, per = 0;
  size_t smem = 0;
  const double shift = 11.0 * ((double)nlong * c + (double)c * (c + 1)) * kUnit;
  if (cqr_cluster_plan(nlong, c, &grid, &per, &smem)) {
    *st = cqr_cluster(W, Q, R, nlong, c, tall, shift, cx.dstat, grid, per, smem, cx.st, W2, c1);
    return true;
  }
  if (!cholqr3_plan(nlong, c, cx.coop_ctas, &grid, &per, &smem)) return false;
  const size_t mk = cx.ar->mark();
  double* scratch = aget<double>(cx, cholqr3_scratch_doubles(nlong, c, grid));
  if (!scratch) {
    cx.ar->release(mk);
    return false;
  }
  *st = cholqr3_fused(W, Q, R, nlong, c, tall, shift, scratch, cx.dstat, grid, per, smem, cx.st, W2, c1);
  cx.ar->release(mk);
  return true;
}

bool qr_tall_async(Ctx& cx, const double* W, int rows, int cols, double* Q, double* R, cudaStream_t side,
                   t2s2_status* st) {
  int grid = 0, per = 0;
  size_t smem = 0;
  if (cols < 1 || cols > kSmallMax || rows < cols) return false;
  const double shift = 11.0 * ((double)rows * cols + (double)cols * (cols + 1)) * kUnit;
  if (cqr_cluster_plan(rows, cols, &grid, &per, &smem)) {
    *st = cqr_cluster(W, Q, R, rows, cols, true, shift, cx.dstat, grid, per, smem, side);
    return true;
  }
  if (!cholqr3_plan(rows, cols, cx.coop_ctas, &grid, &per, &smem)) return false;
  // held (not released) until the caller joins the side stream
  double* scratch = aget<double>(cx, cholqr3_scratch_doubles(rows, cols, grid));
  if (!scratch) return false;
  *st = cholqr3_fused(W, Q, R, rows, cols, true, shift, scratch, cx.dstat, grid, per, smem, side);
  return true;
}

t2s2_status qr_tall(Ctx& cx, const double* W, int rows, int cols, double* Q, double* R) {
  if (cols > kSmallMax || rows < cols || cols <= 0) return T2S2_EINVAL;
  {
    t2s2_status fs = T2S2_OK;
    if (qr_fused(cx, W, rows, cols, true, Q, R, &fs)) return fs;
  }
  size_t mk = cx.ar->mark();
  const int c = cols;
  double* G = aget<double>(cx, (size_t)c * c);
  double* L = aget<double>(cx, (size_t)c * c);
  double* Li = aget<double>(cx, (size_t)c * c);
  double* Lacc = aget<double>(cx, (size_t)c * c);
  double* Ltmp = aget<double>(cx, (size_t)c * c);
  double* T0 = aget<double>(cx, (size_t)rows * c);
  double* T1 = aget<double>(cx, (size_t)rows * c);
  if (!G || !L || !Li || !Lacc || !Ltmp || !T0 || !T1) return T2S2_ENOMEM;
  const double shift = 11.0 * ((double)rows * c + (double)c * (c + 1)) * kUnit;
  const double* cur = W;
  double* outs[kCqrMaxPass] = {T0, T1, T0, Q};
  for (int pass = 0; pass < kCqrMaxPass; ++pass) {
    T2S2_TRY(gemm_ex<double>(cx, c, c, rows, true, false, 1.0, cur, c, cur, c, 0.0, G, c));
    T2S2_TRY(chol_inv(G, c, pass < kCqrShiftedPasses ? shift : 0.0, L, Li, cx.dstat, cx.st));
    // cur = next * L^T  =>  next = cur * L^{-T}
    T2S2_TRY(gemm_ex<double>(cx, rows, c, c, false, true, 1.0, cur, c, Li, c, 0.0, outs[pass], c));
    if (pass == 0) {
      T2S2_CUDA_TRY(cudaMemcpyAsync(Lacc, L, sizeof(double) * c * c, cudaMemcpyDeviceToDevice, cx.st));
    } else {
      T2S2_TRY(gemm_ex<double>(cx, c, c, c, false, false, 1.0, Lacc, c, L, c, 0.0, Ltmp, c));
      std::swap(Lacc, Ltmp);
    }
    cur = outs[pass];
  }
  // W = Q (L1 L2 L3)^T  ->  R = Lacc^T
  { TraceScope ts_(kTrElem, cx.st, 0.0, 16.0 * c * c); (void)launch_pdl(k_transpose, blocks_for((size_t)c * c), 256, 0, cx.st, R, Lacc, c, c); }
  T2S2_CUDA_TRY(cudaGetLastError());
  cx.ar->release(mk);
  return T2S2_OK;
}

t2s2_status qr_tall2(Ctx& cx, const double* U, int c1, const double* W2, int c2, int rows, double* Q, double* R,
                     double* scratch) {
  const int cols = c1 + c2;
  if (cols > kSmallMax || rows < cols || c1 <= 0 || c2 <= 0) return T2S2_EINVAL;
  {
    t2s2_status fs = T2S2_OK;
    if (qr_fused(cx, U, rows, cols, true, Q, R, &fs, W2, c1)) return fs;
  }
  // the pass-by-pass path wants one block
  T2S2_CUDA_TRY(cudaMemcpy2DAsync(scratch, sizeof(double) * cols, U, sizeof(double) * c1, sizeof(double) * c1, rows,
                                  cudaMemcpyDeviceToDevice, cx.st));
  T2S2_CUDA_TRY(cudaMemcpy2DAsync(scratch + c1, sizeof(double) * cols, W2, sizeof(double) * c2, sizeof(double) * c2,
                                  rows, cudaMemcpyDeviceToDevice, cx.st));
  return qr_tall(cx, scratch, rows, cols, Q, R);
}

t2s2_status lq_wide(Ctx& cx, const double* W, int rows, int cols, double* Q, double* Lout) {
  if (rows > kSmallMax || rows > cols || rows <= 0) return T2S2_EINVAL;
  {
    t2s2_status fs = T2S2_OK;
    if (qr_fused(cx, W, cols, rows, false, Q, Lout, &fs)) return fs;
  }
  size_t mk = cx.ar->mark();
  const int c = rows;
  double* G = aget<double>(cx, (size_t)c * c);
  double* L = aget<double>(cx, (size_t)c * c);
  double* Li = aget<double>(cx, (size_t)c * c);
  double* Lacc = aget<double>(cx, (size_t)c * c);
  double* Ltmp = aget<double>(cx, (size_t)c * c);
  double* T0 = aget<double>(cx, (size_t)rows * cols);
  double* T1 = aget<double>(cx, (size_t)rows * cols);
  if (!G || !L || !Li || !Lacc || !Ltmp || !T0 || !T1) return T2S2_ENOMEM;
  const double shift = 11.0 * ((double)rows * cols + (double)c * (c + 1)) * kUnit;
  const double* cur = W;
  double* outs[kCqrMaxPass] = {T0, T1, T0, Q};
  for (int pass = 0; pass < kCqrMaxPass; ++pass) {
    // G = cur cur^T
    T2S2_TRY(gemm_ex<double>(cx, c, c, cols, false, true, 1.0, cur, cols, cur, cols, 0.0, G, c));
    T2S2_TRY(chol_inv(G, c, pass < kCqrShiftedPasses ? shift : 0.0, L, Li, cx.dstat, cx.st));
    // cur = L next  =>  next = L^{-1} cur
    T2S2_TRY(gemm_ex<double>(cx, c, cols, c, false, false, 1.0, Li, c, cur, cols, 0.0, outs[pass], cols));
    if (pass == 0) {
      T2S2_CUDA_TRY(cudaMemcpyAsync(Lacc, L, sizeof(double) * c * c, cudaMemcpyDeviceToDevice, cx.st));
    } else {
      T2S2_TRY(gemm_ex<double>(cx, c, c, c, false, false, 1.0, Lacc, c, L, c, 0.0, Ltmp, c));
      std::swap(Lacc, Ltmp);
    }
    cur = outs[pass];
  }
  T2S2_CUDA_TRY(cudaMemcpyAsync(Lout, Lacc, sizeof(double) * c * c, cudaMemcpyDeviceToDevice, cx.st));
  cx.ar->release(mk);
  return T2S2_OK;
}

t2s2_status tt_alloc(Ctx& cx, DevTT& t, int d, const int* m, const int* r, int rcap) {
  t.d = d;
  for (int k = 0; k <= d; ++k) t.r[k] = r[k];
  for (int k = 0; k < d; ++k) {
    t.m[k] = m[k];
    int r0 = (k == 0) ? 1 : std::max(r[k], rcap);
    int r1 = (k == d - 1) ? 1 : std::max(r[k + 1], rcap);
    t.cap[k] = (size_t)r0 * m[k] * r1;
    t.c[k] = aget<double>(cx, t.cap[k]);
    if (!t.c[k]) return T2S2_ENOMEM;
  }
  return T2S2_OK;
}

t2s2_status tt_copy(Ctx& cx, const DevTT& src, DevTT& dst) {
  for (int k = 0; k < src.d; ++k)
    if (src.core_elems(k) > dst.cap[k]) return T2S2_ENOMEM;
  dst.d = src.d;
  for (int k = 0; k <= src.d; ++k) dst.r[k] = src.r[k];
  for (int k = 0; k < src.d; ++k) {
    dst.m[k] = src.m[k];
    T2S2_CUDA_TRY(cudaMemcpyAsync(dst.c[k], src.c[k], sizeof(double) * src.core_elems(k),
                                  cudaMemcpyDeviceToDevice, cx.st));
  }
  return T2S2_OK;
}

namespace {
struct OrthArgs1 {
  int d;
  int m[T2S2_MAX_D];
  double* c[T2S2_MAX_D];
};
}  // namespace

namespace {
// Cores of z = alpha x + beta y (block structure: first core [alpha X | beta Y],
// middle cores diag(X, Y), last core [X; Y]) for all cores in one launch.
struct SumArgs {
  int d;
  int m[T2S2_MAX_D];
  int rx[T2S2_MAX_D + 1], ry[T2S2_MAX_D + 1], rz[T2S2_MAX_D + 1];
  const double* x[T2S2_MAX_D];
  const double* y[T2S2_MAX_D];
  double* z[T2S2_MAX_D];
  long off[T2S2_MAX_D + 1];
  double alpha, beta;
};

__global__ void k_tt_sum(SumArgs a) {
  pdl_wait();
  pdl_trigger();
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < a.off[a.d]; e += (long)gridDim.x * blockDim.x) {
    int k = 0;
    while (e >= a.off[k + 1]) ++k;
    const long q = e - a.off[k];
    const int m = a.m[k];
    double v;
    if (a.d == 1) {
      v = a.alpha * a.x[0][q] + a.beta * a.y[0][q];
    } else {
      const int rz1 = a.rz[k + 1];
      const int b = (int)(q % rz1);
      const long t = q / rz1;
      const int i = (int)(t % m), aa = (int)(t / m);
      const double ax = (k == 0) ? a.alpha : 1.0, by = (k == 0) ? a.beta : 1.0;
      const int a0y = (k == 0) ? 0 : a.rx[k];
      const int b0y = (k == a.d - 1) ? 0 : a.rx[k + 1];
      const int ya = aa - a0y, yb = b - b0y;
      v = 0.0;
      if (aa < a.rx[k] && b < a.rx[k + 1])
        v = ax * a.x[k][((long)aa * m + i) * a.rx[k + 1] + b];
      else if (ya >= 0 && ya < a.ry[k] && yb >= 0 && yb < a.ry[k + 1])
        v = by * a.y[k][((long)ya * m + i) * a.ry[k + 1] + yb];
    }
    a.z[k][q] = v;
  }
}
}  // namespace

t2s2_status tt_axpby(Ctx& cx, double alpha, const DevTT& x, double beta, const DevTT& y, DevTT& z) {
  const int d = x.d;
  if (y.d != d) return T2S2_EINVAL;
  int r[T2S2_MAX_D + 1];
  r[0] = 1;
  r[d] = 1;
  for (int k = 1; k < d; ++k) r[k] = x.r[k] + y.r[k];
  T2S2_TRY(tt_alloc(cx, z, d, x.m, r, 0));
  SumArgs a;
  a.d = d;
  a.alpha = alpha;
  a.beta = beta;
  a.off[0] = 0;
  for (int k = 0; k <= d; ++k) {
    a.rx[k] = x.r[k];
    a.ry[k] = y.r[k];
    a.rz[k] = z.r[k];
  }
  for (int k = 0; k < d; ++k) {
    if (y.m[k] != x.m[k]) return T2S2_EINVAL;
    a.m[k] = x.m[k];
    a.x[k] = x.c[k];
    a.y[k] = y.c[k];
    a.z[k] = z.c[k];
    a.off[k + 1] = a.off[k] + (long)z.core_elems(k);
  }
  {
    TraceScope ts_(kTrElem, cx.st, 0.0, 16.0 * a.off[d]);
    (void)launch_pdl(k_tt_sum, blocks_for((size_t)a.off[d]), 256, 0, cx.st, a);
  }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

namespace {
// Right orthogonalisation of a TT whose interior ranks are all 1: core k
// (k >= 1) becomes x_k / |x_k| and core 0 takes the product of the norms
// (the LQ factor of a single row is its norm).  One CTA; sums in a fixed
// order.
__global__ void k_orth_rank1(OrthArgs1 a) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[8];
  __shared__ double scale_s;
  double prod = 1.0;
  for (int k = a.d - 1; k >= 0; --k) {
    double* c = a.c[k];
    const int m = a.m[k];
    double s;
    if (k > 0) {
      double p = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) p = fma(c[i], c[i], p);
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double nrm = sqrt(t);
        scale_s = nrm > 0.0 ? 1.0 / nrm : 0.0;
        red[0] = nrm;
      }
      __syncthreads();
      s = scale_s;
      prod *= red[0];
      __syncthreads();
    } else {
      s = prod;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) c[i] *= s;
    __syncthreads();
  }
}
}  // namespace

t2s2_status tt_orth_right(Ctx& cx, DevTT& x) {
  const int d = x.d;
  {
    bool rank1 = true;
    for (int k = 1; k < d; ++k) rank1 = rank1 && x.r[k] == 1;
    if (rank1 && d > 1) {
      OrthArgs1 a;
      a.d = d;
      for (int k = 0; k < d; ++k) {
        a.m[k] = x.m[k];
        a.c[k] = x.c[k];
      }
      {
        TraceScope ts_(kTrSmall, cx.st, 2.0 * d * 64, 16.0 * d * 64);
        (void)launch_pdl(k_orth_rank1, 1, 256, 0, cx.st, a);
      }
      T2S2_CUDA_TRY(cudaGetLastError());
      return T2S2_OK;
    }
  }
  for (int k = d - 1; k >= 1; --k) {
    const int rk = x.r[k], mk_ = x.m[k], rk1 = x.r[k + 1];
    const int cols = mk_ * rk1;
    const int rp = x.r[k - 1], mp = x.m[k - 1];
    size_t mark = cx.ar->mark();
    if (rk <= cols) {
      if (rk > kSmallMax) return T2S2_EINVAL;
      double* Q = aget<double>(cx, (size_t)rk * cols);
      double* L = aget<double>(cx, (size_t)rk * rk);
      double* P = aget<double>(cx, (size_t)rp * mp * rk);
      if (!Q || !L || !P) return T2S2_ENOMEM;
      T2S2_TRY(lq_wide(cx, x.c[k], rk, cols, Q, L));
      T2S2_CUDA_TRY(cudaMemcpyAsync(x.c[k], Q, sizeof(double) * rk * cols, cudaMemcpyDeviceToDevice, cx.st));
      // core k-1 <- core k-1 x_3 L
      T2S2_TRY(gemm_ex<double>(cx, rp * mp, rk, rk, false, false, 1.0, x.c[k - 1], rk, L, rk, 0.0, P, rk));
      T2S2_CUDA_TRY(cudaMemcpyAsync(x.c[k - 1], P, sizeof(double) * rp * mp * rk, cudaMemcpyDeviceToDevice, cx.st));
    } else {
      // rank reduces to cols: core k-1 <- core k-1 x_3 W, core k <- identity
      if ((size_t)rp * mp * cols > x.cap[k - 1] || (size_t)cols * cols > x.cap[k]) return T2S2_ENOMEM;
      double* P = aget<double>(cx, (size_t)rp * mp * cols);
      if (!P) return T2S2_ENOMEM;
      T2S2_TRY(gemm_ex<double>(cx, rp * mp, cols, rk, false, false, 1.0, x.c[k - 1], rk, x.c[k], cols, 0.0, P, cols));
      T2S2_CUDA_TRY(cudaMemcpyAsync(x.c[k - 1], P, sizeof(double) * rp * mp * cols, cudaMemcpyDeviceToDevice, cx.st));
      T2S2_TRY(dev_identity(cx, x.c[k], cols));
      x.r[k] = cols;
    }
    cx.ar->release(mark);
  }
  return T2S2_OK;
}

t2s2_status tt_norm(Ctx& cx, const DevTT& x, double* out) {
  size_t mark = cx.ar->mark();
  DevTT t;
  int rc = 0;
  for (int k = 0; k <= x.d; ++k) rc = std::max(rc, x.r[k]);
  T2S2_TRY(tt_alloc(cx, t, x.d, x.m, x.r, rc));
  T2S2_TRY(tt_copy(cx, x, t));
  T2S2_TRY(tt_orth_right(cx, t));
  T2S2_TRY(core_norm(cx, t.c[0], t.core_elems(0), out));
  cx.ar->release(mark);
  return T2S2_OK;
}

t2s2_status tt_round(Ctx& cx, DevTT& x, double tol, int rmax) {
  const int d = x.d;
  if (d == 1) return T2S2_OK;
  T2S2_TRY(tt_orth_right(cx, x));
  double nrm;
  T2S2_TRY(core_norm(cx, x.c[0], x.core_elems(0), &nrm));
  if (nrm == 0.0) {
    for (int k = 0; k < d; ++k) {
      x.r[k] = 1;
      T2S2_TRY(dev_fill(cx, x.c[k], x.m[k], 0.0));
    }
    x.r[d] = 1;
    return T2S2_OK;
  }
  const double delta = tol * nrm / std::sqrt((double)(d - 1));
  for (int k = 0; k + 1 < d; ++k) {
    const int rk = x.r[k], mk_ = x.m[k], rk1 = x.r[k + 1];
    const int rows = rk * mk_;
    const int mn = x.m[k + 1], rn = x.r[k + 2];
    size_t mark = cx.ar->mark();
    const int kk = std::min(rows, rk1);
    double* U = aget<double>(cx, (size_t)kk * kk);
    double* s = aget<double>(cx, (size_t)kk);
    double* V = aget<double>(cx, (size_t)rk1 * kk);
    double* Q = aget<double>(cx, (size_t)rows * rk1);
    double* R = aget<double>(cx, (size_t)rk1 * rk1);
    double* SV = aget<double>(cx, (size_t)kk * rk1);
    double* P = aget<double>(cx, (size_t)kk * mn * rn);
    if (!U || !s || !V || !Q || !R || !SV || !P) return T2S2_ENOMEM;
    if (rk1 > kSmallMax || kk > kSmallMax) return T2S2_EINVAL;
    if (rows >= rk1) {
      T2S2_TRY(qr_tall(cx, x.c[k], rows, rk1, Q, R));
      T2S2_TRY(jacobi_svd(R, rk1, rk1, U, s, V, nullptr, cx.st));
    } else {
      T2S2_TRY(jacobi_svd(x.c[k], rows, rk1, U, s, V, nullptr, cx.st));
    }
    T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, s, sizeof(double) * kk, cudaMemcpyDeviceToHost, cx.st));
    T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
    const int rn_new = trunc_rank(cx.hbuf, kk, delta, rmax);
    // core k <- Q U[:, :rn_new]  (or U[:, :rn_new] when the unfolding is wide)
    if (rows >= rk1) {
      T2S2_TRY(gemm_ex<double>(cx, rows, rn_new, rk1, false, false, 1.0, Q, rk1, U, kk, 0.0, x.c[k], rn_new));
    } else {
      // U is rows x kk with kk = rows; take its first rn_new columns
      T2S2_CUDA_TRY(cudaMemcpy2DAsync(x.c[k], sizeof(double) * rn_new, U, sizeof(double) * kk,
                                      sizeof(double) * rn_new, rows, cudaMemcpyDeviceToDevice, cx.st));
    }
    // core k+1 <- diag(s) V^T [:rn_new] x_1 core k+1
    T2S2_TRY(dev_sv_t(cx, SV, s, V, rn_new, rk1, kk));
    T2S2_TRY(gemm_ex<double>(cx, rn_new, mn * rn, rk1, false, false, 1.0, SV, rk1, x.c[k + 1], mn * rn, 0.0, P, mn * rn));
    T2S2_CUDA_TRY(cudaMemcpyAsync(x.c[k + 1], P, sizeof(double) * rn_new * mn * rn, cudaMemcpyDeviceToDevice, cx.st));
    x.r[k + 1] = rn_new;
    cx.ar->release(mark);
  }
  return T2S2_OK;
}

}  // namespace t2s2
