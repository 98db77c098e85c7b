// Learned warm start: an MLP from problem parameters to the TT cores of an
// initial guess for the alternating solver, trained on the GPU by this file's
// kernels.  The solver accepts any initial guess and always runs to the same
// residual tolerance, so the network can only change the number of sweeps,
// never the answer.
//
//   h1 = relu(W1 p + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,
//
// y holds raw cores Y_k (core 0: 1 x m_1 x r, middle: r x m_k x r, last:
// r x m_d x 1, row-major, concatenated) and a log-scale sigma; X(p) has the
// cores Y_k / ||Y_k||, core 0 times exp(sigma), so the network learns each
// core's direction and one overall size (the solver does not depend on the
// scale of its initial guess; raw cores would make the loss a polynomial of
// degree 2d).  Loss per sample with target U: ||X - U||^2 / ||U||^2 =
// (<X,X> - 2 <X,U> + <U,U>) / <U,U>, independent of the TT gauge of X; its
// gradient with respect to core k comes from the left and right environments
// of <X,X> and <X,U>, then through the normalisation.
//
// Kernels: the six layer products (three forward, three backward per layer
// pair) run on the tcgen05 GEMM with BF16 operands (weights and activations
// rounded as they are staged) and FP32 accumulation; bias/ReLU, the TT loss
// and its core gradient (one CTA per sample, environments in shared memory),
// the column sums for the bias gradients and Adam are FP32 SIMT kernels.
// Parameters, gradients and Adam moments are FP32 master copies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_bf16.h>

#include "api_internal.h"
#include "gemm_tc.h"
#include "trace.h"

struct t2s2_mlp_s {
  int device = 0;
  int in_dim = 0, hidden = 0, d = 0, r = 0, ru = 0, odim = 0, ncore = 0, mmax = 0;
  int m[T2S2_MAX_D] = {0};
  int off[T2S2_MAX_D + 1] = {0};  // offsets of the cores in y; y[ncore] = sigma
  double* ystage = nullptr;        // ncore doubles: the cores of one prediction
  long long nparams = 0;
  long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float* params = nullptr;  // W1 b1 W2 b2 W3 b3
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long step = 0;
  int bcap = 0;  // batch capacity of the activation buffers
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr;
  float *dh = nullptr, *dz = nullptr, *loss = nullptr, *xx = nullptr;
  float* pbuf = nullptr;  // in_dim floats: the input of a single prediction
  long long* dstep = nullptr;  // device copy of the Adam step count
  float* dlr = nullptr;        // device learning rate
  float* hlr = nullptr;        // pinned host staging of the learning rate
  struct GraphEntry {
    const float *P, *targets, *uu;
    int batch;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;  // captured training steps, one per minibatch
  cudaStream_t gstream = nullptr;  // non-blocking stream for capture and replay
  cudaEvent_t gev = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* dstat = nullptr;
  float* hbuf = nullptr;  // pinned host scratch (bcap floats)
};

namespace t2s2 {

namespace {

constexpr int kLossThreads = 256;
constexpr int kMlpMaxRank = 16;
constexpr int kMlpMaxTargetRank = 32;
constexpr int kMlpMaxM = 64;

struct LossArgs {
  const float* y;        // batch x odim (odim = ncore + 1: cores, then sigma)
  const float* targets;  // batch x d x ru x mmax x ru (zero padded)
  const float* uu;       // batch: <U,U>
  float* dy;             // batch x odim: dL/dy, already divided by the batch size
  float* loss;           // batch
  float* xx;             // batch: <X,X> (optional)
  int batch, odim, ncore, d, r, ru, mmax;
  int m[T2S2_MAX_D];
  int off[T2S2_MAX_D + 1];
  float inv_batch;
};

size_t loss_smem_floats(const LossArgs& a) {
  const size_t env = (size_t)(a.d + 1) * (2 * a.r * a.r + 2 * a.r * a.ru);
  const size_t W = (size_t)std::max(a.r, a.ru) * a.mmax * a.r;
  const size_t G = (size_t)a.r * a.mmax * a.r;
  return 2 * (size_t)a.ncore + env + W + G + kLossThreads + 2 * T2S2_MAX_D;
}

// One CTA per sample.  Every core of X is treated as r x m_k x r with zeros
// outside its true shape (the boundary cores have one row / column), and every
// target core as ru x m_k x ru (zero padded), so the same contraction loops
// serve all cores; the zeros leave every inner product unchanged.
__global__ void __launch_bounds__(kLossThreads) tt_loss_grad_kernel(LossArgs a) {
  extern __shared__ float sm[];
  const int s = blockIdx.x, tid = threadIdx.x;
  const int d = a.d, r = a.r, ru = a.ru, mmax = a.mmax;
  float* sX = sm;
  float* Gall = sX + a.ncore;  // dL/dX, all cores
  float* Lxx = Gall + a.ncore;
  float* Rxx = Lxx + (d + 1) * r * r;
  float* Lxu = Rxx + (d + 1) * r * r;
  float* Rxu = Lxu + (d + 1) * r * ru;
  float* W = Rxu + (d + 1) * r * ru;
  float* G = W + max(r, ru) * mmax * r;
  float* red = G + r * mmax * r;  // block-reduction scratch
  float* invn = red + kLossThreads;  // 1 / ||Y_k||
  float* dots = invn + T2S2_MAX_D;   // <dL/dX_k, X_k>
  const float* U = a.targets + (size_t)s * d * ru * mmax * ru;
  for (int e = tid; e < a.ncore; e += kLossThreads) sX[e] = a.y[(size_t)s * a.odim + e];
  const float sigma = a.y[(size_t)s * a.odim + a.ncore];
  const float esig = expf(sigma);
  __syncthreads();
  // X_k = Y_k / ||Y_k|| (core 0 times exp(sigma)); sums in a fixed order
  for (int k = 0; k < d; ++k) {
    float acc = 0.f;
    for (int e = a.off[k] + tid; e < a.off[k + 1]; e += kLossThreads) acc = fmaf(sX[e], sX[e], acc);
    red[tid] = acc;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) invn[k] = red[0] > 0.f ? rsqrtf(red[0]) : 0.f;
    __syncthreads();
  }
  for (int k = 0; k < d; ++k) {
    const float f = invn[k] * (k == 0 ? esig : 1.f);
    for (int e = a.off[k] + tid; e < a.off[k + 1]; e += kLossThreads) sX[e] *= f;
  }
  for (int e = tid; e < (d + 1) * r * r; e += kLossThreads) Lxx[e] = Rxx[e] = 0.f;
  for (int e = tid; e < (d + 1) * r * ru; e += kLossThreads) Lxu[e] = Rxu[e] = 0.f;
  __syncthreads();
  if (tid == 0) {
    Lxx[0] = 1.f;
    Lxu[0] = 1.f;
    Rxx[d * r * r] = 1.f;
    Rxu[d * r * ru] = 1.f;
  }
  __syncthreads();
  auto X = [&](int k, int aa, int i, int b) -> float {
    const int ra = (k == 0) ? 1 : r, rb = (k == d - 1) ? 1 : r;
    return (aa < ra && b < rb) ? sX[a.off[k] + (aa * a.m[k] + i) * rb + b] : 0.f;
  };
  auto Ut = [&](int k, int c, int i, int c2) -> float {
    return U[(((size_t)k * ru + c) * mmax + i) * ru + c2];
  };
  // left environments
  for (int k = 0; k < d; ++k) {
    const int mk = a.m[k];
    const float* L = Lxx + k * r * r;
    // W[a2, i, b] = sum_a L[a, a2] X[a, i, b]
    for (int e = tid; e < r * mk * r; e += kLossThreads) {
      const int a2 = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int aa = 0; aa < r; ++aa) acc = fmaf(L[aa * r + a2], X(k, aa, i, b), acc);
      W[e] = acc;
    }
    __syncthreads();
    // Lxx[k+1][b, b2] = sum_{a2, i} W[a2, i, b] X[a2, i, b2]
    for (int e = tid; e < r * r; e += kLossThreads) {
      const int b = e / r, b2 = e % r;
      float acc = 0.f;
      for (int a2 = 0; a2 < r; ++a2)
        for (int i = 0; i < mk; ++i) acc = fmaf(W[(a2 * mk + i) * r + b], X(k, a2, i, b2), acc);
      Lxx[(k + 1) * r * r + e] = acc;
    }
    __syncthreads();
    const float* F = Lxu + k * r * ru;
    // W[c, i, b] = sum_a F[a, c] X[a, i, b]
    for (int e = tid; e < ru * mk * r; e += kLossThreads) {
      const int c = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int aa = 0; aa < r; ++aa) acc = fmaf(F[aa * ru + c], X(k, aa, i, b), acc);
      W[e] = acc;
    }
    __syncthreads();
    // Lxu[k+1][b, c2] = sum_{c, i} W[c, i, b] U[c, i, c2]
    for (int e = tid; e < r * ru; e += kLossThreads) {
      const int b = e / ru, c2 = e % ru;
      float acc = 0.f;
      for (int c = 0; c < ru; ++c)
        for (int i = 0; i < mk; ++i) acc = fmaf(W[(c * mk + i) * r + b], Ut(k, c, i, c2), acc);
      Lxu[(k + 1) * r * ru + e] = acc;
    }
    __syncthreads();
  }
  // right environments
  for (int k = d - 1; k >= 1; --k) {
    const int mk = a.m[k];
    const float* Rn = Rxx + (k + 1) * r * r;
    // W[a2, i, b] = sum_b2 X[a2, i, b2] Rn[b, b2]
    for (int e = tid; e < r * mk * r; e += kLossThreads) {
      const int a2 = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int b2 = 0; b2 < r; ++b2) acc = fmaf(X(k, a2, i, b2), Rn[b * r + b2], acc);
      W[e] = acc;
    }
    __syncthreads();
    // Rxx[k][aa, a2] = sum_{i, b} X[aa, i, b] W[a2, i, b]
    for (int e = tid; e < r * r; e += kLossThreads) {
      const int aa = e / r, a2 = e % r;
      float acc = 0.f;
      for (int i = 0; i < mk; ++i)
        for (int b = 0; b < r; ++b) acc = fmaf(X(k, aa, i, b), W[(a2 * mk + i) * r + b], acc);
      Rxx[k * r * r + e] = acc;
    }
    __syncthreads();
    const float* Fn = Rxu + (k + 1) * r * ru;
    // W[c, i, b] = sum_c2 U[c, i, c2] Fn[b, c2]
    for (int e = tid; e < ru * mk * r; e += kLossThreads) {
      const int c = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int c2 = 0; c2 < ru; ++c2) acc = fmaf(Ut(k, c, i, c2), Fn[b * ru + c2], acc);
      W[e] = acc;
    }
    __syncthreads();
    // Rxu[k][aa, c] = sum_{i, b} X[aa, i, b] W[c, i, b]
    for (int e = tid; e < r * ru; e += kLossThreads) {
      const int aa = e / ru, c = e % ru;
      float acc = 0.f;
      for (int i = 0; i < mk; ++i)
        for (int b = 0; b < r; ++b) acc = fmaf(X(k, aa, i, b), W[(c * mk + i) * r + b], acc);
      Rxu[k * r * ru + e] = acc;
    }
    __syncthreads();
  }
  const float xx = Lxx[d * r * r], xu = Lxu[d * r * ru], uu = a.uu[s];
  if (tid == 0) {
    a.loss[s] = (xx - 2.f * xu + uu) / uu;
    if (a.xx) a.xx[s] = xx;
  }
  const float scale = a.inv_batch / uu;
  // gradient, core by core
  for (int k = 0; k < d; ++k) {
    const int mk = a.m[k];
    const float* L = Lxx + k * r * r;
    const float* Rn = Rxx + (k + 1) * r * r;
    // W[a2, i, b] = sum_b2 X[a2, i, b2] Rn[b, b2];  G[a, i, b] = 2 sum_a2 L[a, a2] W[a2, i, b]
    for (int e = tid; e < r * mk * r; e += kLossThreads) {
      const int a2 = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int b2 = 0; b2 < r; ++b2) acc = fmaf(X(k, a2, i, b2), Rn[b * r + b2], acc);
      W[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * mk * r; e += kLossThreads) {
      const int aa = e / (mk * r), rem = e % (mk * r);
      float acc = 0.f;
      for (int a2 = 0; a2 < r; ++a2) acc = fmaf(L[aa * r + a2], W[a2 * mk * r + rem], acc);
      G[e] = 2.f * acc;
    }
    __syncthreads();
    const float* F = Lxu + k * r * ru;
    const float* Fn = Rxu + (k + 1) * r * ru;
    // W[c, i, b] = sum_c2 U[c, i, c2] Fn[b, c2];  G[a, i, b] -= 2 sum_c F[a, c] W[c, i, b]
    for (int e = tid; e < ru * mk * r; e += kLossThreads) {
      const int c = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int c2 = 0; c2 < ru; ++c2) acc = fmaf(Ut(k, c, i, c2), Fn[b * ru + c2], acc);
      W[e] = acc;
    }
    __syncthreads();
    const int ra = (k == 0) ? 1 : r, rb = (k == d - 1) ? 1 : r;
    for (int e = tid; e < r * mk * r; e += kLossThreads) {
      const int aa = e / (mk * r), rem = e % (mk * r), i = rem / r, b = rem % r;
      float acc = 0.f;
      for (int c = 0; c < ru; ++c) acc = fmaf(F[aa * ru + c], W[c * mk * r + rem], acc);
      if (aa < ra && b < rb) Gall[a.off[k] + (aa * mk + i) * rb + b] = G[e] - 2.f * acc;
    }
    __syncthreads();
  }
  // through the normalisation: with Yhat = Y / ||Y|| and g = dL/dYhat,
  // dL/dY = (g - <g, Yhat> Yhat) / ||Y||; for every core <g, Yhat> equals
  // <dL/dX_k, X_k>, which for core 0 is also dL/dsigma
  for (int k = 0; k < d; ++k) {
    float acc = 0.f;
    for (int e = a.off[k] + tid; e < a.off[k + 1]; e += kLossThreads) acc = fmaf(Gall[e], sX[e], acc);
    red[tid] = acc;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) dots[k] = red[0];
    __syncthreads();
  }
  for (int k = 0; k < d; ++k) {
    const float gs = (k == 0) ? esig : 1.f;      // g = gs * dL/dX_k
    const float ys = (k == 0) ? 1.f / esig : 1.f;  // Yhat = ys * X_k
    for (int e = a.off[k] + tid; e < a.off[k + 1]; e += kLossThreads)
      a.dy[(size_t)s * a.odim + e] = (gs * Gall[e] - dots[k] * ys * sX[e]) * invn[k] * scale;
  }
  if (tid == 0) a.dy[(size_t)s * a.odim + a.ncore] = dots[0] * scale;
}

// z += bias (per column); h = relu(z) if h != nullptr.
__global__ void bias_act_kernel(float* z, float* h, const float* bias, int rows, int cols) {
  const long n = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const float v = z[e] + bias[e % cols];
    z[e] = v;
    if (h) h[e] = v > 0.f ? v : 0.f;
  }
}

// dz = dh * (z > 0)
__global__ void relu_back_kernel(float* dz, const float* dh, const float* z, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dz[e] = z[e] > 0.f ? dh[e] : 0.f;
}

// out[j] = sum_i v[i][j] (rows summed in order: deterministic)
__global__ void colsum_kernel(float* out, const float* v, int rows, int cols) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int i = 0; i < rows; ++i) acc += v[(long)i * cols + j];
    out[j] = acc;
  }
}

// Adam with bias correction (Kingma & Ba): bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
// The step t (after this update) and the learning rate are read from device
// memory, so that a captured CUDA graph of the training step stays valid from
// one replay to the next.
__global__ void adam_kernel(float* p, const float* g, float* mo, float* ve, long n, const float* lr_p,
                            const long long* step_p, float beta1, float beta2, float eps) {
  const double t = (double)(*step_p + 1);
  const float bc1 = (float)(1.0 - pow((double)beta1, t));
  const float bc2 = (float)(1.0 - pow((double)beta2, t));
  const float lr = *lr_p;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float m1 = beta1 * mo[e] + (1.f - beta1) * gg;
    const float v1 = beta2 * ve[e] + (1.f - beta2) * gg * gg;
    mo[e] = m1;
    ve[e] = v1;
    p[e] -= lr * (m1 / bc1) / (sqrtf(v1 / bc2) + eps);
  }
}

__global__ void step_increment_kernel(long long* step_p) { *step_p += 1; }

// Packs one FP64 target TT into the zero-padded FP32 slot (d x ru x mmax x ru).
__global__ void pack_core_kernel(float* slot, const double* core, int ra, int m, int rb, int ru, int mmax) {
  const long n = (long)ru * mmax * ru;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((long)mmax * ru)), rem = (int)(e % ((long)mmax * ru)), i = rem / ru, c2 = rem % ru;
    slot[e] = (c < ra && i < m && c2 < rb) ? (float)core[((long)c * m + i) * rb + c2] : 0.f;
  }
}

// Writes one rounded FP64 core (ra x m x rb) into the network's output bias
// as an FP32 core of the network's shape (na x m x nb), zero outside it.
__global__ void bias_core_kernel(float* bias, const double* core, int ra, int m, int rb, int na, int nb) {
  const long n = (long)na * m * nb;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long)m * nb)), rem = (int)(e % ((long)m * nb)), i = rem / nb, b = rem % nb;
    bias[e] = (a < ra && b < rb) ? (float)core[((long)a * m + i) * rb + b] : 0.f;
  }
}

__global__ void scale_kernel(float* v, long n, float f) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) v[e] *= f;
}

// The cores of X(p) for one sample: block k normalises raw core k of y
// (fixed-order block sum) and scales core 0 by exp(sigma); FP64 out.
struct UnpackArgs {
  const float* y;
  double* out;
  int off[T2S2_MAX_D + 1];
  int ncore;
};
__global__ void unpack_cores_kernel(UnpackArgs u) {
  __shared__ float red[256];
  const int k = blockIdx.x, t = threadIdx.x;
  const int o0 = u.off[k], o1 = u.off[k + 1];
  float acc = 0.f;
  for (int e = o0 + t; e < o1; e += blockDim.x) acc = fmaf(u.y[e], u.y[e], acc);
  red[t] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double f = (red[0] > 0.f ? 1.0 / sqrt((double)red[0]) : 0.0) * (k == 0 ? exp((double)u.y[u.ncore]) : 1.0);
  for (int e = o0 + t; e < o1; e += blockDim.x) u.out[e] = f * (double)u.y[e];
}

int ew_blocks(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 8L * kNumSMs)); }

// Prediction for one parameter vector in one CTA: the three layers as
// warp-per-row products with the operands rounded to BF16 and FP32 sums (the
// arithmetic of the batched tensor-core layers, summed in another order),
// then the cores of X(p) normalised and written as FP64 straight into the
// caller's cores.  One launch instead of the batched path's GEMM, bias and
// unpack launches; used for warm starts, where the solve waits on it.
constexpr int kPredictInline = 64;  // inputs passed inside the launch arguments
struct PredictArgs {
  const float* p;                 // device input, or null: pin holds it
  float pin[kPredictInline];
  const float* w;
  long long oW1, ob1, oW2, ob2, oW3, ob3;
  int in_dim, hidden, odim, ncore, d;
  int off[T2S2_MAX_D + 1];
  double* out[T2S2_MAX_D];
};
constexpr int kPredictThreads = 512;
constexpr size_t kPredictMaxSmem = 96 * 1024;

size_t predict_smem_bytes(int in_dim, int hidden, int odim) {
  return sizeof(float) * ((size_t)in_dim + 2 * (size_t)hidden + (size_t)odim + 32);
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// out[row] = act(sum_i bf16(W[row, i]) bf16(x[i]) + bias[row]) for row < rows.
__device__ void gemv_rows(const float* W, const float* bias, const float* x, float* out, int rows, int K,
                          bool relu) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < rows; row += nw) {
    const float* wr = W + (long)row * K;
    float acc = 0.f;
    for (int i = lane; i < K; i += 32) acc = fmaf(bf16r(wr[i]), bf16r(x[i]), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const float v = acc + bias[row];
      out[row] = relu ? fmaxf(v, 0.f) : v;
    }
  }
}

__global__ void __launch_bounds__(kPredictThreads) predict_kernel(PredictArgs a) {
  extern __shared__ float sm[];
  float* xin = sm;
  float* h1 = xin + a.in_dim;
  float* h2 = h1 + a.hidden;
  float* y = h2 + a.hidden;
  float* red = y + a.odim;
  for (int i = threadIdx.x; i < a.in_dim; i += blockDim.x) xin[i] = a.p ? a.p[i] : a.pin[i];
  __syncthreads();
  gemv_rows(a.w + a.oW1, a.w + a.ob1, xin, h1, a.hidden, a.in_dim, true);
  __syncthreads();
  gemv_rows(a.w + a.oW2, a.w + a.ob2, h1, h2, a.hidden, a.hidden, true);
  __syncthreads();
  gemv_rows(a.w + a.oW3, a.w + a.ob3, h2, y, a.odim, a.hidden, false);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < a.d; ++k) {
    const int o0 = a.off[k], o1 = a.off[k + 1];
    float acc = 0.f;
    for (int e = o0 + threadIdx.x; e < o1; e += blockDim.x) acc = fmaf(y[e], y[e], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    float ss = 0.f;
    for (int w = 0; w < nw; ++w) ss += red[w];  // fixed order
    const double f = (ss > 0.f ? 1.0 / sqrt((double)ss) : 0.0) * (k == 0 ? exp((double)y[a.ncore]) : 1.0);
    for (int e = o0 + threadIdx.x; e < o1; e += blockDim.x) a.out[k][e - o0] = f * (double)y[e];
    __syncthreads();
  }
}

// Captured graphs hold buffer addresses: drop them whenever a buffer moves.
void drop_graphs(t2s2_mlp net) {
  for (auto& g : net->graphs) cudaGraphExecDestroy(g.exec);
  net->graphs.clear();
}

t2s2_status mm(t2s2_mlp net, int M, int N, int K, bool tA, bool tB, const float* A, long lda, const float* B,
               long ldb, float* C, long ldc, cudaStream_t st) {
  Gemm<float> g;
  g.M = M; g.N = N; g.K = K; g.tA = tA; g.tB = tB; g.alpha = 1.f; g.beta = 0.f;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc; g.batch = 1;
  const size_t need = gemm_tc_workspace_bytes(g, T2S2_BF16_REFINE);
  if (need > net->ws_bytes) {
    T2S2_CUDA_TRY(cudaStreamSynchronize(st));  // earlier launches may still read the old buffer
    drop_graphs(net);
    if (net->ws) cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_bytes = 0;
    T2S2_CUDA_TRY(cudaMalloc(&net->ws, need));
    net->ws_bytes = need;
  }
  return gemm_tc(g, T2S2_BF16_REFINE, net->ws, net->ws_bytes, net->dstat, st);
}

t2s2_status ensure_batch(t2s2_mlp net, int batch) {
  if (batch <= net->bcap) return T2S2_OK;
  drop_graphs(net);
  float** bufs[] = {&net->z1, &net->h1, &net->z2, &net->h2, &net->dh, &net->dz, &net->y, &net->dy, &net->loss,
                    &net->xx};
  for (auto b : bufs)
    if (*b) cudaFree(*b), *b = nullptr;
  if (net->hbuf) cudaFreeHost(net->hbuf), net->hbuf = nullptr;
  const size_t H = (size_t)batch * net->hidden, Y = (size_t)batch * net->odim;
  const size_t sizes[] = {H, H, H, H, H, H, Y, Y, (size_t)batch, (size_t)batch};
  for (int i = 0; i < 10; ++i) T2S2_CUDA_TRY(cudaMalloc(bufs[i], sizes[i] * sizeof(float)));
  T2S2_CUDA_TRY(cudaMallocHost(&net->hbuf, (size_t)batch * sizeof(float)));
  net->bcap = batch;
  return T2S2_OK;
}

t2s2_status forward(t2s2_mlp net, const float* P, int B, cudaStream_t st) {
  const int h = net->hidden;
  float* w = net->params;
  T2S2_TRY(mm(net, B, h, net->in_dim, false, true, P, net->in_dim, w + net->oW1, net->in_dim, net->z1, h, st));
  {
    TraceScope ts(kTrMlp, st, 2.0 * B * h, 8.0 * B * h);
    bias_act_kernel<<<ew_blocks((long)B * h), 256, 0, st>>>(net->z1, net->h1, w + net->ob1, B, h);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  T2S2_TRY(mm(net, B, h, h, false, true, net->h1, h, w + net->oW2, h, net->z2, h, st));
  {
    TraceScope ts(kTrMlp, st, 2.0 * B * h, 8.0 * B * h);
    bias_act_kernel<<<ew_blocks((long)B * h), 256, 0, st>>>(net->z2, net->h2, w + net->ob2, B, h);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  T2S2_TRY(mm(net, B, net->odim, h, false, true, net->h2, h, w + net->oW3, h, net->y, net->odim, st));
  {
    TraceScope ts(kTrMlp, st, 1.0 * B * net->odim, 8.0 * B * net->odim);
    bias_act_kernel<<<ew_blocks((long)B * net->odim), 256, 0, st>>>(net->y, nullptr, w + net->ob3, B, net->odim);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  return T2S2_OK;
}

t2s2_status loss_grad(t2s2_mlp net, const float* P, int B, const float* targets, const float* uu, cudaStream_t st) {
  T2S2_TRY(forward(net, P, B, st));
  LossArgs a;
  a.y = net->y;
  a.targets = targets;
  a.uu = uu;
  a.dy = net->dy;
  a.loss = net->loss;
  a.xx = net->xx;
  a.batch = B;
  a.odim = net->odim;
  a.ncore = net->ncore;
  a.d = net->d;
  a.r = net->r;
  a.ru = net->ru;
  a.mmax = net->mmax;
  for (int k = 0; k < net->d; ++k) a.m[k] = net->m[k];
  for (int k = 0; k <= net->d; ++k) a.off[k] = net->off[k];
  a.inv_batch = 1.f / (float)B;
  const size_t smem = loss_smem_floats(a) * sizeof(float);
  {
    double fl = 0.0;
    for (int k = 0; k < net->d; ++k) {
      const double mk = net->m[k], r = net->r, ru = net->ru;
      fl += 2.0 * (2 * r * mk * r * r + 2 * ru * mk * r * r + 2 * ru * mk * r * ru) * 1.5;
    }
    TraceScope ts(kTrMlp, st, fl * B, 4.0 * B * ((double)net->odim * 2 + (double)net->d * net->ru * net->mmax * net->ru));
    T2S2_CUDA_TRY(cudaFuncSetAttribute(tt_loss_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(smem, 200 * 1024)));
    tt_loss_grad_kernel<<<B, kLossThreads, smem, st>>>(a);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  // backward through the layers
  const int h = net->hidden, od = net->odim;
  float* w = net->params;
  float* g = net->grads;
  T2S2_TRY(mm(net, od, h, B, true, false, net->dy, od, net->h2, h, g + net->oW3, h, st));  // dW3 = dy^T h2
  {
    TraceScope ts(kTrMlp, st, 1.0 * B * od, 4.0 * B * od);
    colsum_kernel<<<ew_blocks(od), 256, 0, st>>>(g + net->ob3, net->dy, B, od);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  T2S2_TRY(mm(net, B, h, od, false, false, net->dy, od, w + net->oW3, h, net->dh, h, st));  // dh2 = dy W3
  {
    TraceScope ts(kTrMlp, st, 2.0 * B * h, 12.0 * B * h);
    relu_back_kernel<<<ew_blocks((long)B * h), 256, 0, st>>>(net->dz, net->dh, net->z2, (long)B * h);
    colsum_kernel<<<ew_blocks(h), 256, 0, st>>>(g + net->ob2, net->dz, B, h);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  T2S2_TRY(mm(net, h, h, B, true, false, net->dz, h, net->h1, h, g + net->oW2, h, st));  // dW2 = dz2^T h1
  T2S2_TRY(mm(net, B, h, h, false, false, net->dz, h, w + net->oW2, h, net->dh, h, st));  // dh1 = dz2 W2
  {
    TraceScope ts(kTrMlp, st, 2.0 * B * h, 12.0 * B * h);
    relu_back_kernel<<<ew_blocks((long)B * h), 256, 0, st>>>(net->dz, net->dh, net->z1, (long)B * h);
    colsum_kernel<<<ew_blocks(h), 256, 0, st>>>(g + net->ob1, net->dz, B, h);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  T2S2_TRY(mm(net, h, net->in_dim, B, true, false, net->dz, h, P, net->in_dim, g + net->oW1, net->in_dim, st));
  return T2S2_OK;
}

t2s2_status check_status(t2s2_mlp net, cudaStream_t st) {
  int h = 0;
  T2S2_CUDA_TRY(cudaMemcpyAsync(&h, net->dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  return h ? T2S2_ETIMEOUT : T2S2_OK;
}

t2s2_status mean_loss(t2s2_mlp net, int B, float* out, cudaStream_t st) {
  T2S2_CUDA_TRY(cudaMemcpyAsync(net->hbuf, net->loss, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
  T2S2_TRY(check_status(net, st));
  double s = 0.0;
  for (int i = 0; i < B; ++i) s += net->hbuf[i];
  *out = (float)(s / B);
  return T2S2_OK;
}

t2s2_status set_lr(t2s2_mlp net, float lr, cudaStream_t st) {
  // the previous copy out of the pinned slot must be done before it is reused
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  *net->hlr = lr;
  T2S2_CUDA_TRY(cudaMemcpyAsync(net->dlr, net->hlr, sizeof(float), cudaMemcpyHostToDevice, st));
  return T2S2_OK;
}

// One training step as a fixed sequence of launches (capturable): loss and
// gradient, Adam update, step counter.
t2s2_status train_launches(t2s2_mlp net, const float* P, int batch, const float* targets, const float* uu,
                           cudaStream_t st) {
  T2S2_TRY(loss_grad(net, P, batch, targets, uu, st));
  TraceScope ts(kTrMlp, st, 10.0 * net->nparams, 4.0 * 7 * net->nparams);
  adam_kernel<<<ew_blocks(net->nparams), 256, 0, st>>>(net->params, net->grads, net->adam_m, net->adam_v,
                                                     net->nparams, net->dlr, net->dstep, 0.9f, 0.999f, 1e-8f);
  step_increment_kernel<<<1, 1, 0, st>>>(net->dstep);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" {

t2s2_status t2s2_mlp_create(int in_dim, int hidden, int d, const int* m, int r, int ru, unsigned long long seed,
                            t2s2_mlp* out) {
  if (!out || !m || in_dim < 1 || hidden < 1 || d < 2 || d > T2S2_MAX_D) return T2S2_EINVAL;
  if (r < 1 || r > kMlpMaxRank || ru < 1 || ru > kMlpMaxTargetRank) return T2S2_EINVAL;
  *out = nullptr;
  t2s2_mlp net = new t2s2_mlp_s;
  cudaGetDevice(&net->device);
  net->in_dim = in_dim;
  net->hidden = hidden;
  net->d = d;
  net->r = r;
  net->ru = ru;
  int o = 0;
  for (int k = 0; k < d; ++k) {
    if (m[k] < 1 || m[k] > kMlpMaxM) {
      delete net;
      return T2S2_EINVAL;
    }
    net->m[k] = m[k];
    net->mmax = std::max(net->mmax, m[k]);
    net->off[k] = o;
    o += (k == 0 ? 1 : r) * m[k] * (k == d - 1 ? 1 : r);
  }
  net->off[d] = o;
  net->ncore = o;
  net->odim = o + 1;  // the cores, then the log-scale
  {
    LossArgs a{};
    a.odim = o + 1; a.ncore = o; a.d = d; a.r = r; a.ru = ru; a.mmax = net->mmax;
    if (loss_smem_floats(a) * sizeof(float) > 200 * 1024) {
      delete net;
      return T2S2_EINVAL;
    }
  }
  const long long h = hidden;
  o = net->odim;  // network outputs
  net->oW1 = 0;
  net->ob1 = h * in_dim;
  net->oW2 = net->ob1 + h;
  net->ob2 = net->oW2 + h * h;
  net->oW3 = net->ob2 + h;
  net->ob3 = net->oW3 + (long long)o * h;
  net->nparams = net->ob3 + o;
  // He-normal weights (std sqrt(2 / fan_in); sqrt(1 / fan_in) for the linear
  // output layer), zero biases, from a seeded host generator
  std::vector<float> p(net->nparams, 0.f);
  std::mt19937_64 gen(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (long long i = 0; i < h * in_dim; ++i) p[net->oW1 + i] = (float)(nd(gen) * std::sqrt(2.0 / in_dim));
  for (long long i = 0; i < h * h; ++i) p[net->oW2 + i] = (float)(nd(gen) * std::sqrt(2.0 / h));
  for (long long i = 0; i < (long long)o * h; ++i) p[net->oW3 + i] = (float)(nd(gen) * std::sqrt(1.0 / h));
  const size_t bytes = sizeof(float) * net->nparams;
  cudaError_t e = cudaMalloc(&net->params, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&net->grads, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&net->adam_m, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&net->adam_v, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&net->dstat, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&net->pbuf, sizeof(float) * in_dim);
  if (e == cudaSuccess) e = cudaMalloc(&net->ystage, sizeof(double) * net->ncore);
  if (e == cudaSuccess) e = cudaMalloc(&net->dstep, sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&net->dlr, sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost(&net->hlr, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(net->dstep, 0, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemcpy(net->params, p.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->grads, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(net->adam_m, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(net->adam_v, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(net->dstat, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "t2s2_mlp_create", __FILE__, __LINE__);
    t2s2_mlp_destroy(net);
    return e == cudaErrorMemoryAllocation ? T2S2_ENOMEM : T2S2_ECUDA;
  }
  *out = net;
  return T2S2_OK;
}

t2s2_status t2s2_mlp_destroy(t2s2_mlp net) {
  if (!net) return T2S2_OK;
  void* bufs[] = {net->params, net->grads, net->adam_m, net->adam_v, net->z1, net->h1, net->z2, net->h2,
                  net->y,      net->dy,    net->dh,     net->dz,     net->loss, net->xx, net->ws, net->dstat,
                  net->pbuf,   net->dstep, net->dlr,    net->ystage};
  for (auto& g : net->graphs) cudaGraphExecDestroy(g.exec);
  if (net->gstream) cudaStreamDestroy(net->gstream);
  if (net->gev) cudaEventDestroy(net->gev);
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (net->hbuf) cudaFreeHost(net->hbuf);
  if (net->hlr) cudaFreeHost(net->hlr);
  delete net;
  return T2S2_OK;
}

t2s2_status t2s2_mlp_info(t2s2_mlp net, long long* nparams, int* out_dim) {
  if (!net) return T2S2_EINVAL;
  if (nparams) *nparams = net->nparams;
  if (out_dim) *out_dim = net->odim;
  return T2S2_OK;
}

t2s2_status t2s2_mlp_get_params(t2s2_mlp net, float* params, float* grads, void* stream) {
  if (!net) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(float) * net->nparams;
  if (params) T2S2_CUDA_TRY(cudaMemcpyAsync(params, net->params, bytes, cudaMemcpyDefault, st));
  if (grads) T2S2_CUDA_TRY(cudaMemcpyAsync(grads, net->grads, bytes, cudaMemcpyDefault, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  return T2S2_OK;
}

t2s2_status t2s2_mlp_set_params(t2s2_mlp net, const float* params, void* stream) {
  if (!net || !params) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  T2S2_CUDA_TRY(cudaMemcpyAsync(net->params, params, sizeof(float) * net->nparams, cudaMemcpyDefault, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  return T2S2_OK;
}

t2s2_status t2s2_mlp_pack_target(t2s2_mlp net, t2s2_op op, const t2s2_tt* u, float* slot, float* uu,
                                 void* stream) {
  if (!net || !op || !u || !slot || !uu || u->d != net->d || u->loc != T2S2_DEVICE) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, u));
  for (int k = 0; k < net->d; ++k) {
    if (u->m[k] != net->m[k]) return T2S2_EINVAL;
    if (u->r[k + 1] > net->ru) return T2S2_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long per = (long)net->ru * net->mmax * net->ru;
  for (int k = 0; k < net->d; ++k) {
    pack_core_kernel<<<ew_blocks(per), 256, 0, st>>>(slot + k * per, static_cast<const double*>(u->cores[k]),
                                                     u->r[k], u->m[k], u->r[k + 1], net->ru, net->mmax);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  double nrm = 0.0;
  T2S2_TRY(t2s2_norm(op, u, &nrm, stream));
  const float v = (float)(nrm * nrm);
  T2S2_CUDA_TRY(cudaMemcpyAsync(uu, &v, sizeof(float), cudaMemcpyHostToDevice, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  return T2S2_OK;
}

t2s2_status t2s2_mlp_loss_grad(t2s2_mlp net, const float* P, int batch, const float* targets, const float* uu,
                               float* loss, void* stream) {
  if (!net || !P || !targets || !uu || batch < 1) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  T2S2_TRY(ensure_batch(net, batch));
  T2S2_CUDA_TRY(cudaMemsetAsync(net->dstat, 0, sizeof(int), st));
  T2S2_TRY(loss_grad(net, P, batch, targets, uu, st));
  float l = 0.f;
  T2S2_TRY(mean_loss(net, batch, &l, st));
  if (loss) *loss = l;
  return T2S2_OK;
}

t2s2_status t2s2_mlp_calibrate_scale(t2s2_mlp net, const float* P, int batch, const float* targets,
                                     const float* uu, float* shift, void* stream) {
  if (!net || !P || !targets || !uu || batch < 1) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  T2S2_TRY(ensure_batch(net, batch));
  T2S2_CUDA_TRY(cudaMemsetAsync(net->dstat, 0, sizeof(int), st));
  T2S2_TRY(loss_grad(net, P, batch, targets, uu, st));
  std::vector<float> hx(batch), hu(batch);
  T2S2_CUDA_TRY(cudaMemcpyAsync(hx.data(), net->xx, sizeof(float) * batch, cudaMemcpyDeviceToHost, st));
  T2S2_CUDA_TRY(cudaMemcpyAsync(hu.data(), uu, sizeof(float) * batch, cudaMemcpyDeviceToHost, st));
  T2S2_TRY(check_status(net, st));
  double sx = 0.0, su = 0.0;
  for (int i = 0; i < batch; ++i) sx += hx[i], su += hu[i];
  if (!(sx > 0.0) || !(su > 0.0)) return T2S2_EINVAL;
  // sigma enters X linearly through exp(sigma): shift its bias by half the log
  // of the mean ratio <U,U> / <X,X>
  const float d_sigma = (float)(0.5 * std::log(su / sx));
  float b = 0.f;
  float* bptr = net->params + net->ob3 + net->ncore;
  T2S2_CUDA_TRY(cudaMemcpyAsync(&b, bptr, sizeof(float), cudaMemcpyDeviceToHost, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  b += d_sigma;
  T2S2_CUDA_TRY(cudaMemcpyAsync(bptr, &b, sizeof(float), cudaMemcpyHostToDevice, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  if (shift) *shift = d_sigma;
  return T2S2_OK;
}

t2s2_status t2s2_mlp_train_step(t2s2_mlp net, const float* P, int batch, const float* targets, const float* uu,
                                float lr, float* loss, void* stream) {
  if (!net || !P || !targets || !uu || batch < 1 || !(lr > 0.f)) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  T2S2_TRY(ensure_batch(net, batch));
  T2S2_TRY(set_lr(net, lr, st));
  T2S2_CUDA_TRY(cudaMemsetAsync(net->dstat, 0, sizeof(int), st));
  T2S2_TRY(train_launches(net, P, batch, targets, uu, st));
  net->step += 1;
  if (loss) {
    float l = 0.f;
    T2S2_TRY(mean_loss(net, batch, &l, st));
    *loss = l;
  }
  return T2S2_OK;
}

t2s2_status t2s2_mlp_train(t2s2_mlp net, const float* P, int n, const float* targets, const float* uu, int batch,
                           int steps, float lr, int use_graph, float* loss, void* stream) {
  if (!net || !P || !targets || !uu || batch < 1 || n < batch || steps < 0 || !(lr > 0.f)) return T2S2_EINVAL;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaStream_t st = caller;
  if (use_graph) {
    // the legacy default stream cannot be captured: work on the network's
    // own stream, ordered after the caller's prior work and before its later work
    if (!net->gstream) {
      T2S2_CUDA_TRY(cudaStreamCreateWithFlags(&net->gstream, cudaStreamNonBlocking));
      T2S2_CUDA_TRY(cudaEventCreateWithFlags(&net->gev, cudaEventDisableTiming));
    }
    T2S2_CUDA_TRY(cudaEventRecord(net->gev, caller));
    T2S2_CUDA_TRY(cudaStreamWaitEvent(net->gstream, net->gev, 0));
    st = net->gstream;
  }
  T2S2_TRY(ensure_batch(net, batch));
  T2S2_TRY(set_lr(net, lr, st));
  T2S2_CUDA_TRY(cudaMemsetAsync(net->dstat, 0, sizeof(int), st));
  const long per = (long)net->d * net->ru * net->mmax * net->ru;
  const int slots = n - batch + 1;
  int last_lo = 0;
  for (int i = 0; i < steps; ++i) {
    const int lo = (int)(((long)i * batch) % slots);
    last_lo = lo;
    const float* Pb = P + (long)lo * net->in_dim;
    const float* Tb = targets + (long)lo * per;
    const float* Ub = uu + lo;
    if (!use_graph) {
      T2S2_TRY(train_launches(net, Pb, batch, Tb, Ub, st));
    } else {
      cudaGraphExec_t exec = nullptr;
      for (auto& e : net->graphs)
        if (e.P == Pb && e.targets == Tb && e.uu == Ub && e.batch == batch) exec = e.exec;
      if (exec) {
        T2S2_CUDA_TRY(cudaGraphLaunch(exec, st));
      } else {
        // the first visit of a minibatch runs eagerly (sizing every workspace,
        // so that nothing is allocated during capture), then the same launch
        // sequence is captured for the later visits
        T2S2_TRY(train_launches(net, Pb, batch, Tb, Ub, st));
        cudaGraph_t graph = nullptr;
        T2S2_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const t2s2_status cs = train_launches(net, Pb, batch, Tb, Ub, st);
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (cs != T2S2_OK) {
          if (graph) cudaGraphDestroy(graph);
          return cs;
        }
        T2S2_CUDA_TRY(ce);
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        T2S2_CUDA_TRY(ie);
        net->graphs.push_back({Pb, Tb, Ub, batch, exec});
      }
    }
    net->step += 1;
  }
  if (loss) {
    // the per-sample losses of the last step's minibatch
    float l = 0.f;
    T2S2_TRY(mean_loss(net, batch, &l, st));
    *loss = l;
    (void)last_lo;
  } else {
    T2S2_TRY(check_status(net, st));
  }
  if (st != caller) {
    T2S2_CUDA_TRY(cudaEventRecord(net->gev, st));
    T2S2_CUDA_TRY(cudaStreamWaitEvent(caller, net->gev, 0));
  }
  return T2S2_OK;
}

t2s2_status t2s2_mlp_init_output(t2s2_mlp net, t2s2_op op, const t2s2_tt* u, float weight_scale, void* stream) {
  if (!net || !op || !u || u->d != net->d || !std::isfinite(weight_scale)) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, u));
  for (int k = 0; k < net->d; ++k)
    if (u->m[k] != net->m[k]) return T2S2_EINVAL;
  const size_t mc = max_core(u);
  T2S2_TRY(ensure_arena(op, tt_bytes(u) * 3 + 10 * mc * sizeof(double) + ((size_t)8 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT du, v;
  T2S2_TRY(bind_tt(cx, u, du, true));
  int rc = 1;
  for (int k = 0; k <= u->d; ++k) rc = std::max(rc, u->r[k]);
  T2S2_TRY(tt_alloc(cx, v, du.d, du.m, du.r, rc));
  T2S2_TRY(tt_copy(cx, du, v));
  // u rounded to the network's rank (FP64 rounding, no tolerance)
  T2S2_TRY(tt_round(cx, v, 0.0, net->r));
  for (int k = 1; k < net->d; ++k)
    if (v.r[k] > net->r) return T2S2_EINVAL;
  for (int k = 0; k < net->d; ++k) {
    const int na = k == 0 ? 1 : net->r, nb = k == net->d - 1 ? 1 : net->r;
    const long n = (long)na * net->m[k] * nb;
    bias_core_kernel<<<ew_blocks(n), 256, 0, cx.st>>>(net->params + net->ob3 + net->off[k], v.c[k], v.r[k],
                                                     net->m[k], v.r[k + 1], na, nb);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  const long nw = (long)net->odim * net->hidden;
  scale_kernel<<<ew_blocks(nw), 256, 0, cx.st>>>(net->params + net->oW3, nw, weight_scale);
  T2S2_CUDA_TRY(cudaGetLastError());
  // the log-scale output starts at zero (0.0f is all zero bits)
  T2S2_CUDA_TRY(cudaMemsetAsync(net->params + net->ob3 + net->ncore, 0, sizeof(float), cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  return T2S2_OK;
}

t2s2_status t2s2_mlp_predict(t2s2_mlp net, const float* p, t2s2_tt* x, void* stream) {
  if (!net || !p || !x || x->d != net->d || !x->r || !x->cores || !x->cap) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t psmem = predict_smem_bytes(net->in_dim, net->hidden, net->odim);
  if (x->loc == T2S2_DEVICE && psmem <= kPredictMaxSmem) {
    // one launch, written straight into the caller's device cores; stream
    // ordered (no synchronisation)
    PredictArgs a;
    for (int k = 0; k < net->d; ++k) {
      const int ra = k == 0 ? 1 : net->r, rb = k == net->d - 1 ? 1 : net->r;
      if ((size_t)ra * net->m[k] * rb > x->cap[k] || (x->m && x->m[k] != net->m[k]) || !x->cores[k])
        return T2S2_EINVAL;
      a.out[k] = x->cores[k];
    }
    static bool attr = false;
    if (!attr) {
      T2S2_CUDA_TRY(cudaFuncSetAttribute(predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPredictMaxSmem));
      attr = true;
    }
    // a host input travels inside the launch arguments (no copy); a device
    // input is read where it is
    cudaPointerAttributes pa;
    const bool on_device = cudaPointerGetAttributes(&pa, p) == cudaSuccess &&
                           (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    (void)cudaGetLastError();  // a plain host pointer may leave an error behind on older runtimes
    if (on_device || net->in_dim > kPredictInline) {
      if (!on_device) T2S2_CUDA_TRY(cudaMemcpyAsync(net->pbuf, p, sizeof(float) * net->in_dim, cudaMemcpyDefault, st));
      a.p = on_device ? p : net->pbuf;
    } else {
      a.p = nullptr;
      std::memcpy(a.pin, p, sizeof(float) * net->in_dim);
    }
    a.w = net->params;
    a.oW1 = net->oW1; a.ob1 = net->ob1; a.oW2 = net->oW2; a.ob2 = net->ob2; a.oW3 = net->oW3; a.ob3 = net->ob3;
    a.in_dim = net->in_dim; a.hidden = net->hidden; a.odim = net->odim; a.ncore = net->ncore; a.d = net->d;
    for (int k = 0; k <= net->d; ++k) a.off[k] = net->off[k];
    {
      const double h = net->hidden;
      TraceScope ts(kTrMlp, st, 2.0 * h * (net->in_dim + h + net->odim), 4.0 * h * (net->in_dim + h + net->odim));
      predict_kernel<<<1, kPredictThreads, psmem, st>>>(a);
      T2S2_CUDA_TRY(cudaGetLastError());
    }
    x->r[0] = 1;
    for (int k = 1; k < net->d; ++k) x->r[k] = net->r;
    x->r[net->d] = 1;
    return T2S2_OK;
  }
  T2S2_TRY(ensure_batch(net, 1));
  float* dp = net->pbuf;
  T2S2_CUDA_TRY(cudaMemcpyAsync(dp, p, sizeof(float) * net->in_dim, cudaMemcpyDefault, st));
  T2S2_CUDA_TRY(cudaMemsetAsync(net->dstat, 0, sizeof(int), st));
  T2S2_TRY(forward(net, dp, 1, st));
  {
    UnpackArgs u;
    u.y = net->y;
    u.out = net->ystage;
    for (int k = 0; k <= net->d; ++k) u.off[k] = net->off[k];
    u.ncore = net->ncore;
    TraceScope ts(kTrMlp, st, 3.0 * net->ncore, 12.0 * net->ncore);
    unpack_cores_kernel<<<net->d, 256, 0, st>>>(u);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  for (int k = 0; k < net->d; ++k) {
    const int ra = k == 0 ? 1 : net->r, rb = k == net->d - 1 ? 1 : net->r;
    const long n = (long)ra * net->m[k] * rb;
    if ((size_t)n > x->cap[k] || (x->m && x->m[k] != net->m[k])) return T2S2_EINVAL;
    T2S2_CUDA_TRY(cudaMemcpyAsync(x->cores[k], net->ystage + net->off[k], sizeof(double) * n,
                                  x->loc == T2S2_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  x->r[0] = 1;
  for (int k = 1; k < net->d; ++k) x->r[k] = net->r;
  x->r[net->d] = 1;
  return check_status(net, st);
}

}  // extern "C"
