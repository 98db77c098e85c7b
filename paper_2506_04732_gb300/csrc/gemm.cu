// Tiled SIMT GEMM for the small dense contractions of the TT sweeps.
// 64x64 output tile per CTA, 256 threads with a 4x4 register micro-tile,
// K staged through shared memory in slices of 16.  Used for FP64 work, whose
// throughput on sm_103 is bounded by the DFMA pipe rather than by memory.
#include "gemm.h"
#include "trace.h"

namespace t2s2 {

namespace {
constexpr int BK = 16, NT = 256;

// Tile of (16*TM) x (16*TN) outputs; 16 x 16 threads, each a TM x TN micro-tile.
template <typename T, int TM, int TN>
__global__ void __launch_bounds__(NT) gemm_kernel(Gemm<T> g, int splits, int kchunk, T* ws) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int bz = blockIdx.z;
  const int b = bz / splits, sidx = bz % splits;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int k_begin = sidx * kchunk;
  const int k_end = min(g.K, k_begin + kchunk);
  const T* A = g.A + (long)b * g.sA;
  const T* B = g.B + (long)b * g.sB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;

  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += NT) {
      int mm, kk;
      if (g.tA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      int gm = m0 + mm, gk = k0 + kk;
      T v = 0;
      if (gm < g.M && gk < k_end) v = g.tA ? A[(long)gk * g.lda + gm] : A[(long)gm * g.lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += NT) {
      int nn, kk;
      if (g.tB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int gn = n0 + nn, gk = k0 + kk;
      T v = 0;
      if (gn < g.N && gk < k_end) v = g.tB ? B[(long)gn * g.ldb + gk] : B[(long)gk * g.ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splits == 1) {
    T* C = g.C + (long)b * g.sC;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int gm = m0 + ty + 16 * i;
      if (gm >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        T* c = C + (long)gm * g.ldc + gn;
        T v = g.alpha * acc[i][j];
        if (g.beta != T(0)) v = fma(g.beta, *c, v);
        *c = v;
      }
    }
  } else {
    T* P = ws + ((long)sidx * g.batch + b) * (long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int gm = m0 + ty + 16 * i;
      if (gm >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn < g.N) P[(long)gm * g.N + gn] = acc[i][j];
      }
    }
  }
}

template <typename T>
__global__ void splitk_reduce(Gemm<T> g, int splits, const T* ws) {
  long total = (long)g.batch * g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long b = e / ((long)g.M * g.N);
    long rem = e % ((long)g.M * g.N);
    int gm = (int)(rem / g.N), gn = (int)(rem % g.N);
    T s = 0;
    for (int p = 0; p < splits; ++p) s += ws[((long)p * g.batch + b) * (long)g.M * g.N + rem];
    T* c = g.C + b * g.sC + (long)gm * g.ldc + gn;
    T v = g.alpha * s;
    if (g.beta != T(0)) v = fma(g.beta, *c, v);
    *c = v;
  }
}

inline int tile_code(int x) { return x <= 16 ? 1 : (x <= 32 ? 2 : 4); }

// Tile shape and split-K.  FP64 runs at 2 DFMA/clk/SM on this part, so a
// CTA's time is about BM*BN*K/2 cycles: start from tiles that fit M and N,
// then halve the larger tile side while the grid has fewer CTAs than SMs, and
// finally split long K over the SMs.
struct TilePlan {
  int tm, tn, splits, kc;
};

template <typename T>
TilePlan plan_tiles(const Gemm<T>& g) {
  TilePlan p{tile_code(g.M), tile_code(g.N), 1, g.K};
  auto tiles = [&]() { return (long)cdiv(g.M, 16 * p.tm) * cdiv(g.N, 16 * p.tn) * g.batch; };
  if (sizeof(T) == 8) {
    while (tiles() < kNumSMs && (p.tm > 1 || p.tn > 1)) {
      if (p.tm >= p.tn) p.tm /= 2; else p.tn /= 2;
    }
  }
  if (g.K <= 0) {
    p.kc = 0;
    return p;
  }
  const long t = tiles();
  const long target = (sizeof(T) == 8) ? 2L * kNumSMs : kNumSMs;
  if (t < target && g.K > 2 * BK) {
    long want = (target + t - 1) / t;
    long maxs = g.K / (2 * BK);
    p.splits = (int)std::max(1L, std::min(std::min(want, maxs), 128L));
  }
  int kc = cdiv(g.K, p.splits);
  kc = cdiv(kc, BK) * BK;
  p.splits = cdiv(g.K, kc);
  p.kc = kc;
  return p;
}

template <typename T, int TM, int TN>
void launch_tile(const Gemm<T>& g, int splits, int kc, T* ws, cudaStream_t st) {
  dim3 grid(cdiv(g.N, 16 * TN), cdiv(g.M, 16 * TM), g.batch * splits);
  gemm_kernel<T, TM, TN><<<grid, NT, 0, st>>>(g, splits, std::max(kc, 1), ws);
}

template <typename T>
void launch_any(const Gemm<T>& g, int tm, int tn, int splits, int kc, T* ws, cudaStream_t st) {
#define T2S2_TILE(a, b) if (tm == a && tn == b) { launch_tile<T, a, b>(g, splits, kc, ws, st); return; }
  T2S2_TILE(1, 1) T2S2_TILE(1, 2) T2S2_TILE(1, 4)
  T2S2_TILE(2, 1) T2S2_TILE(2, 2) T2S2_TILE(2, 4)
  T2S2_TILE(4, 1) T2S2_TILE(4, 2) T2S2_TILE(4, 4)
#undef T2S2_TILE
}
}  // namespace

template <typename T>
size_t gemm_workspace(const Gemm<T>& g) {
  const TilePlan p = plan_tiles(g);
  return p.splits > 1 ? (size_t)p.splits * g.batch * g.M * g.N : 0;
}

template <typename T>
t2s2_status gemm(const Gemm<T>& g, T* ws, size_t ws_elems, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return T2S2_OK;
  const TilePlan plan = plan_tiles(g);
  int splits = plan.splits, kc = plan.kc;
  if (splits > 1 && (ws == nullptr || ws_elems < (size_t)splits * g.batch * g.M * g.N)) {
    splits = 1;
    kc = g.K;
  }
  if (g.batch * (long)splits > 65535L) return T2S2_EINVAL;
  {
    const double fl = 2.0 * g.M * g.N * (double)g.K * g.batch;
    const double by = (double)sizeof(T) * g.batch * ((double)g.M * g.K + (double)g.K * g.N + 2.0 * g.M * g.N);
    TraceScope ts(kTrGemm, st, fl, by);
    launch_any<T>(g, plan.tm, plan.tn, splits, kc, ws, st);
  }
  T2S2_CUDA_TRY(cudaGetLastError());
  if (splits > 1) {
    long total = (long)g.batch * g.M * g.N;
    int blocks = (int)std::min<long>(cdiv(total, 256), 4L * kNumSMs);
    TraceScope ts(kTrElem, st, 0.0, (double)sizeof(T) * total * (splits + 2));
    splitk_reduce<T><<<blocks, 256, 0, st>>>(g, splits, ws);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  return T2S2_OK;
}

template size_t gemm_workspace<double>(const Gemm<double>&);
template size_t gemm_workspace<float>(const Gemm<float>&);
template t2s2_status gemm<double>(const Gemm<double>&, double*, size_t, cudaStream_t);
template t2s2_status gemm<float>(const Gemm<float>&, float*, size_t, cudaStream_t);

}  // namespace t2s2
