// Tiled SIMT GEMM for the small dense contractions of the TT sweeps.
//
// Two kernels.  gemm_kernel: up to 64x64 outputs per CTA, 256 threads with a
// register micro-tile, K staged through shared memory in slices of 16; for
// larger products and for FP32.  small_kernel: the FP64 contractions of the
// sweeps (M, N of a few tens to a few hundreds, K from ~10 to ~1000) cost
// ~0.3 MFLOP each -- a quarter of a microsecond of the whole GPU's binary64
// rate -- so their time is latency: one output per thread, 8x8 to 16x16
// thread tiles chosen so that the grid covers the SMs, K in slices of 32,
// and long K split over CTAs with the partial sums added, in split order, by
// the last CTA of each tile to arrive (a per-tile counter that the adding CTA
// resets), so no second launch is needed and the result does not depend on
// timing.
#include <type_traits>

#include "gemm.h"
#include "trace.h"

namespace t2s2 {

namespace {
constexpr int BK = 16, NT = 256;

// Tile of (16*TM) x (16*TN) outputs; 16 x 16 threads, each a TM x TN micro-tile.
template <typename T, int TM, int TN>
__global__ void __launch_bounds__(NT) gemm_kernel(Gemm<T> g, int splits, int kchunk, T* ws) {
  pdl_wait();
  pdl_trigger();
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
  pdl_wait();
  pdl_trigger();
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

// 256 threads on a BM x BN output tile: KG = 256 / (BM BN) threads share an
// output, each taking every KG-th k of a slice of SBK with two accumulators,
// so that the dependent chain per thread is SBK / (2 KG) binary64 FMAs (each
// ~150 cycles of latency on this part).  The KG partial sums are added in a
// fixed order.  With splits > 1 the CTA of split s writes its partial tile to
// ws[s], and the last CTA of the tile to finish (counter cnt[tile]) adds the
// partials in split order.
constexpr int SBK = 64, SNT = 256;

// One BM x BN tile (column tile nt, row tile mt) of batch entry / split bz;
// tiles_m x tiles_n tiles per batch entry (the counter index of the tile).
template <int BM, int BN>
__device__ __forceinline__ void small_tile(const Gemm<double>& g, int splits, int kchunk, double* ws, int* cnt,
                                           int nt, int mt, int bz, int tiles_m, int tiles_n) {
  constexpr int NO = BM * BN, KG = SNT / NO;
  static_assert(NO * KG == SNT, "tile must divide the CTA");
  __shared__ double As[SBK][BM + 1];
  __shared__ double Bs[SBK][BN + 1];
  __shared__ double red[KG][NO];
  __shared__ int last;
  const int b = bz / splits, sidx = bz % splits;
  const int m0 = mt * BM, n0 = nt * BN;
  const int k_begin = sidx * kchunk;
  const int k_end = min(g.K, k_begin + kchunk);
  const double* A = g.A + (long)b * g.sA;
  const double* B = g.B + (long)b * g.sB;
  const int t = threadIdx.x, o = t % NO, kg = t / NO, tx = o % BN, ty = o / BN;
  double acc0 = 0.0, acc1 = 0.0;
  for (int k0 = k_begin; k0 < k_end; k0 += SBK) {
    const int kn = min(SBK, k_end - k0);
    for (int e = t; e < BM * kn; e += SNT) {
      int mm, kk;
      if (g.tA) { mm = e % BM; kk = e / BM; } else { kk = e % kn; mm = e / kn; }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < g.M) v = g.tA ? A[(long)gk * g.lda + gm] : A[(long)gm * g.lda + gk];
      As[kk][mm] = v;
    }
    for (int e = t; e < BN * kn; e += SNT) {
      int nn, kk;
      if (g.tB) { kk = e % kn; nn = e / kn; } else { nn = e % BN; kk = e / BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < g.N) v = g.tB ? B[(long)gn * g.ldb + gk] : B[(long)gk * g.ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
    int kk = kg;
    for (; kk + KG < kn; kk += 2 * KG) {
      acc0 = fma(As[kk][ty], Bs[kk][tx], acc0);
      acc1 = fma(As[kk + KG][ty], Bs[kk + KG][tx], acc1);
    }
    if (kk < kn) acc0 = fma(As[kk][ty], Bs[kk][tx], acc0);
    __syncthreads();
  }
  red[kg][o] = acc0 + acc1;
  __syncthreads();
  const int gm = m0 + ty, gn = n0 + tx;
  const bool in = kg == 0 && gm < g.M && gn < g.N;
  double acc = 0.0;
  if (kg == 0)
#pragma unroll
    for (int q = 0; q < KG; ++q) acc += red[q][o];
  const long mn = (long)g.M * g.N;
  if (splits == 1) {
    if (in) {
      double* c = g.C + (long)b * g.sC + (long)gm * g.ldc + gn;
      double v = g.alpha * acc;
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
    return;
  }
  if (in) ws[((long)sidx * g.batch + b) * mn + (long)gm * g.N + gn] = acc;
  if (!cnt) return;  // the caller adds the partials with splitk_reduce
  __threadfence();
  __syncthreads();
  const long tile = ((long)b * tiles_m + mt) * tiles_n + nt;
  if (t == 0) last = (atomicAdd(cnt + tile, 1) == splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // partials q = kg, kg + KG, ... per thread, then the KG sums in order
  double s = 0.0;
  if (gm < g.M && gn < g.N) {
    const volatile double* p = ws + (long)b * mn + (long)gm * g.N + gn;
    for (int q = kg; q < splits; q += KG) s += p[(long)q * g.batch * mn];
  }
  red[kg][o] = s;
  __syncthreads();
  if (in) {
    double tot = 0.0;
#pragma unroll
    for (int q = 0; q < KG; ++q) tot += red[q][o];
    double* c = g.C + (long)b * g.sC + (long)gm * g.ldc + gn;
    double v = g.alpha * tot;
    if (g.beta != 0.0) v = fma(g.beta, *c, v);
    *c = v;
  }
  if (t == 0) cnt[tile] = 0;  // ready for the next launch on this stream
}

template <int BM, int BN>
__global__ void __launch_bounds__(SNT) small_kernel(Gemm<double> g, int splits, int kchunk, double* ws,
                                                    int* cnt) {
  pdl_wait();
  pdl_trigger();
  small_tile<BM, BN>(g, splits, kchunk, ws, cnt, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.y, gridDim.x);
}

// Independent GEMMs of one group in one launch: CTA ranges start[i] ..
// start[i+1] belong to GEMM i, each with its own split plan, workspace and
// counter range.
struct GroupArgs {
  int n;
  Gemm<double> g[kMaxGroup];
  int splits[kMaxGroup], kc[kMaxGroup], tm[kMaxGroup], tn[kMaxGroup];
  long start[kMaxGroup + 1];
  long wsoff[kMaxGroup], cntoff[kMaxGroup];
  double* ws;
  int* cnt;
};

template <int BM, int BN>
__global__ void __launch_bounds__(SNT) small_group_kernel(GroupArgs a) {
  pdl_wait();
  pdl_trigger();
  const long bid = blockIdx.x;
  int i = 0;
  while (i + 1 < a.n && bid >= a.start[i + 1]) ++i;
  long q = bid - a.start[i];
  const int nt = (int)(q % a.tn[i]);
  q /= a.tn[i];
  const int mt = (int)(q % a.tm[i]);
  const int bz = (int)(q / a.tm[i]);
  small_tile<BM, BN>(a.g[i], a.splits[i], a.kc[i], a.ws + a.wsoff[i], a.cnt + a.cntoff[i], nt, mt, bz, a.tm[i],
                     a.tn[i]);
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

// Plan of the small FP64 kernel from a latency model (cycles on one SM):
// the dependent FMA chain of a thread (~150 cycles per binary64 FMA), one
// global-load round trip per K slice (~800), the cross-CTA addition when K is
// split, and the binary64 issue limit of the busiest SM (2 FMAs per cycle).
struct SmallPlan {
  bool use;
  int bm, bn, splits, kc;
};
constexpr double kSmallMaxFmas = 16e6;
constexpr int kShapes[][2] = {{16, 16}, {8, 16}, {16, 8}, {8, 8}, {4, 16}, {16, 4},
                              {1, 64},  {64, 1}, {4, 4}};

// Best split of g for tile shape bm x bn under the latency model; returns
// its cost (cycles) and fills splits / kc.
double plan_shape(const Gemm<double>& g, int bm, int bn, int* splits, int* kcout) {
  const int kgr = SNT / (bm * bn);
  const long tiles = (long)cdiv(g.M, bm) * cdiv(g.N, bn) * g.batch;
  if (g.K <= 0) {
    *splits = 1;
    *kcout = 0;
    return 900.0;
  }
  double best = 1e300;
  const int maxs = (int)std::min<long>(64, std::max(1, cdiv(g.K, 32)));
  for (int s = 1; s <= maxs; s = (s < 4 ? s + 1 : s * 2)) {
    if ((long)g.batch * s > 65535L) break;
    const int kc = cdiv(cdiv(g.K, s), 8) * 8;
    const int sp = cdiv(g.K, kc);
    const double chain = 150.0 * ((double)kc / (2.0 * kgr) + kgr);
    const double loads = 800.0 * cdiv(kc, SBK);
    const double reduce = sp > 1 ? 900.0 + 150.0 * ((double)sp / kgr + kgr) : 0.0;
    const long ctas = tiles * sp;
    const double issue = (double)((ctas + kNumSMs - 1) / kNumSMs) * bm * bn * (double)kc / 2.0;
    const double cost = std::max(chain + loads, issue) + reduce;
    if (cost < best * 0.98) {
      best = cost;
      *splits = sp;
      *kcout = kc;
    }
  }
  return best;
}

SmallPlan plan_small(const Gemm<double>& g) {
  SmallPlan best{false, 8, 8, 1, g.K};
  if ((double)g.M * g.N * (double)std::max(g.K, 1) * g.batch > kSmallMaxFmas) return best;
  best.use = true;
  double best_cost = 1e300;
  for (auto& sh : kShapes) {
    int sp = 1, kc = 0;
    const double cost = plan_shape(g, sh[0], sh[1], &sp, &kc);
    if (cost < best_cost * 0.98) {
      best_cost = cost;
      best.bm = sh[0];
      best.bn = sh[1];
      best.splits = sp;
      best.kc = kc;
    }
  }
  return best;
}

void launch_small(const Gemm<double>& g, const SmallPlan& p, double* ws, int* cnt, cudaStream_t st) {
  dim3 grid(cdiv(g.N, p.bn), cdiv(g.M, p.bm), g.batch * p.splits);
  const int kc = std::max(p.kc, 1);
#define T2S2_SMALL(a, b) \
  if (p.bm == a && p.bn == b) { (void)launch_pdl(small_kernel<a, b>, grid, SNT, 0, st, g, p.splits, kc, ws, cnt); return; }
  T2S2_SMALL(16, 16) T2S2_SMALL(8, 16) T2S2_SMALL(16, 8) T2S2_SMALL(8, 8) T2S2_SMALL(4, 16)
  T2S2_SMALL(16, 4) T2S2_SMALL(1, 64) T2S2_SMALL(64, 1) T2S2_SMALL(4, 4)
#undef T2S2_SMALL
}

void launch_group(const GroupArgs& a, int bm, int bn, cudaStream_t st) {
  const long ctas = a.start[a.n];
#define T2S2_GROUP(x, y) \
  if (bm == x && bn == y) { (void)launch_pdl(small_group_kernel<x, y>, (unsigned)ctas, SNT, 0, st, a); return; }
  T2S2_GROUP(16, 16) T2S2_GROUP(8, 16) T2S2_GROUP(16, 8) T2S2_GROUP(8, 8) T2S2_GROUP(4, 16)
  T2S2_GROUP(16, 4) T2S2_GROUP(1, 64) T2S2_GROUP(64, 1) T2S2_GROUP(4, 4)
#undef T2S2_GROUP
}

// Shape of a group: the tile shape whose worst member cost is least.
struct GroupPlan {
  bool ok;
  int bm, bn;
  int splits[kMaxGroup], kc[kMaxGroup];
};

GroupPlan plan_group(const Gemm<double>* gs, int n) {
  GroupPlan gp;
  gp.ok = false;
  gp.bm = gp.bn = 8;
  for (int i = 0; i < n; ++i)
    if ((double)gs[i].M * gs[i].N * (double)std::max(gs[i].K, 1) * gs[i].batch > kSmallMaxFmas) return gp;
  double best = 1e300;
  for (auto& sh : kShapes) {
    double worst = 0.0;
    int sp[kMaxGroup], kc[kMaxGroup];
    for (int i = 0; i < n; ++i) worst = std::max(worst, plan_shape(gs[i], sh[0], sh[1], &sp[i], &kc[i]));
    if (worst < best * 0.98) {
      best = worst;
      gp.bm = sh[0];
      gp.bn = sh[1];
      for (int i = 0; i < n; ++i) gp.splits[i] = sp[i], gp.kc[i] = kc[i];
    }
  }
  gp.ok = true;
  return gp;
}

template <typename T, int TM, int TN>
void launch_tile(const Gemm<T>& g, int splits, int kc, T* ws, cudaStream_t st) {
  dim3 grid(cdiv(g.N, 16 * TN), cdiv(g.M, 16 * TM), g.batch * splits);
  (void)launch_pdl(gemm_kernel<T, TM, TN>, grid, NT, 0, st, g, splits, std::max(kc, 1), ws);
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
  if constexpr (std::is_same<T, double>::value) {
    const SmallPlan sp = plan_small(g);
    if (sp.use) return sp.splits > 1 ? (size_t)sp.splits * g.batch * g.M * g.N : 0;
  }
  const TilePlan p = plan_tiles(g);
  return p.splits > 1 ? (size_t)p.splits * g.batch * g.M * g.N : 0;
}

template <typename T>
t2s2_status gemm(const Gemm<T>& g, T* ws, size_t ws_elems, cudaStream_t st, int* cnt, long ncnt) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return T2S2_OK;
  const double fl = 2.0 * g.M * g.N * (double)g.K * g.batch;
  const double by = (double)sizeof(T) * g.batch * ((double)g.M * g.K + (double)g.K * g.N + 2.0 * g.M * g.N);
  if constexpr (std::is_same<T, double>::value) {
    SmallPlan sp = plan_small(g);
    if (sp.use) {
      if (sp.splits > 1 && (ws == nullptr || ws_elems < (size_t)sp.splits * g.batch * g.M * g.N)) {
        sp.splits = 1;
        sp.kc = g.K;
      }
      if (g.batch * (long)sp.splits > 65535L) return T2S2_EINVAL;
      const long tiles = (long)cdiv(g.M, sp.bm) * cdiv(g.N, sp.bn) * g.batch;
      int* c = (sp.splits > 1 && cnt && tiles <= ncnt) ? cnt : nullptr;
      {
        TraceScope ts(kTrGemm, st, fl, by);
        launch_small(g, sp, ws, c, st);
      }
      T2S2_CUDA_TRY(cudaGetLastError());
      if (sp.splits > 1 && !c) {
        const long total = (long)g.batch * g.M * g.N;
        const int blocks = (int)std::min<long>(cdiv(total, 256), 4L * kNumSMs);
        TraceScope ts(kTrElem, st, 0.0, (double)sizeof(T) * total * (sp.splits + 2));
        (void)launch_pdl(splitk_reduce<T>, blocks, 256, 0, st, g, sp.splits, ws);
        T2S2_CUDA_TRY(cudaGetLastError());
      }
      return T2S2_OK;
    }
  }
  const TilePlan plan = plan_tiles(g);
  int splits = plan.splits, kc = plan.kc;
  if (splits > 1 && (ws == nullptr || ws_elems < (size_t)splits * g.batch * g.M * g.N)) {
    splits = 1;
    kc = g.K;
  }
  if (g.batch * (long)splits > 65535L) return T2S2_EINVAL;
  {
    TraceScope ts(kTrGemm, st, fl, by);
    launch_any<T>(g, plan.tm, plan.tn, splits, kc, ws, st);
  }
  T2S2_CUDA_TRY(cudaGetLastError());
  if (splits > 1) {
    long total = (long)g.batch * g.M * g.N;
    int blocks = (int)std::min<long>(cdiv(total, 256), 4L * kNumSMs);
    TraceScope ts(kTrElem, st, 0.0, (double)sizeof(T) * total * (splits + 2));
    (void)launch_pdl(splitk_reduce<T>, blocks, 256, 0, st, g, splits, ws);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  return T2S2_OK;
}

size_t gemm_group_workspace(const Gemm<double>* gs, int n) {
  if (n < 1 || n > kMaxGroup) return 0;
  const GroupPlan gp = plan_group(gs, n);
  if (!gp.ok) return 0;
  size_t w = 0;
  for (int i = 0; i < n; ++i)
    if (gp.splits[i] > 1) w += (size_t)gp.splits[i] * gs[i].batch * gs[i].M * gs[i].N;
  return w;
}

t2s2_status gemm_group(const Gemm<double>* gs, int n, double* ws, size_t ws_elems, cudaStream_t st, int* cnt,
                       long ncnt) {
  if (n < 1 || n > kMaxGroup) return T2S2_EINVAL;
  const GroupPlan gp = plan_group(gs, n);
  bool fallback = !gp.ok || !cnt;
  GroupArgs a;
  a.n = 0;
  long ctas = 0, wso = 0, cno = 0;
  double fl = 0.0, by = 0.0;
  if (!fallback) {
    for (int i = 0; i < n; ++i) {
      const Gemm<double>& g = gs[i];
      if (g.M <= 0 || g.N <= 0 || g.batch <= 0) continue;
      const int j = a.n++;
      a.g[j] = g;
      a.splits[j] = gp.splits[i];
      a.kc[j] = std::max(gp.kc[i], 1);
      a.tm[j] = cdiv(g.M, gp.bm);
      a.tn[j] = cdiv(g.N, gp.bn);
      a.start[j] = ctas;
      const long tiles = (long)a.tm[j] * a.tn[j] * g.batch;
      ctas += tiles * a.splits[j];
      a.wsoff[j] = wso;
      a.cntoff[j] = cno;
      if (a.splits[j] > 1) {
        wso += (long)a.splits[j] * g.batch * g.M * g.N;
        cno += tiles;
      }
      if ((long)g.batch * a.splits[j] > 65535L) fallback = true;
      fl += 2.0 * g.M * g.N * (double)g.K * g.batch;
      by += 8.0 * g.batch * ((double)g.M * g.K + (double)g.K * g.N + 2.0 * g.M * g.N);
    }
    a.start[a.n] = ctas;
    if ((size_t)wso > ws_elems || (wso > 0 && !ws) || cno > ncnt || ctas > (1L << 30)) fallback = true;
  }
  if (fallback) {
    // one launch per product, in stream order, each reusing the workspace
    // (a product whose split does not fit runs unsplit)
    for (int i = 0; i < n; ++i) T2S2_TRY(gemm(gs[i], ws, ws ? ws_elems : 0, st, cnt, ncnt));
    return T2S2_OK;
  }
  if (a.n == 0) return T2S2_OK;
  a.ws = ws;
  a.cnt = cnt;
  {
    TraceScope ts(kTrGemm, st, fl, by);
    launch_group(a, gp.bm, gp.bn, st);
  }
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

template size_t gemm_workspace<double>(const Gemm<double>&);
template size_t gemm_workspace<float>(const Gemm<float>&);
template t2s2_status gemm<double>(const Gemm<double>&, double*, size_t, cudaStream_t, int*, long);
template t2s2_status gemm<float>(const Gemm<float>&, float*, size_t, cudaStream_t, int*, long);

}  // namespace t2s2
