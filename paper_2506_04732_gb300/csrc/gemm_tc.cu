// Strided-batched GEMM on tcgen05 tensor cores (the mixed-precision solver's
// contractions and the warm-start network's layers):
//   C_b = alpha * op(A_b) * op(B_b) + beta * C_b
// with FP64 or FP32 operands and result in HBM, operands rounded to BF16 or
// TF32 while they are staged in shared memory, and FP32 accumulation in TMEM.
//
// The MMA's M side (128 TMEM lanes per CTA) takes the longer of the two
// output dimensions: when N > M the kernel computes C^T = op(B)^T op(A)^T and
// writes it transposed, so small-by-large products of the sweep (r x (m r)
// mode products, r x r interface updates over long K) do not waste 128-row
// tiles.  Each K stage (one 128-byte swizzle row: 64 BF16 / 32 TF32 values)
// is loaded coalesced along whichever operand index is contiguous, rounded,
// stored in the 128-byte-swizzled K-major layout, and consumed by four MMAs
// that one thread issues; their completion is committed to an mbarrier that
// every thread waits on (bounded) before the buffer is refilled.  Long K is
// split across CTAs; the split partials (FP32) are summed in a fixed order by
// a second kernel, so results are deterministic.
#include <algorithm>

#include "gemm_tc.h"
#include "tc_common.cuh"
#include "trace.h"

namespace t2s2 {

namespace {

using namespace tc;

constexpr int kRows = 128;    // MMA M = TMEM lanes
constexpr int kThreads = 128;

template <typename T>
struct TcGemm {
  int M, N, K;  // after the optional swap: M rows (MMA M), N cols (MMA N)
  const T* R;  // row operand, element (i, k)
  long ldr, sR;
  int r_kc;  // 1: (i, k) at R[i * ldr + k]; 0: at R[k * ldr + i]
  const T* Q;  // column operand, element (j, k)
  long ldq, sQ;
  int q_kc;
  T* C;
  long ldc, sC;
  int c_trans;  // 1: C(i, j) at C[j * ldc + i]; 0: at C[i * ldc + j]
  double alpha, beta;
  int batch, splits, kchunk;
  float* ws;  // [batch][splits][M][N] partial sums when splits > 1
};

// Shared memory per CTA for a BN-column tile: both operand tiles, alignment
// slack, and at least enough that no more CTAs fit on an SM than its 512 TMEM
// columns can serve (BN columns each).
template <int E, int BN>
constexpr int gemm_smem_bytes() {
  constexpr int tiles = (kRows + BN) * 128 + 2048;
  constexpr int max_ctas = 512 / BN;
  constexpr int floor_bytes = (228 * 1024) / (max_ctas + 1) + 1024;
  return tiles > floor_bytes ? tiles : floor_bytes;
}

template <int P, int BN, typename T>
__global__ void __launch_bounds__(kThreads) gemm_tc_kernel(TcGemm<T> g, int* err) {
  using O = Op<P>;
  constexpr int E = O::kBytes;
  constexpr int BK = 128 / E;  // K elements per stage (one swizzle row)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sR = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* sQ = sR + kRows * 128;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sQ + BN * 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int bz = blockIdx.z;
  const int b = bz / g.splits, sidx = bz % g.splits;
  const int i0 = blockIdx.x * kRows, j0 = blockIdx.y * BN;
  const int k_begin = sidx * g.kchunk;
  const int k_end = min(g.K, k_begin + g.kchunk);
  const T* R = g.R + (long)b * g.sR;
  const T* Q = g.Q + (long)b * g.sQ;

  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), BN);
  if (tid == 0) mbar_init(smem_u32(mbar), 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t bar = smem_u32(mbar);
  const uint32_t idesc = make_idesc(O::kFmt, kRows, BN);

  bool ok = true;
  int stage = 0;
  for (int k0 = k_begin; k0 < k_end; k0 += BK, ++stage) {
    if (stage > 0) {
      // the previous stage's MMAs must have read the buffer before it is refilled
      ok = __syncthreads_and(mbar_wait(bar, (stage - 1) & 1)) != 0;
      if (!ok) break;
    }
    const int kn = min(BK, k_end - k0);
    // row operand tile: 128 x BK
    if (g.r_kc) {
#pragma unroll 8
      for (int e = tid; e < kRows * BK; e += kThreads) {
        const int i = e / BK, k = e % BK;
        const int gi = i0 + i;
        const double v = (gi < g.M && k < kn) ? (double)R[(long)gi * g.ldr + (k0 + k)] : 0.0;
        O::store(sR + sw128_off<E>(i, k, kRows), v);
      }
    } else {
#pragma unroll 8
      for (int e = tid; e < kRows * BK; e += kThreads) {
        const int k = e / kRows, i = e % kRows;
        const int gi = i0 + i;
        const double v = (gi < g.M && k < kn) ? (double)R[(long)(k0 + k) * g.ldr + gi] : 0.0;
        O::store(sR + sw128_off<E>(i, k, kRows), v);
      }
    }
    // column operand tile: BN x BK
    if (g.q_kc) {
#pragma unroll 8
      for (int e = tid; e < BN * BK; e += kThreads) {
        const int j = e / BK, k = e % BK;
        const int gj = j0 + j;
        const double v = (gj < g.N && k < kn) ? (double)Q[(long)gj * g.ldq + (k0 + k)] : 0.0;
        O::store(sQ + sw128_off<E>(j, k, BN), v);
      }
    } else {
#pragma unroll 8
      for (int e = tid; e < BN * BK; e += kThreads) {
        const int k = e / BN, j = e % BN;
        const int gj = j0 + j;
        const double v = (gj < g.N && k < kn) ? (double)Q[(long)(k0 + k) * g.ldq + gj] : 0.0;
        O::store(sQ + sw128_off<E>(j, k, BN), v);
      }
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < BK; kk += O::kMmaK) {
        const uint64_t da = sdesc_sw128(smem_u32(sR) + kk * E);
        const uint64_t db = sdesc_sw128(smem_u32(sQ) + kk * E);
        issue_mma<P>(tmem, da, db, idesc, (stage > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(bar);
    }
  }
  const int nstages = stage;
  if (ok && nstages > 0) ok = __syncthreads_and(mbar_wait(bar, (nstages - 1) & 1)) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(bar, (nstages - 1) & 1);  // bounded second wait for MMAs still in flight
  }
  fence_after_sync();
  if (ok) {
    const int i = i0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      if (j0 + c0 >= g.N) break;  // warp-uniform
      uint32_t v[32];
      if (nstages > 0) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0u;  // empty K range: the product is zero
      }
      if (i >= g.M) continue;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = j0 + c0 + q;
        if (j >= g.N) break;
        const float acc = __uint_as_float(v[q]);
        if (g.splits > 1) {
          g.ws[(((long)b * g.splits + sidx) * g.M + i) * g.N + j] = acc;
        } else {
          T* c = g.C + (long)b * g.sC + (g.c_trans ? (long)j * g.ldc + i : (long)i * g.ldc + j);
          double r = g.alpha * (double)acc;
          if (g.beta != 0.0) r = fma(g.beta, (double)*c, r);
          *c = (T)r;
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// C = alpha * sum_s ws[b][s] + beta * C, summed over s in order.
template <typename T>
__global__ void splitk_sum_kernel(TcGemm<T> g) {
  const long total = (long)g.batch * g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.N);
    const long t = e / g.N;
    const int i = (int)(t % g.M);
    const int b = (int)(t / g.M);
    double s = 0.0;
    for (int p = 0; p < g.splits; ++p) s += (double)g.ws[(((long)b * g.splits + p) * g.M + i) * g.N + j];
    T* c = g.C + (long)b * g.sC + (g.c_trans ? (long)j * g.ldc + i : (long)i * g.ldc + j);
    double r = g.alpha * s;
    if (g.beta != 0.0) r = fma(g.beta, (double)*c, r);
    *c = (T)r;
  }
}

// Convert the public description into the kernel's, choosing the swap.
template <typename T>
TcGemm<T> describe(const Gemm<T>& in) {
  TcGemm<T> g{};
  const bool swap = in.N > in.M;
  g.K = in.K;
  g.alpha = in.alpha;
  g.beta = in.beta;
  g.batch = in.batch;
  g.C = in.C;
  g.ldc = in.ldc;
  g.sC = in.sC;
  // op(A)(i, k) = tA ? A[k lda + i] : A[i lda + k];  op(B)(k, j) = tB ? B[j ldb + k] : B[k ldb + j]
  if (!swap) {
    g.M = in.M; g.N = in.N;
    g.R = in.A; g.ldr = in.lda; g.sR = in.sA; g.r_kc = in.tA ? 0 : 1;
    g.Q = in.B; g.ldq = in.ldb; g.sQ = in.sB; g.q_kc = in.tB ? 1 : 0;
    g.c_trans = 0;
  } else {
    g.M = in.N; g.N = in.M;
    g.R = in.B; g.ldr = in.ldb; g.sR = in.sB; g.r_kc = in.tB ? 1 : 0;
    g.Q = in.A; g.ldq = in.lda; g.sQ = in.sA; g.q_kc = in.tA ? 0 : 1;
    g.c_trans = 1;
  }
  return g;
}

int pick_bn(int N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  return 256;
}

// Split K so that the grid reaches about two CTAs per SM.
template <typename T>
void plan_splits(TcGemm<T>& g, int bn, int bk) {
  const long tiles = (long)cdiv(g.M, kRows) * cdiv(g.N, bn) * g.batch;
  const int stages = std::max(1, cdiv(g.K, bk));
  int splits = 1;
  if (tiles < 2 * kNumSMs) splits = (int)std::min<long>(stages, std::max<long>(1, (2 * kNumSMs) / tiles));
  splits = std::min(splits, 64);
  const int per = cdiv(stages, splits);
  g.kchunk = per * bk;
  g.splits = std::max(1, cdiv(g.K, g.kchunk));
  if ((long)g.batch * g.splits > 65535) g.splits = 1, g.kchunk = std::max(g.K, 1);
}

template <int P, int BN, typename T>
t2s2_status launch(const TcGemm<T>& g, int* err, cudaStream_t st) {
  constexpr int smem = gemm_smem_bytes<Op<P>::kBytes, BN>();
  T2S2_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<P, BN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  dim3 grid(cdiv(g.M, kRows), cdiv(g.N, BN), g.batch * g.splits);
  gemm_tc_kernel<P, BN, T><<<grid, kThreads, smem, st>>>(g, err);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

template <int P, typename T>
t2s2_status launch_bn(const TcGemm<T>& g, int bn, int* err, cudaStream_t st) {
  switch (bn) {
    case 32: return launch<P, 32, T>(g, err, st);
    case 64: return launch<P, 64, T>(g, err, st);
    case 128: return launch<P, 128, T>(g, err, st);
    default: return launch<P, 256, T>(g, err, st);
  }
}

}  // namespace

template <typename T>
size_t gemm_tc_workspace_bytes(const Gemm<T>& in, int prec) {
  TcGemm<T> g = describe(in);
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return 0;
  const int bk = prec == T2S2_BF16_REFINE ? 64 : 32;
  plan_splits(g, pick_bn(g.N), bk);
  if (g.splits <= 1) return 0;
  return (size_t)g.batch * g.splits * g.M * g.N * sizeof(float);
}

template <typename T>
t2s2_status gemm_tc(const Gemm<T>& in, int prec, void* ws, size_t ws_bytes, int* err, cudaStream_t st) {
  if (prec != T2S2_BF16_REFINE && prec != T2S2_TF32_REFINE) return T2S2_EINVAL;
  if (!err || in.M < 0 || in.N < 0 || in.K < 0 || in.batch < 0) return T2S2_EINVAL;
  if (in.M == 0 || in.N == 0 || in.batch == 0) return T2S2_OK;
  TcGemm<T> g = describe(in);
  const int bk = prec == T2S2_BF16_REFINE ? 64 : 32;
  const int bn = pick_bn(g.N);
  plan_splits(g, bn, bk);
  if (g.splits > 1) {
    if (!ws || ws_bytes < gemm_tc_workspace_bytes(in, prec)) return T2S2_ENOMEM;
    g.ws = reinterpret_cast<float*>(ws);
  }
  const double fl = 2.0 * in.M * in.N * (double)in.K * in.batch;
  const double by = (double)sizeof(T) * in.batch *
                    ((double)in.M * in.K + (double)in.K * in.N + (in.beta != 0 ? 2.0 : 1.0) * in.M * in.N);
  {
    TraceScope ts(kTrGemmTc, st, fl, by);
    if (prec == T2S2_BF16_REFINE) {
      T2S2_TRY(launch_bn<T2S2_BF16_REFINE>(g, bn, err, st));
    } else {
      T2S2_TRY(launch_bn<T2S2_TF32_REFINE>(g, bn, err, st));
    }
  }
  if (g.splits > 1) {
    TraceScope ts(kTrGemmTc, st, 0.0, 0.0);
    const long total = (long)g.batch * g.M * g.N;
    const int blocks = (int)std::min<long>(cdiv(total, 256), 4L * kNumSMs);
    splitk_sum_kernel<T><<<blocks, 256, 0, st>>>(g);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  return T2S2_OK;
}

template size_t gemm_tc_workspace_bytes<double>(const Gemm<double>&, int);
template size_t gemm_tc_workspace_bytes<float>(const Gemm<float>&, int);
template t2s2_status gemm_tc<double>(const Gemm<double>&, int, void*, size_t, int*, cudaStream_t);
template t2s2_status gemm_tc<float>(const Gemm<float>&, int, void*, size_t, int*, cudaStream_t);

}  // namespace t2s2
