// TT apply of the rank-2 collocation operator on the 5th-generation tensor
// cores (tcgen05): BF16 or TF32 operands, FP32 accumulation in tensor memory.
//
// The mode-k contraction of core k is the GEMM
//     D[(a,b), ii] = sum_j X_k[a, j, b] * M2[ii, j],   M2 = [S_k ; G_k]  (2m x m),
// with the (a, b) pairs as the MMA's M dimension (128 per CTA), the 2m
// stacked operator rows as N (<= 128) and j as K (<= 64).  Both operands are
// K-major.  Each CTA rounds its slice of X (FP64 in HBM, read coalesced along
// b) and the two operator matrices to the operand type and stores them in
// shared memory in the 128-byte-swizzled canonical layout; one thread issues
// the K/kMmaK MMAs and commits their completion to an mbarrier; each warp then
// reads its 32 TMEM lanes (tcgen05.ld) and writes the FP32 sums as FP64 into
// the block pattern of Y (the same pattern as the FP64 kernel in apply.cu).
// All cores of the train go in one launch.
//
// Staged variant (kStage): the rows of X a tile needs form one contiguous
// range of the core (whole r_b-blocks of the a it touches).  One thread copies
// that range into a shared-memory stage with a one-dimensional bulk TMA copy
// (cp.async.bulk, completion counted on an mbarrier) for the NEXT tile while
// the CTA runs the current tile's MMAs and epilogue; the operand tile is then
// converted from the stage instead of from global memory.  The copy starts at
// the even element at or below the range (16-byte aligned, the cores being
// 16-byte aligned) and covers an even number of elements; an odd last element
// is read with a plain load.  Every byte copied lies inside the core.
//
// The waits on the mbarriers are bounded: on timeout the CTA sets *err, waits
// once more (bounded) for its MMAs and for a bulk copy in flight, frees its
// TMEM and returns without writing Y.
#include <algorithm>

#include "apply.h"
#include "tc_common.cuh"
#include "trace.h"

namespace t2s2 {

namespace {

using namespace tc;

constexpr int kTileM = 128;    // (a, b) rows per CTA = TMEM lanes
constexpr int kMaxK = 64;      // contraction length m (zero padded)
constexpr int kTileN = 128;    // 2m stacked rows (zero padded) = TMEM columns
constexpr int kThreads = 256;  // 8 warps: two per 32-lane TMEM quarter (column halves)
// Dynamic shared memory per CTA: the two operand tiles plus alignment slack,
// and never less than 48 KB, so that at most 4 CTAs share an SM and the
// 4 x 128 TMEM columns they allocate never exceed the SM's 512.
constexpr int smem_bytes(int elem_bytes) {
  return 2 * kTileM * kMaxK * elem_bytes + 2048 > 48 * 1024 ? 2 * kTileM * kMaxK * elem_bytes + 2048
                                                            : 48 * 1024;
}

// Where a CTA finds its work: the cores of one train in kernel parameters, or
// a device array of cores from many trains (grouped launch).  start[i] is the
// first tile of core i; start[n] the total.
struct ParamWork {
  ApplyBatch p;
  int start[T2S2_MAX_D + 1];
  __device__ int n() const { return p.ncores; }
  __device__ int first(int i) const { return start[i]; }
  __device__ ApplyCore core(int i) const { return p.c[i]; }
};
struct GlobalWork {
  const ApplyCore* c;
  const int* start;
  int ncores;
  __device__ int n() const { return ncores; }
  __device__ int first(int i) const { return start[i]; }
  __device__ ApplyCore core(int i) const { return c[i]; }
};

template <class Work>
__device__ __forceinline__ int find_core(const Work& w, int tile) {
  int lo = 0, hi = w.n() - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.first(mid) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The contiguous range of core elements [e0, e0 + n) that tile `tl` of core
// c reads: whole r_b-blocks of the a its rows touch, e0 rounded down to even.
__host__ __device__ inline void stage_range(const ApplyCore& c, long tl, long* e0, long* n) {
  const long row0 = tl * kTileM;
  const long a0 = row0 / c.rb;
  const long last = (row0 + kTileM - 1) / c.rb;
  const long a1 = last < c.ra - 1 ? last : (long)c.ra - 1;
  const long s0 = a0 * c.m * c.rb, s1 = (a1 + 1) * c.m * c.rb;
  *e0 = s0 & ~1L;
  *n = s1 - *e0;
}

// Issue the staged copy of `tile` (thread 0 only): the even part by TMA, an
// odd last element by a plain load; the arrive announces the TMA bytes.
template <class Work>
__device__ __forceinline__ void stage_issue(const Work& w, int tile, double* stage, uint32_t tbar) {
  const int ci = find_core(w, tile);
  const ApplyCore c = w.core(ci);
  long e0, n;
  stage_range(c, tile - w.first(ci), &e0, &n);
  const uint32_t bytes = (uint32_t)((n & ~1L) * 8);
  if (n & 1) stage[n - 1] = c.X[e0 + n - 1];
  mbar_arrive_expect_tx(tbar, bytes);
  if (bytes) bulk_g2s(smem_u32(stage), c.X + e0, bytes, tbar);
}

// Persistent: CTA b handles tiles b, b + gridDim.x, ...  TMEM and the
// mbarriers are set up once; the operator tile is restaged only when the core
// changes.
template <int P, class Work, bool kStage>
__global__ void __launch_bounds__(kThreads, kStage ? 2 : 4) apply_tc_kernel(Work w, int total, int* err) {
  using O = Op<P>;
  constexpr int E = O::kBytes;
  constexpr int kTileBytes = kTileM * kMaxK * E;  // 16 KB (BF16) or 32 KB (TF32)
  constexpr int W = 128 / E;                      // elements per swizzle row
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of both tiles (the swizzle pattern repeats every 1024 B)
  unsigned char* sA = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* sB = sA + kTileBytes;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sB + kTileBytes);
  unsigned long long* tbarp = mbar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  double* stage = reinterpret_cast<double*>(sB + kTileBytes + 128);  // 128-byte aligned
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kTileN);
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    if (kStage) mbar_init(smem_u32(tbarp), 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t bar = smem_u32(mbar);
  const uint32_t tbar = smem_u32(tbarp);
  if (kStage && tid == 0 && blockIdx.x < total) stage_issue(w, blockIdx.x, stage, tbar);

  int staged = -1;  // core whose operator tile sits in sB
  uint32_t phase = 0, tphase = 0;
  bool inflight = kStage && blockIdx.x < total;  // a staged copy not yet waited for
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x, phase ^= 1u) {
    const int ci = find_core(w, tile);
    const ApplyCore c = w.core(ci);
    const int m = c.m, ra = c.ra, rb = c.rb;
    const long nrows = (long)ra * rb;
    const long row0 = (long)(tile - w.first(ci)) * kTileM;
    long e0 = 0;
    if (kStage) {
      long n;
      stage_range(c, tile - w.first(ci), &e0, &n);
      const bool tok = __syncthreads_and(mbar_wait(tbar, tphase)) != 0;
      tphase ^= 1u;
      inflight = false;
      if (!tok) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait(tbar, tphase ^ 1u);  // bounded second wait for the copy
        break;
      }
    }
    // element g of the core: xbase[g - xoff]
    const double* xbase = kStage ? stage : c.X;
    const long xoff = kStage ? e0 : 0;
    // K padded to whole MMAs; N = 2m padded to a multiple of 16 (M = 128 form)
    const int kpad = ((m + O::kMmaK - 1) / O::kMmaK) * O::kMmaK;
    const int npad = ((2 * m + 15) / 16) * 16;
    // A tile: row t <-> pair g = row0 + t = (a, b); zero rows past the core.
    // Work items are 16-byte chunks of one row (8 BF16 / 4 TF32 values): a
    // warp takes 32 consecutive rows of one chunk, so each of its loads reads
    // 32 consecutive b (coalesced), each thread keeps a chunk's loads in
    // flight together, and one 16-byte shared store lands the chunk in its
    // swizzled slot.
    {
      constexpr int kPer = 16 / E;
      const int nch = kpad / kPer;
      for (int it = tid; it < kTileM * nch; it += kThreads) {
        const int t = it % kTileM, ch = it / kTileM;
        const long g = row0 + t;
        const bool valid = g < nrows;
        const long a = valid ? g / rb : 0, b = valid ? g % rb : 0;
        const double* xr = xbase + (a * (long)m * rb + b - xoff);
        double v[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const int j = ch * kPer + q;
          v[q] = (valid && j < m) ? xr[(long)j * rb] : 0.0;
        }
        *reinterpret_cast<uint4*>(sA + sw128_off<E>(t, ch * kPer, kTileM)) = O::pack16(v);
      }
    }
    // B tile: row ii < m: S row ii; m <= ii < 2m: G row ii - m; zero padded
    if (ci != staged) {
      for (int e = tid; e < npad * kpad; e += kThreads) {
        const int ii = e / kpad, j = e % kpad;
        double v = 0.0;
        if (ii < 2 * m && j < m) {
          if (ii < m) {
            v = c.S[(long)ii * m + j];
          } else {
            const long o = (long)(ii - m) * m + j;
            v = c.g_op * c.L[o];
            if (c.g_mass != 0.0) v += c.g_mass * c.S[o];
          }
        }
        O::store(sB + sw128_off<E>(ii, j, kTileM), v);
      }
      staged = ci;
    }
    // generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    // the stage has been read: bring in the next tile's rows while this
    // tile's MMAs and epilogue run
    if (kStage && tile + (int)gridDim.x < total) {
      if (tid == 0) stage_issue(w, tile + gridDim.x, stage, tbar);
      inflight = true;
    }
    if (tid == 0) {
      const uint32_t idesc = make_idesc(O::kFmt, kTileM, npad);
      for (int k0 = 0; k0 < kpad; k0 += O::kMmaK) {
        // K-block base, then 32 bytes per MMA step inside the 128-byte row
        const uint32_t off = (uint32_t)((k0 / W) * (kTileM * 128) + (k0 % W) * E);
        const uint64_t da = sdesc_sw128(smem_u32(sA) + off);
        const uint64_t db = sdesc_sw128(smem_u32(sB) + off);
        issue_mma<P>(tmem, da, db, idesc, k0 > 0 ? 1u : 0u);
      }
      mma_commit(bar);
    }
    // every thread waits (bounded); the block-wide vote keeps the
    // warp-collective TMEM loads below uniform even if one wait ran out
    const bool ok = __syncthreads_and(mbar_wait(bar, phase)) != 0;
    if (!ok) {
      if (tid == 0) atomicExch(err, 1);
      mbar_wait(bar, phase);  // bounded second wait for MMAs still in flight
      if (inflight) mbar_wait(tbar, tphase);  // and for the next tile's copy
      break;
    }
    fence_after_sync();
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (= tile rows)
    // and every other 32-column chunk, starting at chunk w / 4
    const int quarter = warp & 3;
    const int t = quarter * 32 + lane;
    const long g = row0 + t;
    const bool valid = g < nrows;
    const long a = valid ? g / rb : 0, b = valid ? g % rb : 0;
    double* Y = c.Y;
    for (int c0 = 32 * (warp >> 2); c0 < 2 * m; c0 += 64) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
      if (!valid) continue;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int row = c0 + q;
        if (row >= 2 * m) break;
        const double val = (double)__uint_as_float(v[q]);
        const bool gpart = row >= m;
        const int ii = gpart ? row - m : row;
        switch (c.kind) {
          case kApplySingle:  // 1 x m x 1: G X
            if (gpart) Y[ii] = val;
            break;
          case kApplyFirst: {  // 1 x m x 2rb: [G X, S X]
            const long base = (long)ii * 2 * rb;
            if (gpart) Y[base + b] = val; else Y[base + rb + b] = val;
            break;
          }
          case kApplyLast: {  // 2ra x m x 1: [S X; G X]
            const long r = gpart ? (ra + a) : a;
            Y[r * m + ii] = val;
            break;
          }
          default: {  // middle: 2ra x m x 2rb
            const long wd = 2L * rb;
            if (gpart) {
              Y[((long)(ra + a) * m + ii) * wd + b] = val;
            } else {
              Y[((long)a * m + ii) * wd + b] = val;
              Y[((long)(ra + a) * m + ii) * wd + rb + b] = val;
              Y[((long)a * m + ii) * wd + rb + b] = 0.0;
            }
          }
        }
      }
    }
    fence_before_sync();  // TMEM reads done before the next tile's MMAs
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTileN);
}

// Dynamic shared memory of the staged variant: the operand tiles, the
// barriers and a stage of stage_elems doubles.
size_t staged_smem_bytes(int elem_bytes, long stage_elems) {
  return (size_t)2 * kTileM * kMaxK * elem_bytes + 1024 + 128 + (size_t)stage_elems * 8;
}

template <int P, class Work>
t2s2_status launch_tc(const Work& w, int total, int grid, int* err, long stage_elems, cudaStream_t st) {
  if (stage_elems > 0) {
    const size_t smem = staged_smem_bytes(Op<P>::kBytes, stage_elems);
    T2S2_CUDA_TRY(cudaFuncSetAttribute(apply_tc_kernel<P, Work, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    apply_tc_kernel<P, Work, true><<<grid, kThreads, smem, st>>>(w, total, err);
    T2S2_CUDA_TRY(cudaGetLastError());
    return T2S2_OK;
  }
  constexpr int kSmem = smem_bytes(Op<P>::kBytes);
  // the attribute is per function and device; setting it each call is cheap
  T2S2_CUDA_TRY(
      cudaFuncSetAttribute(apply_tc_kernel<P, Work, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  apply_tc_kernel<P, Work, false><<<grid, kThreads, kSmem, st>>>(w, total, err);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

void work_totals(const ApplyCore& c, double& fl, double& by) {
  fl += 2.0 * (2.0 * c.m) * c.m * (double)c.ra * c.rb;
  const int ny = (c.kind == kApplyMiddle) ? 4 : ((c.kind == kApplySingle) ? 1 : 2);
  by += 8.0 * ((double)c.ra * c.m * c.rb * (1 + ny) + 2.0 * c.m * c.m);
}

}  // namespace

bool apply_tc_supported(const ApplyBatch& p) {
  for (int k = 0; k < p.ncores; ++k)
    if (p.c[k].m > kMaxK || p.c[k].m < 1) return false;
  return true;
}

int apply_tc_tiles(const ApplyCore& c) { return (int)((((long)c.ra * c.rb) + kTileM - 1) / kTileM); }

int apply_tc_max_ctas_per_sm(int prec, long stage_elems) {
  const int eb = prec == T2S2_BF16_REFINE ? 2 : 4;
  const size_t smem = stage_elems > 0 ? staged_smem_bytes(eb, stage_elems) : (size_t)smem_bytes(eb);
  return std::min<int>(std::min(512 / kTileN, stage_elems > 0 ? 2 : 4), (int)((227 * 1024) / smem));
}

long apply_tc_stage_elems(const ApplyCore& c) {
  if (reinterpret_cast<uintptr_t>(c.X) % 16 != 0) return -1;  // the bulk copy needs 16-byte alignment
  const long tiles = apply_tc_tiles(c);
  long most = 0;
  for (long tl = 0; tl < tiles; ++tl) {
    long e0, n;
    stage_range(c, tl, &e0, &n);
    most = std::max(most, n);
  }
  return most;
}

t2s2_status apply_tc(const ApplyBatch& p, int prec, int* err, cudaStream_t st) {
  if (prec != T2S2_BF16_REFINE && prec != T2S2_TF32_REFINE) return T2S2_EINVAL;
  if (!apply_tc_supported(p) || !err) return T2S2_EINVAL;
  ParamWork w;
  w.p = p;
  int total = 0;
  double fl = 0.0, by = 0.0;
  for (int k = 0; k < p.ncores; ++k) {
    w.start[k] = total;
    total += apply_tc_tiles(p.c[k]);
    work_totals(p.c[k], fl, by);
  }
  w.start[p.ncores] = total;
  if (total == 0) return T2S2_OK;
  TraceScope ts(kTrApplyTc, st, fl, by);
  if (prec == T2S2_BF16_REFINE) return launch_tc<T2S2_BF16_REFINE>(w, total, total, err, 0, st);
  return launch_tc<T2S2_TF32_REFINE>(w, total, total, err, 0, st);
}

t2s2_status apply_tc_grouped(const ApplyCore* dcores, const int* dstart, int ncores, int total, int grid,
                             double flops, double bytes, int prec, int* err, long stage_elems, cudaStream_t st) {
  if (prec != T2S2_BF16_REFINE && prec != T2S2_TF32_REFINE) return T2S2_EINVAL;
  if (!err || ncores < 1 || total < 0 || grid < 1) return T2S2_EINVAL;
  if (stage_elems > 0 && staged_smem_bytes(prec == T2S2_BF16_REFINE ? 2 : 4, stage_elems) > 227 * 1024)
    return T2S2_EINVAL;
  if (total == 0) return T2S2_OK;
  GlobalWork w{dcores, dstart, ncores};
  TraceScope ts(kTrApplyTc, st, flops, bytes);
  if (prec == T2S2_BF16_REFINE)
    return launch_tc<T2S2_BF16_REFINE>(w, total, std::min(grid, total), err, stage_elems, st);
  return launch_tc<T2S2_TF32_REFINE>(w, total, std::min(grid, total), err, stage_elems, st);
}

void apply_work_totals(const ApplyCore& c, double* flops, double* bytes) { work_totals(c, *flops, *bytes); }

}  // namespace t2s2
