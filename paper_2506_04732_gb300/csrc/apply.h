// Fused TT-apply of the rank-2 collocation operator (see apply.cu).
#pragma once
#include "common.cuh"

namespace t2s2 {

enum { kApplyMiddle = 0, kApplyFirst = 1, kApplyLast = 2, kApplySingle = 3 };

struct ApplyCore {
  const double* S;   // m x m (Rt_k, or the identity)
  const double* L;   // m x m (Lt_k, or B_k)
  const double* X;   // ra x m x rb
  double* Y;         // output core (layout set by kind)
  int ra, m, rb, kind;
  double g_mass, g_op;  // G = g_op * L + g_mass * S
};

struct ApplyBatch {
  int ncores;
  ApplyCore c[T2S2_MAX_D];
};

__host__ __device__ inline int cdiv_dev(int a, int b) { return (a + b - 1) / b; }

t2s2_status apply_fp64(const ApplyBatch& p, cudaStream_t st);

// Same product on tcgen05 tensor cores with BF16 (prec = T2S2_BF16_REFINE) or
// TF32 (T2S2_TF32_REFINE) operands and FP32 accumulation; needs m <= 64 for
// every core.  A device wait that gives up sets *err (device int) to 1.
bool apply_tc_supported(const ApplyBatch& p);
t2s2_status apply_tc(const ApplyBatch& p, int prec, int* err, cudaStream_t st);

// Grouped, persistent launches over the cores of many trains: dcores (device)
// holds ncores descriptors, dstart (device) the prefix sums of their tile
// counts (apply_fp64_tiles / apply_tc_tiles), dstart[ncores] = total; `grid`
// CTAs loop over the tiles.  flops / bytes are the algorithmic totals for
// tracing (apply_work_totals summed over the cores).
int apply_fp64_tiles(const ApplyCore& c);
int apply_tc_tiles(const ApplyCore& c);
// CTAs per SM the tensor-core kernel can hold: the direct variant
// (stage_elems = 0) or the staged one with a stage of stage_elems doubles.
int apply_tc_max_ctas_per_sm(int prec, long stage_elems);
// Doubles the staged variant needs for core c (the largest contiguous range a
// tile reads), or -1 if the core is not 16-byte aligned.
long apply_tc_stage_elems(const ApplyCore& c);
void apply_work_totals(const ApplyCore& c, double* flops, double* bytes);
t2s2_status apply_fp64_grouped(const ApplyCore* dcores, const int* dstart, int ncores, int total, int grid,
                               double flops, double bytes, cudaStream_t st);
// stage_elems > 0: the staged (bulk TMA) variant with a stage of that many
// doubles, at least apply_tc_stage_elems of every core; 0: direct loads.
t2s2_status apply_tc_grouped(const ApplyCore* dcores, const int* dstart, int ncores, int total, int grid,
                             double flops, double bytes, int prec, int* err, long stage_elems, cudaStream_t st);

}  // namespace t2s2
