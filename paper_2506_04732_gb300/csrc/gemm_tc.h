// Strided-batched GEMM on tcgen05 tensor cores (see gemm_tc.cu): the Gemm<double>
// description of gemm.h, FP64 in and out, operands rounded to BF16
// (prec = T2S2_BF16_REFINE) or TF32 (T2S2_TF32_REFINE), FP32 accumulation.
#pragma once
#include "gemm.h"

namespace t2s2 {

// Workspace (doubles) needed for the split-K partial sums; 0 if none.
size_t gemm_tc_workspace(const Gemm<double>& g, int prec);

// Launches the product; a bounded device wait that gives up sets *err (a
// device int) to 1.  T2S2_ENOMEM if ws is smaller than gemm_tc_workspace.
t2s2_status gemm_tc(const Gemm<double>& g, int prec, double* ws, size_t ws_elems, int* err, cudaStream_t st);

}  // namespace t2s2
