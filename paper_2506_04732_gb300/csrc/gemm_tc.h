// Strided-batched GEMM on tcgen05 tensor cores (see gemm_tc.cu): the Gemm<T>
// description of gemm.h with T = double or float in and out, operands rounded
// to BF16 (prec = T2S2_BF16_REFINE) or TF32 (T2S2_TF32_REFINE), FP32
// accumulation.
#pragma once
#include "gemm.h"

namespace t2s2 {

// Workspace bytes needed for the split-K partial sums; 0 if none.
template <typename T>
size_t gemm_tc_workspace_bytes(const Gemm<T>& g, int prec);

// Launches the product; a bounded device wait that gives up sets *err (a
// device int) to 1.  T2S2_ENOMEM if ws is smaller than the workspace.
template <typename T>
t2s2_status gemm_tc(const Gemm<T>& g, int prec, void* ws, size_t ws_bytes, int* err, cudaStream_t st);

}  // namespace t2s2
