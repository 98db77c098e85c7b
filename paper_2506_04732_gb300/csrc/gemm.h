// Strided-batched GEMM on the SIMT pipes (FP64 / FP32), row-major operands:
//   C_b = alpha * op(A_b) * op(B_b) + beta * C_b,   b = 0..batch-1
// op(A) is M x K (A stored M x K with leading dimension lda, or K x M if tA).
// op(B) is K x N (B stored K x N, or N x K if tB).  Small outputs with long K
// are split over K across CTAs into `ws` and reduced in a fixed order.
#pragma once
#include "common.cuh"

namespace t2s2 {

template <typename T>
struct Gemm {
  int M = 0, N = 0, K = 0;
  bool tA = false, tB = false;
  T alpha = 1, beta = 0;
  const T* A = nullptr; long lda = 0, sA = 0;
  const T* B = nullptr; long ldb = 0, sB = 0;
  T* C = nullptr; long ldc = 0, sC = 0;
  int batch = 1;
};

// Workspace (elements of T) needed by gemm() for split-K; 0 if none.
template <typename T>
size_t gemm_workspace(const Gemm<T>& g);

// cnt (ncnt ints, all zero, owned by the caller's stream) lets FP64 split-K
// products add their partials inside the same launch; the counters are left
// at zero.  Without it a second launch adds them.
template <typename T>
t2s2_status gemm(const Gemm<T>& g, T* ws, size_t ws_elems, cudaStream_t st, int* cnt = nullptr, long ncnt = 0);

// Up to kMaxGroup independent FP64 products (no output shared with another's
// input or output) in one launch; each keeps its own split of K, whose
// partials are added inside the launch (cnt required, else one launch per
// product).  Workspace: gemm_group_workspace elements.
constexpr int kMaxGroup = 8;
size_t gemm_group_workspace(const Gemm<double>* gs, int n);
t2s2_status gemm_group(const Gemm<double>* gs, int n, double* ws, size_t ws_elems, cudaStream_t st, int* cnt,
                       long ncnt);

}  // namespace t2s2
