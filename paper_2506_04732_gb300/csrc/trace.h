// Kernel launch accounting and optional CUDA-event timing per kernel family.
#pragma once
#include "common.cuh"

namespace t2s2 {

enum TraceFamily {
  kTrGemm = 0,
  kTrApply = 1,
  kTrLocal = 2,
  kTrSmall = 3,
  kTrElem = 4,
  kTrApplyTc = 5,
  kTrGemmTc = 6,
  kTrMlp = 7,
  kTrCholQR = 8,  // the fused shifted CholeskyQR (one cooperative launch per QR)
  kTrSylv = 9,    // the rank-1-right local solves (Schur-basis Sylvester solver)
  kTrDots = 10,   // TT inner products (binary64 and double-double)
  kTrFamilies = 11
};

// Count one launch of `fam` with its algorithmic FLOPs and DRAM-level bytes;
// when tracing is on, `begin` must have been called on the same stream first.
struct TraceScope {
  int fam;
  cudaStream_t st;
  double flops, bytes;
  int slot;
  TraceScope(int fam, cudaStream_t st, double flops, double bytes);
  ~TraceScope();
};

// Add algorithmic work known only after a launch (e.g. iteration counts).
void trace_add_work(int fam, double flops, double bytes);

}  // namespace t2s2
