// Small dense FP64 factorisations done by a single CTA (c <= kSmallMax).
#pragma once
#include "common.cuh"

namespace t2s2 {

constexpr int kSmallMax = 96;

// L L^T = G + shift_rel * trace(G) * I and Linv = L^{-1}; status[0] = 1 if a
// pivot was not positive (then replaced by a tiny value).
t2s2_status chol_inv(const double* G, int c, double shift_rel, double* L, double* Linv, int* status,
                     cudaStream_t st);

// A (p x q) = U (p x k) diag(s) V^T (V: q x k), k = min(p, q), s decreasing.
t2s2_status jacobi_svd(const double* A, int p, int q, double* U, double* s, double* V, int* sweeps,
                       cudaStream_t st);

}  // namespace t2s2
