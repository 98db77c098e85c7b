// Small dense FP64 factorisations done by a single CTA (c <= kSmallMax).
#pragma once
#include "common.cuh"

namespace t2s2 {

constexpr int kSmallMax = 96;

// Passes of the shifted CholeskyQR (cholqr.cu, cholqr_cluster.cu and the
// chol_inv fallback): the first two passes that are not the last take the
// shift 11 (n c + c (c + 1)) u max(diag G); the rest are plain.  One shifted
// pass maps a direction of W with singular value sigma to ~sigma / sqrt(s) in
// Q; when that is near the roundoff of the next Gram (sigma below ~1e-12 of
// the largest), a plain second pass would zero its pivot in column order and
// lose the whole remainder of that column of W, not just sigma.  A second
// shift lifts such directions above roundoff first; a pass whose Gram is
// within 0.5 / c of the identity is the last, so well-conditioned blocks still
// take two passes.
constexpr int kCqrMaxPass = 4;
constexpr int kCqrShiftedPasses = 2;

// L L^T = G + shift_rel * trace(G) * I and Linv = L^{-1}; status[0] = 1 if a
// pivot was not positive (then replaced by a tiny value).
t2s2_status chol_inv(const double* G, int c, double shift_rel, double* L, double* Linv, int* status,
                     cudaStream_t st);

// A (p x q) = U (p x k) diag(s) V^T (V: q x k), k = min(p, q), s decreasing.
t2s2_status jacobi_svd(const double* A, int p, int q, double* U, double* s, double* V, int* sweeps,
                       cudaStream_t st);

// Shifted CholeskyQR of nlong vectors of length c in one cooperative launch
// (cholqr.cu): up to kCqrMaxPass passes, fewer when a pass's Gram certifies
// that the next one finishes.  tall: W is nlong x c row-major, W = Q R (R = c x c upper);
// wide: W is c x nlong row-major, W = R Q (R lower).  Plan first: false if
// the grid cannot be co-resident or shared memory would not fit; max_grid > 0
// caps the number of CTAs.
bool cholqr3_plan(int nlong, int c, int max_grid, int* grid, int* per, size_t* smem);
size_t cholqr3_scratch_doubles(int nlong, int c, int grid);
// W2 (tall only): the input as two row-major blocks, columns 0 .. c1-1 in W
// (nlong x c1) and c1 .. c-1 in W2 (nlong x (c - c1)).
t2s2_status cholqr3_fused(const double* W, double* Q, double* R, int nlong, int c, bool tall, double shift_rel,
                          double* scratch, int* status, int grid, int per, size_t smem, cudaStream_t st,
                          const double* W2 = nullptr, int c1 = 0);

// The same factorisation in one thread-block cluster of up to 16 CTAs
// (cholqr_cluster.cu), for blocks that fit its shared memory: one cluster
// barrier per pass instead of two grid barriers, and a launch that overlaps
// the previous kernel.  Same layouts, outputs and status as cholqr3_fused;
// plan first (false: take the full-grid kernel).  R is triangular unless
// the last pass took the series of (I + E)^(-1/2), in which case it is a full
// matrix (still W = Q R, resp. W = R Q).
bool cqr_cluster_plan(int nlong, int c, int* cl, int* per, size_t* smem);
t2s2_status cqr_cluster(const double* W, double* Q, double* R, int nlong, int c, bool tall, double shift_rel,
                        int* status, int cl, int per, size_t smem, cudaStream_t st, const double* W2 = nullptr,
                        int c1 = 0);

}  // namespace t2s2
