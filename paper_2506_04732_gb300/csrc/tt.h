// Device tensor trains and their FP64 arithmetic (Methods, "Tensor Train
// representation"): orthogonalisation, rounding, norms, sums.
#pragma once
#include <vector>

#include "common.cuh"
#include "gemm.h"
#include "small.h"

namespace t2s2 {

// Bump allocator over one device buffer; `mark`/`release` give stack scoping.
struct Arena {
  char* base = nullptr;
  size_t size = 0, top = 0, peak = 0;
  void* get(size_t bytes) {
    size_t a = (top + 255) & ~(size_t)255;
    if (a + bytes > size) return nullptr;
    top = a + bytes;
    if (top > peak) peak = top;
    return base + a;
  }
  size_t mark() const { return top; }
  void release(size_t m) { top = m; }
};

struct DevTT {
  int d = 0;
  int m[T2S2_MAX_D] = {0};
  int r[T2S2_MAX_D + 1] = {0};
  double* c[T2S2_MAX_D] = {nullptr};
  size_t cap[T2S2_MAX_D] = {0};
  size_t core_elems(int k) const { return (size_t)r[k] * m[k] * r[k + 1]; }
};

struct Ctx {
  cudaStream_t st = 0;
  Arena* ar = nullptr;
  double* hbuf = nullptr;   // pinned host scratch (>= 4 * kSmallMax doubles)
  int* dstat = nullptr;     // device status word
  // Arithmetic of the sweep's contractions (mode products, interfaces):
  // T2S2_FP64 (SIMT FP64 GEMM) or T2S2_TF32_REFINE / T2S2_BF16_REFINE
  // (tcgen05 GEMM).  QR, SVD and norms always run in FP64.
  int contract_prec = T2S2_FP64;
  // CTAs a cooperative launch may use (0: the whole GPU); concurrent solves
  // split the SMs so that their cooperative grids are co-resident
  int coop_ctas = 0;
  // rank of the solver's enrichment for this call (0: the library default)
  int kick = 0;
  // split-K tile counters of the FP64 GEMM on this context's stream (null:
  // partial sums are added by a second launch)
  int* gcnt = nullptr;
};
constexpr long kGemmCounters = 16384;

template <typename T>
inline T* aget(Ctx& cx, size_t n) {
  return static_cast<T*>(cx.ar->get(n * sizeof(T)));
}

// Allocate a TT in the arena with given ranks (capacities = exact sizes).
t2s2_status tt_alloc(Ctx& cx, DevTT& t, int d, const int* m, const int* r, int rcap);
t2s2_status tt_copy(Ctx& cx, const DevTT& src, DevTT& dst);
// z = alpha x + beta y as block-diagonal concatenation (ranks add); z in arena.
t2s2_status tt_axpby(Ctx& cx, double alpha, const DevTT& x, double beta, const DevTT& y, DevTT& z);
// In place: cores 1..d-1 right-orthonormal (rows), weight in core 0.
t2s2_status tt_orth_right(Ctx& cx, DevTT& x);
// In place rounding with ||x - rndg(x)|| <= tol ||x|| (cap rmax <= 0: none).
t2s2_status tt_round(Ctx& cx, DevTT& x, double tol, int rmax);
// ||x||_F of a TT already right-orthogonalised (norm of core 0).
t2s2_status core_norm(Ctx& cx, const double* v, size_t n, double* out);
// ||x||_F for any TT (works on a copy).
t2s2_status tt_norm(Ctx& cx, const DevTT& x, double* out);

// Dense helpers used by the solver.
// W (rows x cols, rows >= cols) = Q R, Q orthonormal columns (shifted CholeskyQR3).
t2s2_status qr_tall(Ctx& cx, const double* W, int rows, int cols, double* Q, double* R);
// The fused CholeskyQR of a tall block on stream `side` (false, with nothing
// queued, if it does not fit).  Its scratch comes from the arena and stays
// allocated: release the arena mark only after joining `side`.
bool qr_tall_async(Ctx& cx, const double* W, int rows, int cols, double* Q, double* R, cudaStream_t side,
                   t2s2_status* st);
// [U | W2] (rows x (c1 + c2), two row-major blocks) = Q R; scratch holds
// rows x (c1 + c2) for the unfused path.
t2s2_status qr_tall2(Ctx& cx, const double* U, int c1, const double* W2, int c2, int rows, double* Q, double* R,
                     double* scratch);
// W (rows x cols, rows <= cols) = L Q, Q orthonormal rows.
t2s2_status lq_wide(Ctx& cx, const double* W, int rows, int cols, double* Q, double* L);
// Smallest r >= 1 with sqrt(sum_{j >= r} s_j^2) <= delta, capped by rmax (> 0).
int trunc_rank(const double* s, int n, double delta, int rmax);

template <typename T>
inline t2s2_status gemm_ex(Ctx& cx, int M, int N, int K, bool tA, bool tB, T alpha, const T* A,
                           long lda, const T* B, long ldb, T beta, T* C, long ldc, int batch = 1,
                           long sA = 0, long sB = 0, long sC = 0) {
  Gemm<T> g;
  g.M = M; g.N = N; g.K = K; g.tA = tA; g.tB = tB; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.sA = sA; g.B = B; g.ldb = ldb; g.sB = sB;
  g.C = C; g.ldc = ldc; g.sC = sC; g.batch = batch;
  size_t need = gemm_workspace(g);
  size_t mk = cx.ar->mark();
  T* ws = need ? aget<T>(cx, need) : nullptr;
  t2s2_status s = gemm(g, ws, ws ? need : 0, cx.st, cx.gcnt, cx.gcnt ? kGemmCounters : 0);
  cx.ar->release(mk);
  return s;
}

// Elementwise kernels
t2s2_status dev_scale_copy(Ctx& cx, double* dst, const double* src, size_t n, double alpha);
t2s2_status dev_fill(Ctx& cx, double* dst, size_t n, double v);
t2s2_status dev_axpy(Ctx& cx, double* dst, const double* src, size_t n, double beta);
t2s2_status dev_d2f(Ctx& cx, float* dst, const double* src, size_t n);
t2s2_status dev_f2d(Ctx& cx, double* dst, const float* src, size_t n);
t2s2_status dev_identity(Ctx& cx, double* dst, int n);
// M[i][j] = s[i] * V[j][i] for i < r, j < q (V: q x ldv)
t2s2_status dev_sv_t(Ctx& cx, double* M, const double* s, const double* V, int r, int q, int ldv);

}  // namespace t2s2
