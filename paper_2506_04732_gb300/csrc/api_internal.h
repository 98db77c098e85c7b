// Internal state behind the C ABI: the operator handle and shared helpers.
#pragma once
#include <vector>

#include "apply.h"
#include "gemm_tc.h"
#include "host_1d.h"
#include "tt.h"

// Per dimension the device holds kMatsPerDim m x m FP64 matrices:
// Rt, Lt, Rt^{-1}, B = Rt^{-1} Lt, I, and the complex Schur form B = Z T Z^H
// as Re T, Im T, Re Z, Im Z.
constexpr int kMatsPerDim = 9;

struct t2s2_op_s {
  int device = 0;
  int d = 0;
  int n[T2S2_MAX_D] = {0}, m[T2S2_MAX_D] = {0};
  double beta[T2S2_MAX_D] = {0};
  double eps = 0;
  int plain = 0;
  std::vector<t2s2::Dim1D> dims;
  double* dmat = nullptr;
  double *dRt[T2S2_MAX_D] = {nullptr}, *dLt[T2S2_MAX_D] = {nullptr}, *dRinv[T2S2_MAX_D] = {nullptr},
         *dB[T2S2_MAX_D] = {nullptr}, *dI[T2S2_MAX_D] = {nullptr}, *dTr[T2S2_MAX_D] = {nullptr},
         *dTi[T2S2_MAX_D] = {nullptr}, *dZr[T2S2_MAX_D] = {nullptr}, *dZi[T2S2_MAX_D] = {nullptr};
  float* fmat = nullptr;  // FP32 copies of all of the above, same layout
  // space dimensions: the full m x n matrices Rf, Lf (every GLL node a
  // column), for lifting boundary data; null for the time dimension
  double* dfull = nullptr;
  double *dRf[T2S2_MAX_D] = {nullptr}, *dLf[T2S2_MAX_D] = {nullptr};
  // a product reaction prod_k pi_k(x_k): P_k = diag(pi_k(eta)) Rt_k per
  // dimension (m x m) and rho_bar = prod_k mean(pi_k(eta))
  int has_prod = 0;
  double* dprod = nullptr;
  double* dP[T2S2_MAX_D] = {nullptr};
  double rho_bar = 0.0;
  float* fptr[kMatsPerDim][T2S2_MAX_D] = {{nullptr}};
  t2s2::Arena arena;
  int team = 0;            // CTAs per cooperative local solve (0: whole GPU)
  double* hbuf = nullptr;  // pinned host scratch
  int* dstat = nullptr;    // device status words
  int* gcnt = nullptr;     // kGemmCounters split-K tile counters (zero between launches)
  // a second stream for work that overlaps the main one, with its fork and
  // join events (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the solver's right-orthogonalised random start of z for one kick
  double* zcache = nullptr;
  size_t zcache_elems = 0;
  int zcache_kick = 0;
  void free_solver_buffers();
};

namespace t2s2 {
t2s2_status ensure_arena(t2s2_op op, size_t bytes);
Ctx make_ctx(t2s2_op op, void* stream);
size_t tt_bytes(const t2s2_tt* t);
size_t max_core(const t2s2_tt* t);
t2s2_status check_tt(t2s2_op op, const t2s2_tt* t);
t2s2_status check_out_tt(t2s2_op op, const t2s2_tt* t);
t2s2_status bind_tt(Ctx& cx, const t2s2_tt* t, DevTT& dv, bool upload);
t2s2_status unbind_tt(Ctx& cx, const DevTT& dv, t2s2_tt* t);
// Status words in op->dstat: word 0 for the small factorisations, word
// kStatTensorCore for the tensor-core kernels' bounded waits.
constexpr int kStatTensorCore = 16;
// GEMM of the sweep's contractions in the context's contraction arithmetic.
t2s2_status contract_gemm(Ctx& cx, const Gemm<double>& g);
// Independent contractions (no output read or written by another) in one
// launch where the arithmetic allows, else one after another.
t2s2_status contract_group(Ctx& cx, const Gemm<double>* gs, int n);
// Reads (synchronising) and reports the tensor-core wait status word.
t2s2_status tensor_core_status(Ctx& cx);
t2s2_status apply_batch(t2s2_op op, const DevTT& x, DevTT& y, double c_mass, double c_op, bool transformed,
                        ApplyBatch& b);
t2s2_status apply_op(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass, double c_op,
                     bool transformed);
t2s2_status apply_dispatch(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass,
                           double c_op, t2s2_precision prec);
// Up to four TT inner products <u_p, v_p> in one launch (ttdot.cu); reads
// the values back (synchronising).
t2s2_status tt_dots(Ctx& cx, int n, const DevTT* const* u, const DevTT* const* v, double* out);
t2s2_status residual_estimate(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass,
                              double c_op, double* bb_io, double* out);
// <u_p, v_p> in double-double for p < n <= 4 (ttdot.cu), as hi + lo pairs.
t2s2_status tt_dots_dd(Ctx& cx, int n, const DevTT* const* u, const DevTT* const* v, double* hi, double* lo);
// What the residual of one right-hand side b keeps between calls: |b| and
// |b|^2 in double-double (negative: not known yet).
struct ResidualCache {
  double bnorm = -1.0;
  double bb_hi = -1.0, bb_lo = 0.0;
};
// The residual of the original system: |b|^2 - 2<b, A x> + |A x|^2 with the
// inner products in double-double, falling back to residual_impl's
// orthogonalised norm for residuals below 1e-13.  screen: first try binary64
// inner products, and return their value when it is above 1e-5 (a guess far
// from converged).
t2s2_status residual_fast(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass, double c_op,
                          double* out, ResidualCache* rc, bool screen);
t2s2_status residual_impl(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass,
                          double c_op, bool transformed, double* out, double* bnorm_io);
// y = (c_mass M + c_op A) x, plus c_op times the product reaction when the
// operator has one (ranks 3 r_x then, 2 r_x otherwise); y is allocated in
// the arena.
t2s2_status apply_full(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass, double c_op);
// y = ((x)_k mats[k]) x: every core times its m x m matrix along its mode
// (ranks kept); y is allocated in the arena.
t2s2_status apply_kron(Ctx& cx, const DevTT& x, double* const* mats, DevTT& y);
// ||b - (c_mass M + c_op A + c_op P) x|| / ||b|| through the orthogonalised
// difference (operators with a product reaction).
t2s2_status residual_full(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass, double c_op,
                          double* out);
// The alternating solve of (c_mass M + c_op A) x = b on bound TTs (solve.cu).
t2s2_status solve_run(t2s2_op op, Ctx& cx, const DevTT& b, DevTT& xio, double c_mass, double c_op,
                      double tol, int rmax, int max_sweeps, t2s2_precision prec, t2s2_solve_info* info);
// Arena bytes of one alternating solve (solve.cu).
size_t solve_bytes(t2s2_op op, int rmax, int rfmax, t2s2_precision prec);
}  // namespace t2s2
