// C ABI entry points (include/t2s2.h): operator construction, TT apply,
// rounding, norms and residuals.  The solver entry points live in solve.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "api_internal.h"

namespace t2s2 {

// The last CUDA failure, process-wide (worker threads of the batched solve
// report through it too); diagnostics only.
static char g_last_error[256] = "";
static std::mutex g_last_error_mu;

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  std::lock_guard<std::mutex> lk(g_last_error_mu);
  snprintf(g_last_error, sizeof(g_last_error), "%s at %s:%d: %s", cudaGetErrorString(e), file, line,
           what);
}

void note_failure(int status, const char* what, const char* file, int line) {
  static const bool on = [] {
    const char* e = std::getenv("T2S2_VERBOSE");
    return e && e[0] == '1';
  }();
  if (status == T2S2_ENOCONV || !on) return;
  const char* f = std::strrchr(file, '/');
  fprintf(stderr, "[t2s2] status %d from %s at %s:%d\n", status, what, f ? f + 1 : file, line);
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("T2S2_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

t2s2_status ensure_arena(t2s2_op op, size_t bytes) {
  if (op->arena.size >= bytes) {
    op->arena.top = 0;
    return T2S2_OK;
  }
  if (op->arena.base) {
    cudaFree(op->arena.base);
    op->arena.base = nullptr;
    op->arena.size = 0;
  }
  size_t want = std::max(bytes, (size_t)8 << 20);
  void* p = nullptr;
  T2S2_CUDA_TRY(cudaMalloc(&p, want));
  op->arena.base = static_cast<char*>(p);
  op->arena.size = want;
  op->arena.top = 0;
  return T2S2_OK;
}

Ctx make_ctx(t2s2_op op, void* stream) {
  Ctx cx;
  cx.st = static_cast<cudaStream_t>(stream);
  cx.ar = &op->arena;
  cx.hbuf = op->hbuf;
  cx.dstat = op->dstat;
  cx.gcnt = op->gcnt;
  cx.coop_ctas = op->team;
  return cx;
}

size_t tt_bytes(const t2s2_tt* t) {
  size_t s = 0;
  for (int k = 0; k < t->d; ++k) s += t->cap[k];
  return s * sizeof(double);
}

t2s2_status check_tt(t2s2_op op, const t2s2_tt* t) {
  if (!t || !t->r || !t->cores || !t->cap || !t->m) return T2S2_EINVAL;
  if (t->d != op->d) return T2S2_EINVAL;
  if (t->loc != T2S2_DEVICE && t->loc != T2S2_HOST) return T2S2_EINVAL;
  if (t->r[0] != 1 || t->r[t->d] != 1) return T2S2_EINVAL;
  for (int k = 0; k < t->d; ++k) {
    if (t->m[k] != op->m[k]) return T2S2_EINVAL;
    if (t->r[k + 1] < 1 || !t->cores[k]) return T2S2_EINVAL;
    if ((size_t)t->r[k] * t->m[k] * t->r[k + 1] > t->cap[k]) return T2S2_ENOMEM;
  }
  return T2S2_OK;
}

// An output TT: pointers present, the operator's d and mode sizes, a known
// location.  Its ranks are written, not read.
t2s2_status check_out_tt(t2s2_op op, const t2s2_tt* t) {
  if (!t || !t->r || !t->cores || !t->cap || !t->m) return T2S2_EINVAL;
  if (t->d != op->d) return T2S2_EINVAL;
  if (t->loc != T2S2_DEVICE && t->loc != T2S2_HOST) return T2S2_EINVAL;
  for (int k = 0; k < t->d; ++k)
    if (t->m[k] != op->m[k] || !t->cores[k]) return T2S2_EINVAL;
  return T2S2_OK;
}

// Bind a user TT to a DevTT; host TTs get device staging in the arena and,
// if `upload`, their contents copied in.
t2s2_status bind_tt(Ctx& cx, const t2s2_tt* t, DevTT& dv, bool upload) {
  dv.d = t->d;
  for (int k = 0; k <= t->d; ++k) dv.r[k] = t->r[k];
  for (int k = 0; k < t->d; ++k) {
    dv.m[k] = t->m[k];
    dv.cap[k] = t->cap[k];
    if (t->loc == T2S2_DEVICE) {
      dv.c[k] = t->cores[k];
    } else {
      dv.c[k] = aget<double>(cx, t->cap[k]);
      if (!dv.c[k]) return T2S2_ENOMEM;
      if (upload)
        T2S2_CUDA_TRY(cudaMemcpyAsync(dv.c[k], t->cores[k], sizeof(double) * dv.core_elems(k),
                                      cudaMemcpyHostToDevice, cx.st));
    }
  }
  return T2S2_OK;
}

// Write ranks (and, for host TTs, contents) of dv back to the user TT.
t2s2_status unbind_tt(Ctx& cx, const DevTT& dv, t2s2_tt* t) {
  for (int k = 0; k < dv.d; ++k)
    if (dv.core_elems(k) > t->cap[k]) return T2S2_ENOMEM;
  for (int k = 0; k <= dv.d; ++k) t->r[k] = dv.r[k];
  if (t->loc == T2S2_HOST) {
    for (int k = 0; k < dv.d; ++k)
      T2S2_CUDA_TRY(cudaMemcpyAsync(t->cores[k], dv.c[k], sizeof(double) * dv.core_elems(k),
                                    cudaMemcpyDeviceToHost, cx.st));
  } else {
    for (int k = 0; k < dv.d; ++k)
      if (dv.c[k] != t->cores[k])
        T2S2_CUDA_TRY(cudaMemcpyAsync(t->cores[k], dv.c[k], sizeof(double) * dv.core_elems(k),
                                      cudaMemcpyDeviceToDevice, cx.st));
  }
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  return T2S2_OK;
}

// y = (c_mass M + c_op A) x  (S = Rt, L = Lt) or the transformed operator
// (S = I, L = B) when `transformed`.
t2s2_status apply_batch(t2s2_op op, const DevTT& x, DevTT& y, double c_mass, double c_op, bool transformed,
                        ApplyBatch& b) {
  const int d = op->d;
  y.d = d;
  y.r[0] = 1;
  y.r[d] = 1;
  for (int k = 1; k < d; ++k) y.r[k] = 2 * x.r[k];
  for (int k = 0; k < d; ++k) {
    y.m[k] = x.m[k];
    if (y.core_elems(k) > y.cap[k]) return T2S2_ENOMEM;
  }
  b.ncores = d;
  for (int k = 0; k < d; ++k) {
    ApplyCore& c = b.c[k];
    c.S = transformed ? op->dI[k] : op->dRt[k];
    c.L = transformed ? op->dB[k] : op->dLt[k];
    c.X = x.c[k];
    c.Y = y.c[k];
    c.ra = x.r[k];
    c.m = x.m[k];
    c.rb = x.r[k + 1];
    c.kind = (d == 1) ? kApplySingle : (k == 0 ? kApplyFirst : (k == d - 1 ? kApplyLast : kApplyMiddle));
    c.g_op = c_op;
    c.g_mass = (k == 0) ? c_mass : 0.0;
  }
  return T2S2_OK;
}

t2s2_status apply_op(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass, double c_op,
                     bool transformed) {
  ApplyBatch b;
  T2S2_TRY(apply_batch(op, x, y, c_mass, c_op, transformed, b));
  return apply_fp64(b, cx.st);
}

t2s2_status apply_full(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass, double c_op) {
  const int d = op->d;
  int r2[T2S2_MAX_D + 1];
  for (int k = 0; k <= d; ++k) r2[k] = (k == 0 || k == d) ? 1 : 2 * x.r[k];
  if (!op->has_prod) {
    T2S2_TRY(tt_alloc(cx, y, d, x.m, r2, 0));
    return apply_op(op, cx, x, y, c_mass, c_op, false);
  }
  DevTT y2, yp;
  T2S2_TRY(tt_alloc(cx, y2, d, x.m, r2, 0));
  T2S2_TRY(apply_op(op, cx, x, y2, c_mass, c_op, false));
  // the product term keeps the ranks: core k times P_k along its mode
  T2S2_TRY(apply_kron(cx, x, op->dP, yp));
  return tt_axpby(cx, 1.0, y2, c_op, yp, y);
}

t2s2_status apply_kron(Ctx& cx, const DevTT& x, double* const* mats, DevTT& y) {
  const int d = x.d;
  T2S2_TRY(tt_alloc(cx, y, d, x.m, x.r, 0));
  Ctx c64 = cx;
  c64.contract_prec = T2S2_FP64;
  for (int k = 0; k < d; ++k) {
    const int m = x.m[k], ra = x.r[k], rb = x.r[k + 1];
    Gemm<double> g;
    g.M = m; g.N = rb; g.K = m; g.tA = false; g.tB = false; g.alpha = 1.0; g.beta = 0.0;
    g.A = mats[k]; g.lda = m; g.sA = 0;
    g.B = x.c[k]; g.ldb = rb; g.sB = (long)m * rb;
    g.C = y.c[k]; g.ldc = rb; g.sC = (long)m * rb;
    g.batch = ra;
    T2S2_TRY(contract_gemm(c64, g));
  }
  return T2S2_OK;
}

namespace {
// s + e = a + b exactly (no multiplication, so nothing can be fused)
void host_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
}  // namespace

t2s2_status residual_full(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass, double c_op,
                          double* out) {
  // |b|^2 - 2<b, y> + |y|^2 in double-double, y the full operator applied
  // to x (ranks 3 r_x): z = b - y is never formed, so its ranks (r_b + 3 r_x)
  // meet no limit of the orthogonalisation
  const size_t mk = cx.ar->mark();
  DevTT y;
  T2S2_TRY(apply_full(op, cx, x, y, c_mass, c_op));
  const DevTT* pu[3] = {&b, &y, &b};
  const DevTT* pv[3] = {&y, &y, &b};
  double hi[3] = {0.0, 0.0, 0.0}, lo[3] = {0.0, 0.0, 0.0};
  T2S2_TRY(tt_dots_dd(cx, 3, pu, pv, hi, lo));
  cx.ar->release(mk);
  double s1, e1, s2, e2;
  host_two_sum(hi[2], -2.0 * hi[0], s1, e1);
  host_two_sum(s1, hi[1], s2, e2);
  const double r2v = s2 + (((lo[2] - 2.0 * lo[0]) + lo[1]) + (e1 + e2));
  const double bn = std::sqrt(std::max(hi[2] + lo[2], 0.0));
  const double zn = std::sqrt(std::max(r2v, 0.0));
  *out = bn > 0.0 ? zn / bn : zn;
  return T2S2_OK;
}

t2s2_status contract_gemm(Ctx& cx, const Gemm<double>& g) {
  if (cx.contract_prec == T2S2_BF16_REFINE || cx.contract_prec == T2S2_TF32_REFINE) {
    const size_t need = gemm_tc_workspace_bytes(g, cx.contract_prec);
    const size_t mk = cx.ar->mark();
    void* ws = need ? cx.ar->get(need) : nullptr;
    if (need && !ws) return T2S2_ENOMEM;
    const t2s2_status s = gemm_tc(g, cx.contract_prec, ws, need, cx.dstat + kStatTensorCore, cx.st);
    cx.ar->release(mk);
    return s;
  }
  const size_t need = gemm_workspace(g);
  const size_t mk = cx.ar->mark();
  double* ws = need ? aget<double>(cx, need) : nullptr;
  if (need && !ws) return T2S2_ENOMEM;
  const t2s2_status s = gemm(g, ws, need, cx.st, cx.gcnt, cx.gcnt ? kGemmCounters : 0);
  cx.ar->release(mk);
  return s;
}

t2s2_status contract_group(Ctx& cx, const Gemm<double>* gs, int n) {
  if (cx.contract_prec == T2S2_BF16_REFINE || cx.contract_prec == T2S2_TF32_REFINE || !cx.gcnt || n == 1) {
    for (int i = 0; i < n; ++i) T2S2_TRY(contract_gemm(cx, gs[i]));
    return T2S2_OK;
  }
  const size_t need = gemm_group_workspace(gs, n);
  const size_t mk = cx.ar->mark();
  double* ws = need ? aget<double>(cx, need) : nullptr;
  if (need && !ws) return T2S2_ENOMEM;
  const t2s2_status s = gemm_group(gs, n, ws, need, cx.st, cx.gcnt, kGemmCounters);
  cx.ar->release(mk);
  return s;
}

t2s2_status tensor_core_status(Ctx& cx) {
  int h = 0;
  T2S2_CUDA_TRY(cudaMemcpyAsync(cx.hbuf, cx.dstat + kStatTensorCore, sizeof(int), cudaMemcpyDeviceToHost, cx.st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(cx.st));
  std::memcpy(&h, cx.hbuf, sizeof(int));
  return h ? T2S2_ETIMEOUT : T2S2_OK;
}

size_t max_core(const t2s2_tt* t) {
  size_t s = 0;
  for (int k = 0; k < t->d; ++k) s = std::max(s, t->cap[k]);
  return s;
}

t2s2_status residual_impl(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass,
                          double c_op, bool transformed, double* out, double* bnorm_io) {
  size_t mark = cx.ar->mark();
  DevTT y;
  int r2[T2S2_MAX_D + 1];
  for (int k = 0; k <= op->d; ++k) r2[k] = (k == 0 || k == op->d) ? 1 : 2 * x.r[k];
  T2S2_TRY(tt_alloc(cx, y, op->d, x.m, r2, 0));
  T2S2_TRY(apply_op(op, cx, x, y, c_mass, c_op, transformed));
  int rz = 1;
  for (int k = 0; k <= op->d; ++k) rz = std::max(rz, b.r[k] + y.r[k]);
  double rn;
  if (rz > kSmallMax) {
    // z = b - y is past the orthogonalisation's rank limit: |z|^2 from the
    // double-double inner products instead
    const DevTT* pu[3] = {&b, &y, &b};
    const DevTT* pv[3] = {&y, &y, &b};
    double hi[3] = {0.0, 0.0, 0.0}, lo[3] = {0.0, 0.0, 0.0};
    T2S2_TRY(tt_dots_dd(cx, 3, pu, pv, hi, lo));
    double s1, e1, s2, e2;
    host_two_sum(hi[2], -2.0 * hi[0], s1, e1);
    host_two_sum(s1, hi[1], s2, e2);
    rn = std::sqrt(std::max(s2 + (((lo[2] - 2.0 * lo[0]) + lo[1]) + (e1 + e2)), 0.0));
  } else {
    DevTT z;
    T2S2_TRY(tt_axpby(cx, 1.0, b, -1.0, y, z));
    T2S2_TRY(tt_orth_right(cx, z));
    T2S2_TRY(core_norm(cx, z.c[0], z.core_elems(0), &rn));
  }
  double bn = bnorm_io ? *bnorm_io : -1.0;
  if (bn < 0) {
    T2S2_TRY(tt_norm(cx, b, &bn));
    if (bnorm_io) *bnorm_io = bn;
  }
  *out = (bn > 0) ? rn / bn : rn;
  cx.ar->release(mark);
  return T2S2_OK;
}

// ||b - (c_mass M + c_op A) x|| / ||b|| through <z, z> in double-double
// (ttdot.cu), z = b - A x as a TT sum: no orthogonalisation of z.  The
// double-double sums carry ~1e-28 |b|^2 of error, i.e. ~1e-4 relative in a
// residual of 1e-12 |b|; a CholeskyQR-orthogonalised z (residual_impl) would
// drop directions below ~2e-13 of its largest singular value in its unshifted
// passes, so it is only the last resort, below kDDFloor, where neither
// resolves the residual.
constexpr double kDDFloor = 1e-13;
constexpr double kScreen = 1e-5;


t2s2_status residual_fast(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass, double c_op,
                          double* out, ResidualCache* rc, bool screen) {
  size_t mark = cx.ar->mark();
  DevTT y;
  int r2[T2S2_MAX_D + 1];
  for (int k = 0; k <= op->d; ++k) r2[k] = (k == 0 || k == op->d) ? 1 : 2 * x.r[k];
  T2S2_TRY(tt_alloc(cx, y, op->d, x.m, r2, 0));
  T2S2_TRY(apply_op(op, cx, x, y, c_mass, c_op, false));
  if (screen) {
    // binary64 |b|^2 - 2<b, y> + |y|^2: its cancellation noise (~1e-8
    // relative in the norm) is irrelevant for a residual far above kScreen
    const bool with_bb = rc->bnorm < 0.0;
    const DevTT* pu[3] = {&b, &y, &b};
    const DevTT* pv[3] = {&y, &y, &b};
    double dots[3] = {0.0, 0.0, 0.0};
    T2S2_TRY(tt_dots(cx, with_bb ? 3 : 2, pu, pv, dots));
    const double bb = with_bb ? dots[2] : rc->bnorm * rc->bnorm;
    const double r2v = std::max(bb - 2.0 * dots[0] + dots[1], 0.0);
    const double est = (bb > 0) ? std::sqrt(r2v / bb) : std::sqrt(r2v);
    if (est > kScreen) {
      if (with_bb) rc->bnorm = std::sqrt(bb);
      *out = est;
      cx.ar->release(mark);
      return T2S2_OK;
    }
  }
  // |b|^2 - 2<b, y> + |y|^2 with every inner product in double-double (|b|^2
  // once per right-hand side), combined with error-free sums
  const bool with_bb = rc->bb_hi < 0.0;
  const DevTT* pu[3] = {&b, &y, &b};
  const DevTT* pv[3] = {&y, &y, &b};
  double hi[3] = {0.0, 0.0, 0.0}, lo[3] = {0.0, 0.0, 0.0};
  T2S2_TRY(tt_dots_dd(cx, with_bb ? 3 : 2, pu, pv, hi, lo));
  if (with_bb) {
    rc->bb_hi = hi[2];
    rc->bb_lo = lo[2];
  }
  double s1, e1, s2, e2;
  host_two_sum(rc->bb_hi, -2.0 * hi[0], s1, e1);
  host_two_sum(s1, hi[1], s2, e2);
  const double r2v = s2 + (((rc->bb_lo - 2.0 * lo[0]) + lo[1]) + (e1 + e2));
  const double bb = rc->bb_hi + rc->bb_lo;
  if (rc->bnorm < 0.0) rc->bnorm = std::sqrt(std::max(bb, 0.0));
  const double bn = rc->bnorm;
  const double zn = std::sqrt(std::max(r2v, 0.0));
  double res = (bn > 0) ? zn / bn : zn;
  cx.ar->release(mark);
  if (res < kDDFloor) T2S2_TRY(residual_impl(op, cx, b, x, c_mass, c_op, false, &res, &rc->bnorm));
  *out = res;
  return T2S2_OK;
}

// Residual screen sqrt(|b|^2 - 2<b, A x> + |A x|^2) / |b|, with y = A x and
// the two (three, when *bb_io < 0: then |b|^2 is returned in *bb_io) inner
// products in one launch.
t2s2_status residual_estimate(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& x, double c_mass,
                              double c_op, double* bb_io, double* out) {
  size_t mark = cx.ar->mark();
  DevTT y;
  int r2[T2S2_MAX_D + 1];
  for (int k = 0; k <= op->d; ++k) r2[k] = (k == 0 || k == op->d) ? 1 : 2 * x.r[k];
  T2S2_TRY(tt_alloc(cx, y, op->d, x.m, r2, 0));
  T2S2_TRY(apply_op(op, cx, x, y, c_mass, c_op, false));
  const bool with_bb = *bb_io < 0.0;
  const DevTT* pu[3] = {&b, &y, &b};
  const DevTT* pv[3] = {&y, &y, &b};
  double dots[3] = {0.0, 0.0, 0.0};
  T2S2_TRY(tt_dots(cx, with_bb ? 3 : 2, pu, pv, dots));
  if (with_bb) *bb_io = dots[2];
  const double bb = *bb_io;
  const double r2v = bb - 2.0 * dots[0] + dots[1];
  *out = (bb > 0) ? std::sqrt(std::max(r2v, 0.0) / bb) : std::sqrt(std::max(r2v, 0.0));
  cx.ar->release(mark);
  return T2S2_OK;
}

}  // namespace t2s2

using namespace t2s2;

extern "C" {

const char* t2s2_strerror(t2s2_status s) {
  switch (s) {
    case T2S2_OK: return "ok";
    case T2S2_EINVAL: return "invalid argument";
    case T2S2_ENOMEM: return "out of memory or TT capacity exceeded";
    case T2S2_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case T2S2_ENOCONV: return "solver did not reach the tolerance within the sweep cap";
    case T2S2_ETIMEOUT: return "bounded device wait timed out";
    case T2S2_ENOTIMPL: return "not implemented";
    case T2S2_ENODEV: return "no sm_103 CUDA device";
  }
  return "unknown status";
}

int t2s2_device_count(void) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) return 0;
  int good = 0;
  for (int i = 0; i < n; ++i) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, i) == cudaSuccess && p.major == 10 && p.minor == 3) ++good;
  }
  return good;
}

// Device copies of every dimension's matrices (FP64 and FP32) and the
// per-operator buffers, for an operator whose host dimensions are built.
// Frees the operator on failure.
static t2s2_status upload_operator(t2s2_op op, cudaStream_t st, t2s2_op* out) {
  size_t total = 0;
  for (int k = 0; k < op->d; ++k) total += (size_t)kMatsPerDim * op->m[k] * op->m[k];
  std::vector<double> host(total, 0.0);
  size_t off = 0;
  std::vector<size_t> offs(op->d);
  for (int k = 0; k < op->d; ++k) {
    const int m = op->m[k];
    const size_t mm = (size_t)m * m;
    offs[k] = off;
    const Dim1D& D = op->dims[k];
    std::copy(D.Rt.begin(), D.Rt.end(), host.begin() + off + 0 * mm);
    std::copy(D.Lt.begin(), D.Lt.end(), host.begin() + off + 1 * mm);
    std::copy(D.Rinv.begin(), D.Rinv.end(), host.begin() + off + 2 * mm);
    std::copy(D.B.begin(), D.B.end(), host.begin() + off + 3 * mm);
    for (int i = 0; i < m; ++i) host[off + 4 * mm + (size_t)i * m + i] = 1.0;
    std::copy(D.Tr.begin(), D.Tr.end(), host.begin() + off + 5 * mm);
    std::copy(D.Ti.begin(), D.Ti.end(), host.begin() + off + 6 * mm);
    std::copy(D.Zr.begin(), D.Zr.end(), host.begin() + off + 7 * mm);
    std::copy(D.Zi.begin(), D.Zi.end(), host.begin() + off + 8 * mm);
    off += kMatsPerDim * mm;
  }
  std::vector<float> hostf(host.begin(), host.end());
  cudaError_t e = cudaMalloc(&op->dmat, sizeof(double) * total);
  if (e != cudaSuccess) { delete op; return T2S2_ENOMEM; }
  e = cudaMalloc(&op->fmat, sizeof(float) * total);
  if (e != cudaSuccess) { t2s2_op_destroy(op); return T2S2_ENOMEM; }
  e = cudaMemcpyAsync(op->dmat, host.data(), sizeof(double) * total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(op->fmat, hostf.data(), sizeof(float) * total, cudaMemcpyHostToDevice, st);
  // the full matrices of the space dimensions (boundary-data lifting)
  size_t nfull = 0;
  for (int k = 0; k < op->d; ++k) nfull += op->dims[k].Rf.size() + op->dims[k].Lf.size();
  if (e == cudaSuccess && nfull > 0) {
    std::vector<double> hf;
    hf.reserve(nfull);
    for (int k = 0; k < op->d; ++k) {
      hf.insert(hf.end(), op->dims[k].Rf.begin(), op->dims[k].Rf.end());
      hf.insert(hf.end(), op->dims[k].Lf.begin(), op->dims[k].Lf.end());
    }
    e = cudaMalloc(&op->dfull, sizeof(double) * nfull);
    if (e == cudaSuccess) e = cudaMemcpy(op->dfull, hf.data(), sizeof(double) * nfull, cudaMemcpyHostToDevice);
    size_t o = 0;
    for (int k = 0; k < op->d && e == cudaSuccess; ++k) {
      if (op->dims[k].Rf.empty()) continue;
      op->dRf[k] = op->dfull + o;
      o += op->dims[k].Rf.size();
      op->dLf[k] = op->dfull + o;
      o += op->dims[k].Lf.size();
    }
  }
  if (e == cudaSuccess) e = cudaMallocHost(&op->hbuf, sizeof(double) * 4096);
  if (e == cudaSuccess) e = cudaMalloc(&op->dstat, sizeof(int) * 64);
  if (e == cudaSuccess) e = cudaMalloc(&op->gcnt, sizeof(int) * kGemmCounters);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->gcnt, 0, sizeof(int) * kGemmCounters, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "operator upload", __FILE__, __LINE__);
    t2s2_op_destroy(op);
    return T2S2_ECUDA;
  }
  for (int k = 0; k < op->d; ++k) {
    const size_t mm = (size_t)op->m[k] * op->m[k];
    double* base = op->dmat + offs[k];
    op->dRt[k] = base;
    op->dLt[k] = base + mm;
    op->dRinv[k] = base + 2 * mm;
    op->dB[k] = base + 3 * mm;
    op->dI[k] = base + 4 * mm;
    op->dTr[k] = base + 5 * mm;
    op->dTi[k] = base + 6 * mm;
    op->dZr[k] = base + 7 * mm;
    op->dZi[k] = base + 8 * mm;
    for (int j = 0; j < kMatsPerDim; ++j) op->fptr[j][k] = op->fmat + offs[k] + j * mm;
  }
  *out = op;
  return T2S2_OK;
}

t2s2_status t2s2_build_operator(const t2s2_problem* prob, void* stream, t2s2_op* out) {
  if (!prob || !out || !prob->n || !prob->beta) return T2S2_EINVAL;
  *out = nullptr;
  if (prob->d < 1 || prob->d > T2S2_MAX_D || !(prob->eps > 0.0) || !std::isfinite(prob->eps))
    return T2S2_EINVAL;
  for (int k = 0; k < prob->d; ++k) {
    if (prob->n[k] < 3 || prob->n[k] > T2S2_MAX_N || !std::isfinite(prob->beta[k])) return T2S2_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return T2S2_ENODEV;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess || p.major != 10 || p.minor != 3) return T2S2_ENODEV;
  t2s2_op op = new t2s2_op_s();
  op->device = dev;
  op->d = prob->d;
  op->eps = prob->eps;
  op->plain = prob->plain_sc;
  op->dims.resize(op->d);
  for (int k = 0; k < op->d; ++k) {
    op->n[k] = prob->n[k];
    op->m[k] = prob->n[k] - 2;
    op->beta[k] = prob->beta[k];
    if (!build_dimension(op->n[k], op->eps, op->beta[k], op->plain, &op->dims[k])) {
      delete op;
      return T2S2_EINVAL;
    }
  }
  return upload_operator(op, static_cast<cudaStream_t>(stream), out);
}

t2s2_status t2s2_build_operator_var(const t2s2_problem_var* var, void* stream, t2s2_op* out) {
  if (!var || !out) return T2S2_EINVAL;
  const t2s2_problem* prob = &var->base;
  if (!prob->n || !prob->beta || !std::isfinite(var->rho0)) return T2S2_EINVAL;
  *out = nullptr;
  if (prob->d < 1 || prob->d > T2S2_MAX_D || !(prob->eps > 0.0) || !std::isfinite(prob->eps))
    return T2S2_EINVAL;
  for (int k = 0; k < prob->d; ++k) {
    if (prob->n[k] < 3 || prob->n[k] > T2S2_MAX_N || !std::isfinite(prob->beta[k])) return T2S2_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return T2S2_ENODEV;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess || p.major != 10 || p.minor != 3) return T2S2_ENODEV;
  t2s2_op op = new t2s2_op_s();
  op->device = dev;
  op->d = prob->d;
  op->eps = prob->eps;
  op->plain = prob->plain_sc;
  op->dims.resize(op->d);
  for (int k = 0; k < op->d; ++k) {
    op->n[k] = prob->n[k];
    op->m[k] = prob->n[k] - 2;
    op->beta[k] = prob->beta[k];
    std::function<double(double)> b, r;
    if (var->beta_fn) b = [var, k](double x) { return var->beta_fn(k, x, var->ctx); };
    const double r0 = k == 0 ? var->rho0 : 0.0;
    if (var->rho_fn) {
      r = [var, k, r0](double x) { return var->rho_fn(k, x, var->ctx) + r0; };
    } else if (r0 != 0.0) {
      r = [r0](double) { return r0; };
    }
    if (!build_dimension_coef(op->n[k], op->eps, op->beta[k], op->plain, b, r, &op->dims[k])) {
      delete op;
      return T2S2_EINVAL;
    }
  }
  // product reaction: P_k = diag(pi_k(eta)) Rt_k and the product of the means
  std::vector<double> hp;
  if (var->prod_fn) {
    op->has_prod = 1;
    op->rho_bar = 1.0;
    for (int k = 0; k < op->d; ++k) {
      const Dim1D& D = op->dims[k];
      const int m = op->m[k];
      double mean = 0.0;
      for (int j = 0; j < m; ++j) {
        const double pj = var->prod_fn(k, D.eta[j], var->ctx);
        if (!std::isfinite(pj)) {
          delete op;
          return T2S2_EINVAL;
        }
        mean += pj / m;
        for (int i = 0; i < m; ++i) hp.push_back(pj * D.Rt[(size_t)j * m + i]);
      }
      op->rho_bar *= mean;
    }
  }
  t2s2_status st = upload_operator(op, static_cast<cudaStream_t>(stream), out);
  if (st != T2S2_OK || hp.empty()) return st;
  t2s2_op o = *out;
  if (cudaMalloc(&o->dprod, sizeof(double) * hp.size()) != cudaSuccess ||
      cudaMemcpy(o->dprod, hp.data(), sizeof(double) * hp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    t2s2_op_destroy(o);
    *out = nullptr;
    return T2S2_ENOMEM;
  }
  size_t off = 0;
  for (int k = 0; k < o->d; ++k) {
    o->dP[k] = o->dprod + off;
    off += (size_t)o->m[k] * o->m[k];
  }
  return T2S2_OK;
}

t2s2_status t2s2_build_spacetime_operator(const t2s2_problem* space, int n_t, double t_len, void* stream,
                                          t2s2_op* out) {
  if (!space || !out || !space->n || !space->beta) return T2S2_EINVAL;
  *out = nullptr;
  if (space->d < 1 || space->d + 1 > T2S2_MAX_D || !(space->eps > 0.0) || !std::isfinite(space->eps))
    return T2S2_EINVAL;
  if (n_t < 3 || n_t > T2S2_MAX_N || !(t_len > 0.0) || !std::isfinite(t_len)) return T2S2_EINVAL;
  for (int k = 0; k < space->d; ++k) {
    if (space->n[k] < 3 || space->n[k] > T2S2_MAX_N || !std::isfinite(space->beta[k])) return T2S2_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return T2S2_ENODEV;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess || p.major != 10 || p.minor != 3) return T2S2_ENODEV;
  t2s2_op op = new t2s2_op_s();
  op->device = dev;
  op->d = space->d + 1;
  op->eps = space->eps;
  op->plain = space->plain_sc;
  op->dims.resize(op->d);
  // dimension 0: time on [0, t_len] mapped onto [-1, 1]
  op->n[0] = n_t;
  op->m[0] = n_t - 1;
  op->beta[0] = 2.0 / t_len;
  if (!build_time_dimension(n_t, op->beta[0], &op->dims[0])) {
    delete op;
    return T2S2_EINVAL;
  }
  for (int k = 1; k < op->d; ++k) {
    op->n[k] = space->n[k - 1];
    op->m[k] = space->n[k - 1] - 2;
    op->beta[k] = space->beta[k - 1];
    if (!build_dimension(op->n[k], op->eps, op->beta[k], op->plain, &op->dims[k])) {
      delete op;
      return T2S2_EINVAL;
    }
  }
  return upload_operator(op, static_cast<cudaStream_t>(stream), out);
}

t2s2_status t2s2_op_destroy(t2s2_op op) {
  if (!op) return T2S2_OK;
  if (op->dmat) cudaFree(op->dmat);
  if (op->fmat) cudaFree(op->fmat);
  if (op->dfull) cudaFree(op->dfull);
  if (op->dprod) cudaFree(op->dprod);
  if (op->arena.base) cudaFree(op->arena.base);
  if (op->hbuf) cudaFreeHost(op->hbuf);
  if (op->dstat) cudaFree(op->dstat);
  if (op->gcnt) cudaFree(op->gcnt);
  if (op->zcache) cudaFree(op->zcache);
  if (op->ev_fork) cudaEventDestroy(op->ev_fork);
  if (op->ev_join) cudaEventDestroy(op->ev_join);
  if (op->side) cudaStreamDestroy(op->side);
  op->free_solver_buffers();
  delete op;
  return T2S2_OK;
}

t2s2_status t2s2_dim_matrices(int n, double eps, double beta, int kind, double* x, double* eta, double* Rt,
                              double* Lt, double* Rb, double* Lb) {
  if (n < 3 || n > T2S2_MAX_N) return T2S2_EINVAL;
  if (kind != T2S2_DIM_SPACE && kind != T2S2_DIM_SPACE_PLAIN && kind != T2S2_DIM_TIME) return T2S2_EINVAL;
  if (!std::isfinite(eps) || !std::isfinite(beta)) return T2S2_EINVAL;
  const bool time = kind == T2S2_DIM_TIME;
  if (time ? eps < 0.0 : !(eps > 0.0)) return T2S2_EINVAL;
  const int N = n - 1, m = time ? n - 1 : n - 2, nb = time ? 1 : 2;
  std::vector<double> xs(n), pts(m);
  gll_points(N, xs.data());
  if (time) {
    gauss_points(N, pts.data());
  } else {
    collocation_points(N, eps, beta, kind == T2S2_DIM_SPACE_PLAIN, pts.data());
  }
  std::vector<double> R((size_t)m * n), D((size_t)m * n), D2((size_t)m * n);
  lagrange_matrices(N, xs.data(), m, pts.data(), R.data(), D.data(), D2.data());
  auto L = [&](size_t e) { return beta * D[e] - eps * D2[e]; };
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) {
      const size_t e = (size_t)j * n + i + 1;  // unknown i is node i + 1
      if (Rt) Rt[(size_t)j * m + i] = R[e];
      if (Lt) Lt[(size_t)j * m + i] = L(e);
    }
    for (int q = 0; q < nb; ++q) {
      const size_t e = (size_t)j * n + (q == 0 ? 0 : N);
      if (Rb) Rb[(size_t)j * nb + q] = R[e];
      if (Lb) Lb[(size_t)j * nb + q] = L(e);
    }
  }
  if (x) std::copy(xs.begin(), xs.end(), x);
  if (eta) std::copy(pts.begin(), pts.end(), eta);
  return T2S2_OK;
}

t2s2_status t2s2_op_nodes(t2s2_op op, int k, double* x, double* eta) {
  if (!op || k < 0 || k >= op->d) return T2S2_EINVAL;
  const Dim1D& D = op->dims[k];
  if (x) std::copy(D.x.begin(), D.x.end(), x);
  if (eta) std::copy(D.eta.begin(), D.eta.end(), eta);
  return T2S2_OK;
}

t2s2_status t2s2_op_matrices(t2s2_op op, int k, double* Rt, double* Lt) {
  if (!op || k < 0 || k >= op->d) return T2S2_EINVAL;
  const Dim1D& D = op->dims[k];
  if (Rt) std::copy(D.Rt.begin(), D.Rt.end(), Rt);
  if (Lt) std::copy(D.Lt.begin(), D.Lt.end(), Lt);
  return T2S2_OK;
}

t2s2_status t2s2_apply(t2s2_op op, const t2s2_tt* x, t2s2_tt* y, double c_mass, double c_op,
                       t2s2_precision prec, void* stream) {
  if (!op || !x || !y) return T2S2_EINVAL;
  if (prec < T2S2_FP64 || prec > T2S2_BF16_REFINE) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, x));
  T2S2_TRY(check_out_tt(op, y));
  for (int k = 0; k < op->d; ++k)
    if (y->cores[k] == x->cores[k]) return T2S2_EINVAL;
  if (op->has_prod) {
    // the rank-3 operator: FP64, ranks 3 r_x
    T2S2_TRY(ensure_arena(op, 16 * tt_bytes(x) + ((size_t)4 << 20)));
    Ctx cx = make_ctx(op, stream);
    DevTT dx, dy;
    T2S2_TRY(bind_tt(cx, x, dx, true));
    T2S2_TRY(apply_full(op, cx, dx, dy, c_mass, c_op));
    return unbind_tt(cx, dy, y);
  }
  T2S2_TRY(ensure_arena(op, tt_bytes(x) + tt_bytes(y) + ((size_t)1 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT dx, dy;
  T2S2_TRY(bind_tt(cx, x, dx, true));
  T2S2_TRY(bind_tt(cx, y, dy, false));
  T2S2_TRY(apply_dispatch(op, cx, dx, dy, c_mass, c_op, prec));
  return unbind_tt(cx, dy, y);
}

t2s2_status t2s2_spacetime_rhs(t2s2_op op, const t2s2_tt* b, const t2s2_tt* u0, t2s2_tt* out, double tol,
                               int rmax, void* stream) {
  if (!op || !b || !u0 || !out || !(tol >= 0.0)) return T2S2_EINVAL;
  if (op->d < 2 || op->dims[0].R0.empty()) return T2S2_EINVAL;  // not a space-time operator
  T2S2_TRY(check_tt(op, b));
  T2S2_TRY(check_out_tt(op, out));
  const int ds = op->d - 1, mt = op->m[0];
  if (!u0->r || !u0->cores || !u0->cap || !u0->m || u0->d != ds || u0->r[0] != 1 || u0->r[ds] != 1)
    return T2S2_EINVAL;
  if (u0->loc != T2S2_DEVICE && u0->loc != T2S2_HOST) return T2S2_EINVAL;
  for (int k = 0; k < ds; ++k) {
    if (u0->m[k] != op->m[k + 1] || u0->r[k + 1] < 1 || !u0->cores[k]) return T2S2_EINVAL;
    if ((size_t)u0->r[k] * u0->m[k] * u0->r[k + 1] > u0->cap[k]) return T2S2_ENOMEM;
  }
  size_t mc = max_core(b);
  T2S2_TRY(ensure_arena(op, tt_bytes(b) * 4 + tt_bytes(u0) * 16 + tt_bytes(out) + 2 * mt * sizeof(double) +
                                12 * mc * sizeof(double) + ((size_t)16 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT db, du;
  T2S2_TRY(bind_tt(cx, b, db, true));
  T2S2_TRY(bind_tt(cx, u0, du, true));
  // M_x u0 (v = 0) and A_x u0 (v = 1): the rank-2 apply over dimensions 1..d
  DevTT y[2];
  int ry[T2S2_MAX_D + 1];
  for (int k = 0; k <= ds; ++k) ry[k] = (k == 0 || k == ds) ? 1 : 2 * du.r[k];
  for (int v = 0; v < 2; ++v) {
    T2S2_TRY(tt_alloc(cx, y[v], ds, du.m, ry, 0));
    ApplyBatch ab;
    ab.ncores = ds;
    for (int k = 0; k < ds; ++k) {
      ApplyCore& c = ab.c[k];
      c.S = op->dRt[k + 1];
      c.L = op->dLt[k + 1];
      c.X = du.c[k];
      c.Y = y[v].c[k];
      c.ra = du.r[k];
      c.m = du.m[k];
      c.rb = du.r[k + 1];
      c.kind = (ds == 1) ? kApplySingle : (k == 0 ? kApplyFirst : (k == ds - 1 ? kApplyLast : kApplyMiddle));
      c.g_op = (v == 0) ? 0.0 : 1.0;
      c.g_mass = (k == 0 && v == 0) ? 1.0 : 0.0;
    }
    T2S2_TRY(apply_fp64(ab, cx.st));
  }
  // the columns of the initial node s = -1 as rank-1 time cores in front
  double* cols = aget<double>(cx, 2 * (size_t)mt);
  if (!cols) return T2S2_ENOMEM;
  T2S2_CUDA_TRY(cudaMemcpyAsync(cols, op->dims[0].L0.data(), sizeof(double) * mt, cudaMemcpyHostToDevice, cx.st));
  T2S2_CUDA_TRY(cudaMemcpyAsync(cols + mt, op->dims[0].R0.data(), sizeof(double) * mt, cudaMemcpyHostToDevice,
                                cx.st));
  DevTT t[2];
  for (int v = 0; v < 2; ++v) {
    t[v].d = op->d;
    t[v].r[0] = 1;
    t[v].m[0] = mt;
    t[v].c[0] = cols + v * (size_t)mt;
    t[v].cap[0] = mt;
    for (int k = 0; k < ds; ++k) {
      t[v].r[k + 1] = y[v].r[k];
      t[v].m[k + 1] = y[v].m[k];
      t[v].c[k + 1] = y[v].c[k];
      t[v].cap[k + 1] = y[v].cap[k];
    }
    t[v].r[op->d] = 1;
  }
  // b_st = b - L0 (x) M_x u0 - R0 (x) A_x u0, rounded
  DevTT s1, s2;
  T2S2_TRY(tt_axpby(cx, 1.0, db, -1.0, t[0], s1));
  T2S2_TRY(tt_axpby(cx, 1.0, s1, -1.0, t[1], s2));
  T2S2_TRY(tt_round(cx, s2, tol, rmax));
  return unbind_tt(cx, s2, out);
}

t2s2_status t2s2_gemm(t2s2_op op, int M, int N, int K, int tA, int tB, double alpha, const double* A,
                      long lda, long sA, const double* B, long ldb, long sB, double beta, double* C,
                      long ldc, long sC, int batch, t2s2_precision prec, void* stream) {
  if (!op || M < 0 || N < 0 || K < 0 || batch < 0) return T2S2_EINVAL;
  if (prec < T2S2_FP64 || prec > T2S2_BF16_REFINE) return T2S2_EINVAL;
  if (M == 0 || N == 0 || batch == 0) return T2S2_OK;
  if (!C || ldc < N || (K > 0 && (!A || !B))) return T2S2_EINVAL;
  if (K > 0 && (lda < (tA ? M : K) || ldb < (tB ? K : N))) return T2S2_EINVAL;
  if (sA < 0 || sB < 0 || sC < 0) return T2S2_EINVAL;
  Gemm<double> g;
  g.M = M; g.N = N; g.K = K; g.tA = tA != 0; g.tB = tB != 0; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.sA = sA; g.B = B; g.ldb = ldb; g.sB = sB;
  g.C = C; g.ldc = ldc; g.sC = sC; g.batch = batch;
  const bool tc = prec == T2S2_BF16_REFINE || prec == T2S2_TF32_REFINE;
  const size_t ws = tc ? gemm_tc_workspace_bytes(g, prec) : gemm_workspace(g) * sizeof(double);
  T2S2_TRY(ensure_arena(op, ws + ((size_t)1 << 20)));
  Ctx cx = make_ctx(op, stream);
  cx.contract_prec = tc ? prec : T2S2_FP64;
  if (tc) T2S2_CUDA_TRY(cudaMemsetAsync(cx.dstat + kStatTensorCore, 0, sizeof(int), cx.st));
  T2S2_TRY(contract_gemm(cx, g));
  return tc ? tensor_core_status(cx) : T2S2_OK;
}

t2s2_status t2s2_round(t2s2_op op, t2s2_tt* x, double tol, int rmax, void* stream) {
  if (!op || !x || !(tol >= 0.0)) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, x));
  size_t mc = max_core(x);
  T2S2_TRY(ensure_arena(op, tt_bytes(x) * 3 + 10 * mc * sizeof(double) + ((size_t)8 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT dx;
  T2S2_TRY(bind_tt(cx, x, dx, true));
  T2S2_TRY(tt_round(cx, dx, tol, rmax));
  return unbind_tt(cx, dx, x);
}

t2s2_status t2s2_norm(t2s2_op op, const t2s2_tt* x, double* out, void* stream) {
  if (!op || !x || !out) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, x));
  size_t mc = max_core(x);
  T2S2_TRY(ensure_arena(op, tt_bytes(x) * 3 + 10 * mc * sizeof(double) + ((size_t)8 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT dx;
  T2S2_TRY(bind_tt(cx, x, dx, true));
  return tt_norm(cx, dx, out);
}

t2s2_status t2s2_diff_norm(t2s2_op op, const t2s2_tt* x, const t2s2_tt* y, double* out, void* stream) {
  if (!op || !x || !y || !out) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, x));
  T2S2_TRY(check_tt(op, y));
  size_t mc = max_core(x) + max_core(y);
  T2S2_TRY(ensure_arena(op, (tt_bytes(x) + tt_bytes(y)) * 6 + 10 * mc * sizeof(double) + ((size_t)8 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT dx, dy, z;
  T2S2_TRY(bind_tt(cx, x, dx, true));
  T2S2_TRY(bind_tt(cx, y, dy, true));
  T2S2_TRY(tt_axpby(cx, 1.0, dx, -1.0, dy, z));
  T2S2_TRY(tt_orth_right(cx, z));
  return core_norm(cx, z.c[0], z.core_elems(0), out);
}

t2s2_status t2s2_residual(t2s2_op op, const t2s2_tt* b, const t2s2_tt* x, double c_mass, double c_op,
                          double* out, void* stream) {
  if (!op || !b || !x || !out) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, b));
  T2S2_TRY(check_tt(op, x));
  size_t mc = std::max(max_core(x) * 4, max_core(b)) + 4 * max_core(x);
  T2S2_TRY(ensure_arena(op, (tt_bytes(b) + tt_bytes(x)) * 12 + 20 * mc * sizeof(double) + ((size_t)8 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT db, dx;
  T2S2_TRY(bind_tt(cx, b, db, true));
  T2S2_TRY(bind_tt(cx, x, dx, true));
  if (op->has_prod) return residual_full(op, cx, db, dx, c_mass, c_op, out);
  ResidualCache rc;
  return residual_fast(op, cx, db, dx, c_mass, c_op, out, &rc, false);
}

}  // extern "C"
