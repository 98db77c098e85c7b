// Non-zero Dirichlet data (eq. pblm:time:B, u = g on the boundary) by TT
// lifting.  The caller passes g as a TT G on the full GLL grid (n_k nodes per
// dimension; only its boundary values matter).  With the full (n-2) x n 1D
// matrices Rf, Lf (every GLL node a column), the interior equations of
// u_full = G + w, w zero on the boundary, read
//     (c_mass M + c_op A) w = b - (c_mass M_full + c_op A_full) G =: b_g,
// and u = w + G restricted to the interior nodes.  (c_mass M_full + c_op
// A_full) G is a TT-matrix-by-TT product in the rank-2 pattern of the apply,
// with rectangular 1D factors:
//     first [G_1 X, Rf_1 X], middle [[Rf X, 0], [c_op Lf X, Rf X]],
//     last [Rf X; c_op Lf X],  G_1 = c_op Lf_1 + c_mass Rf_1,
// X the cores of G, each block a mode-2 product (n-2) x n by r_a x n x r_b.
// These products are small (2 (n-2) n r_a r_b per block) and run once per
// solve: one thread per output element, the sum over the n nodes in order.
#include <algorithm>
#include <cmath>

#include "api_internal.h"

namespace t2s2 {
namespace {

struct LiftCore {
  const double* G;  // ra x n x rb
  double* Y;        // (ya ra) x m x (yb rb)
  const double* R;  // m x n
  const double* L;  // m x n
  int ra, n, rb, m, kind;
  double cL, cR;    // the lower-left slot holds cL Lf + cR Rf
};

struct LiftArgs {
  LiftCore c[T2S2_MAX_D];
  long start[T2S2_MAX_D + 1];  // prefix sums of output elements
  int ncores;
};

__global__ void lift_kernel(LiftArgs a) {
  const long total = a.start[a.ncores];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    int k = 0;
    while (e >= a.start[k + 1]) ++k;
    const LiftCore& c = a.c[k];
    const long o = e - a.start[k];
    const int ya = (c.kind == kApplyMiddle || c.kind == kApplyLast) ? 2 : 1;
    const int yb = (c.kind == kApplyMiddle || c.kind == kApplyFirst) ? 2 : 1;
    const int cols = yb * c.rb;
    const int B = (int)(o % cols);
    const int i = (int)((o / cols) % c.m);
    const int A = (int)(o / ((long)cols * c.m));
    const int al = A / c.ra, aa = A % c.ra, be = B / c.rb, bb = B % c.rb;
    (void)ya;
    // which 1D factor this block carries (0: none)
    double wr = 0.0, wl = 0.0;
    if (c.kind == kApplySingle) {
      wr = c.cR, wl = c.cL;
    } else if (c.kind == kApplyFirst) {
      if (be == 0) wr = c.cR, wl = c.cL; else wr = 1.0;
    } else if (c.kind == kApplyLast) {
      if (al == 0) wr = 1.0; else wl = c.cL;
    } else {
      if (al == be) wr = 1.0;
      else if (al == 1 && be == 0) wl = c.cL;
    }
    double s = 0.0;
    if (wr != 0.0 || wl != 0.0) {
      const double* Rr = c.R + (long)i * c.n;
      const double* Lr = c.L + (long)i * c.n;
      const double* g = c.G + (long)aa * c.n * c.rb + bb;
      for (int j = 0; j < c.n; ++j) s = fma(wr * Rr[j] + wl * Lr[j], g[(long)j * c.rb], s);
    }
    c.Y[o] = s;
  }
}

// Interior slice of a full-grid core: out[a, i, b] = in[a, i + 1, b].
__global__ void interior_kernel(const double* in, double* out, int ra, int n, int rb) {
  const int m = n - 2;
  const long total = (long)ra * m * rb;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb), i = (int)((e / rb) % m), a = (int)(e / ((long)rb * m));
    out[e] = in[((long)a * n + i + 1) * rb + b];
  }
}

int blocks_for_elems(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 4L * kNumSMs)); }

// A full-grid TT: pointers present, mode sizes n_k of the operator, device
// or host, ranks within capacity.
t2s2_status check_full_tt(t2s2_op op, const t2s2_tt* t) {
  if (!t || !t->r || !t->cores || !t->cap || !t->m) return T2S2_EINVAL;
  if (t->d != op->d) return T2S2_EINVAL;
  if (t->loc != T2S2_DEVICE && t->loc != T2S2_HOST) return T2S2_EINVAL;
  if (t->r[0] != 1 || t->r[t->d] != 1) return T2S2_EINVAL;
  for (int k = 0; k < t->d; ++k) {
    if (t->m[k] != op->n[k] || !op->dRf[k]) return T2S2_EINVAL;
    if (t->r[k + 1] < 1 || !t->cores[k]) return T2S2_EINVAL;
    if ((size_t)t->r[k] * t->m[k] * t->r[k + 1] > t->cap[k]) return T2S2_ENOMEM;
  }
  return T2S2_OK;
}

size_t full_bytes(const t2s2_tt* g) {
  size_t s = 0;
  for (int k = 0; k < g->d; ++k) s += (size_t)g->r[k] * g->m[k] * g->r[k + 1];
  return s * sizeof(double);
}

// y = (c_mass M_full + c_op A_full) g, ranks 2 r_g inside (allocated here).
t2s2_status lift_apply(t2s2_op op, Ctx& cx, const DevTT& g, double c_mass, double c_op, DevTT& y) {
  const int d = op->d;
  int ry[T2S2_MAX_D + 1];
  for (int k = 0; k <= d; ++k) ry[k] = (k == 0 || k == d) ? 1 : 2 * g.r[k];
  T2S2_TRY(tt_alloc(cx, y, d, op->m, ry, 0));
  LiftArgs a;
  a.ncores = d;
  a.start[0] = 0;
  for (int k = 0; k < d; ++k) {
    LiftCore& c = a.c[k];
    c.G = g.c[k];
    c.Y = y.c[k];
    c.R = op->dRf[k];
    c.L = op->dLf[k];
    c.ra = g.r[k];
    c.n = op->n[k];
    c.rb = g.r[k + 1];
    c.m = op->m[k];
    c.kind = (d == 1) ? kApplySingle : (k == 0 ? kApplyFirst : (k == d - 1 ? kApplyLast : kApplyMiddle));
    c.cL = c_op;
    c.cR = (k == 0) ? c_mass : 0.0;
    a.start[k + 1] = a.start[k] + (long)y.core_elems(k);
  }
  lift_kernel<<<blocks_for_elems(a.start[d]), 256, 0, cx.st>>>(a);
  T2S2_CUDA_TRY(cudaGetLastError());
  return T2S2_OK;
}

// b_g = rndg(b - (c_mass M_full + c_op A_full) g, tol, rmax), in the arena.
t2s2_status lifted_rhs(t2s2_op op, Ctx& cx, const DevTT& b, const DevTT& g, double c_mass, double c_op,
                       double tol, int rmax, DevTT& out) {
  DevTT y;
  T2S2_TRY(lift_apply(op, cx, g, c_mass, c_op, y));
  T2S2_TRY(tt_axpby(cx, 1.0, b, -1.0, y, out));
  return tt_round(cx, out, tol, rmax);
}

// The interior slice of a full-grid TT, in the arena.
t2s2_status interior_of(t2s2_op op, Ctx& cx, const DevTT& g, DevTT& gi) {
  T2S2_TRY(tt_alloc(cx, gi, op->d, op->m, g.r, 0));
  for (int k = 0; k < op->d; ++k) {
    const long n = (long)gi.core_elems(k);
    interior_kernel<<<blocks_for_elems(n), 256, 0, cx.st>>>(g.c[k], gi.c[k], g.r[k], op->n[k], g.r[k + 1]);
    T2S2_CUDA_TRY(cudaGetLastError());
  }
  return T2S2_OK;
}

int max_rank(const t2s2_tt* t) {
  int r = 1;
  for (int k = 0; k <= t->d; ++k) r = std::max(r, t->r[k]);
  return r;
}

}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" {

t2s2_status t2s2_dirichlet_rhs(t2s2_op op, const t2s2_tt* b, const t2s2_tt* g, double c_mass, double c_op,
                               t2s2_tt* out, double tol, int rmax, void* stream) {
  if (!op || !b || !g || !out || !(tol >= 0.0) || !std::isfinite(c_mass) || !std::isfinite(c_op))
    return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, b));
  T2S2_TRY(check_full_tt(op, g));
  T2S2_TRY(check_out_tt(op, out));
  const size_t mc = max_core(b) + 16 * (size_t)max_rank(g) * max_rank(g) * T2S2_MAX_N;
  T2S2_TRY(ensure_arena(op, 4 * tt_bytes(b) + 12 * full_bytes(g) + 12 * mc * sizeof(double) +
                                tt_bytes(out) + ((size_t)16 << 20)));
  Ctx cx = make_ctx(op, stream);
  DevTT db, dg, s;
  T2S2_TRY(bind_tt(cx, b, db, true));
  T2S2_TRY(bind_tt(cx, g, dg, true));
  T2S2_TRY(lifted_rhs(op, cx, db, dg, c_mass, c_op, tol, rmax, s));
  return unbind_tt(cx, s, out);
}

t2s2_status t2s2_solve_dirichlet(t2s2_op op, const t2s2_tt* b, const t2s2_tt* g, t2s2_tt* x, double c_mass,
                                 double c_op, double tol, int rmax, int max_sweeps, t2s2_precision prec,
                                 void* stream, t2s2_solve_info* info) {
  if (!g) return t2s2_solve(op, b, x, c_mass, c_op, tol, rmax, max_sweeps, prec, stream, info);
  if (!op || !b || !x || !(tol > 0.0) || rmax < 1 || max_sweeps < 0) return T2S2_EINVAL;
  if (prec < T2S2_FP64 || prec > T2S2_BF16_REFINE) return T2S2_EINVAL;
  if (!std::isfinite(c_mass) || !std::isfinite(c_op)) return T2S2_EINVAL;
  T2S2_TRY(check_tt(op, b));
  T2S2_TRY(check_full_tt(op, g));
  T2S2_TRY(check_tt(op, x));
  const int rg = max_rank(g), rf = max_rank(b) + 2 * rg;
  const size_t mc = max_core(b) + 16 * (size_t)rg * rg * T2S2_MAX_N;
  size_t need = solve_bytes(op, rmax, std::min(rf, kSmallMax), prec) + 4 * tt_bytes(b) + 12 * full_bytes(g) +
                12 * mc * sizeof(double) + 6 * tt_bytes(x) + ((size_t)16 << 20);
  T2S2_TRY(ensure_arena(op, need));
  Ctx cx = make_ctx(op, stream);
  DevTT db, dg, dx, bg, gi, u;
  T2S2_TRY(bind_tt(cx, b, db, true));
  T2S2_TRY(bind_tt(cx, g, dg, true));
  T2S2_TRY(bind_tt(cx, x, dx, true));
  // the lifted source, rounded well below the solve's tolerance
  T2S2_TRY(lifted_rhs(op, cx, db, dg, c_mass, c_op, 1e-2 * tol, kSmallMax, bg));
  t2s2_status st = solve_run(op, cx, bg, dx, c_mass, c_op, tol, rmax, max_sweeps, prec, info);
  if (st != T2S2_OK && st != T2S2_ENOCONV) return st;
  // u = w + g on the interior nodes as the exact TT sum (ranks add), not
  // recompressed: when g carries most of u, w lies in directions of u whose
  // singular values are small next to u's largest, and the orthogonalisation
  // of a recompression would lose them there while the operator amplifies
  // them (the residual of the rounded sum grew a thousandfold in tests)
  T2S2_TRY(interior_of(op, cx, dg, gi));
  T2S2_TRY(tt_axpby(cx, 1.0, dx, 1.0, gi, u));
  if (info) {
    int mr = 1;
    for (int k = 0; k <= op->d; ++k) mr = std::max(mr, u.r[k]);
    info->max_rank = mr;
  }
  t2s2_status st2 = unbind_tt(cx, u, x);
  return st2 != T2S2_OK ? st2 : st;
}

}  // extern "C"
