// Alternating TT solver (AMEn) and time steps.
#include "api_internal.h"

void t2s2_op_s::free_solver_buffers() {}

namespace t2s2 {
t2s2_status apply_dispatch(t2s2_op op, Ctx& cx, const DevTT& x, DevTT& y, double c_mass,
                           double c_op, t2s2_precision prec) {
  (void)prec;
  return apply_op(op, cx, x, y, c_mass, c_op, false);
}
}  // namespace t2s2

extern "C" {
t2s2_status t2s2_solve(t2s2_op op, const t2s2_tt* b, t2s2_tt* x, double c_mass, double c_op,
                       double tol, int rmax, int max_sweeps, t2s2_precision prec, void* stream,
                       t2s2_solve_info* info) {
  (void)op; (void)b; (void)x; (void)c_mass; (void)c_op; (void)tol; (void)rmax; (void)max_sweeps;
  (void)prec; (void)stream; (void)info;
  return T2S2_ENOTIMPL;
}
t2s2_status t2s2_cn_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info) {
  (void)op; (void)u; (void)dt; (void)tol; (void)rmax; (void)prec; (void)stream; (void)info;
  return T2S2_ENOTIMPL;
}
t2s2_status t2s2_be_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info) {
  (void)op; (void)u; (void)dt; (void)tol; (void)rmax; (void)prec; (void)stream; (void)info;
  return T2S2_ENOTIMPL;
}
}
