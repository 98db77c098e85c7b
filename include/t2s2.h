/*
 * t2s2.h - C ABI of the GB300 (sm_103a) T^2S^2 hot path.
 *
 * T^2S^2 (tensor-train superconsistent spectral collocation, arXiv 2506.04732)
 * solves the convection-diffusion problem of the paper's eq. pblm:time:A-C,
 *
 *     du/dt - eps Laplace(u) + beta . grad(u) = b  on [-1,1]^d,  u = g on the boundary,
 *
 * with a Lagrange basis on the n Gauss-Lobatto-Legendre (GLL) points of each
 * dimension (Overview (i)), collocation on per-dimension superconsistent
 * points (Overview (ii), Fig. 1, Fig. 3) and tensor-train (TT) storage of all
 * grid functions and of the operator (Overview (iii), Methods).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - n[k] is the number of GLL nodes of dimension k (polynomial degree n[k]-1,
 *   3 <= n[k] <= T2S2_MAX_N).  With zero Dirichlet data the unknowns are the
 *   m[k] = n[k]-2 interior nodes, so every TT handled here has mode sizes m[k].
 * - A TT is d cores; core k is a row-major array [r[k]][m[k]][r[k+1]] of
 *   doubles (the paper's G_k(alpha, i, beta), eq. TT-format:elementwise), with
 *   r[0] = r[d] = 1.  A TT with `loc == T2S2_DEVICE` holds device pointers of
 *   the current CUDA device; `loc == T2S2_HOST` holds host pointers (the
 *   library stages them through device memory; pinned memory is fastest).
 * - The caller owns every TT buffer.  `cap[k]` is the capacity of core k in
 *   doubles.  Entry points that write a TT set its ranks `r[]`; if a core
 *   would exceed its capacity they fail with T2S2_ENOMEM and leave the
 *   output unspecified.  Ranks are bounded by `rmax` where one is taken.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry points
 *   that return host scalars (norms, residuals, ranks) synchronise with it.
 * - Every entry point returns a status; nothing aborts the process.
 * - An operator handle owns its device matrices and its workspace; calls that
 *   share one handle must not run concurrently (they share the workspace).
 * - Kernels of one call are queued with programmatic dependent launch: a
 *   kernel may become resident while its predecessor in the stream runs, but
 *   touches memory only after that predecessor has completed, so results
 *   equal those of plain stream order.  Environment variable T2S2_PDL=0
 *   launches them plainly.
 */
#ifndef T2S2_H
#define T2S2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define T2S2_MAX_D 16
#define T2S2_MAX_N 128
/* Rank of the enrichment directions the alternating solver adds per core and
 * sweep (environment variable T2S2_KICK overrides it, 1 .. 16): a solution
 * can carry ranks up to rmax + T2S2_RANK_KICK. */
#define T2S2_RANK_KICK 8

typedef enum {
  T2S2_OK = 0,
  T2S2_EINVAL = 1,     /* bad argument (sizes, NULL pointers, tolerances) */
  T2S2_ENOMEM = 2,     /* device allocation failed, or a TT core exceeds its capacity */
  T2S2_ECUDA = 3,      /* a CUDA call or kernel launch failed */
  T2S2_ENOCONV = 4,    /* the solver hit its sweep cap; best iterate and residual written */
  T2S2_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  T2S2_ENOTIMPL = 6,   /* feature not provided */
  T2S2_ENODEV = 7      /* no usable sm_103 device */
} t2s2_status;

/* Arithmetic of the heavy kernels.  T2S2_FP64: everything in binary64.
 * T2S2_FP32_REFINE: inner alternating solve in binary32 (SIMT) wrapped in an
 * FP64 residual / iterative-refinement loop; QR/SVD of rounding, the residual
 * norm and the 1D matrices stay FP64.  T2S2_TF32_REFINE / T2S2_BF16_REFINE:
 * as FP32_REFINE with the core contractions on tcgen05 tensor cores. */
typedef enum {
  T2S2_FP64 = 0,
  T2S2_FP32_REFINE = 1,
  T2S2_TF32_REFINE = 2,
  T2S2_BF16_REFINE = 3
} t2s2_precision;

typedef enum { T2S2_DEVICE = 0, T2S2_HOST = 1 } t2s2_location;

/* The problem of eq. pblm:time:A with rho = 0: d, GLL nodes per dimension,
 * convection field beta (d entries), diffusion eps > 0.  plain_sc = 1
 * collocates at the GLL points themselves (the paper's Plain-SC baseline,
 * Overview (i)); 0 uses the superconsistent points. */
typedef struct {
  int d;
  const int* n;
  const double* beta;
  double eps;
  int plain_sc;
} t2s2_problem;

typedef struct t2s2_op_s* t2s2_op;

/* A coefficient function of one coordinate: value at x of dimension k's
 * function; ctx is passed through. */
typedef double (*t2s2_coef_fn)(int k, double x, void* ctx);

/* Variable coefficients of eq. pblm:time:A in the form the paper's
 * six-dimensional test uses: beta_k(x_k) per dimension, and a reaction
 * rho(x) = rho0 + sum_k rho_k(x_k) + prod_k pi_k(x_k).  base.beta[k] is the
 * reference speed of dimension k that picks its superconsistent points (a
 * reading: the paper does not say which speed picks them with a variable
 * beta).  beta_fn NULL: constant base.beta[k]; rho_fn NULL: no sum term;
 * prod_fn NULL: no product term. */
typedef struct {
  t2s2_problem base;
  t2s2_coef_fn beta_fn;
  t2s2_coef_fn rho_fn;
  double rho0;
  void* ctx;
  t2s2_coef_fn prod_fn;
} t2s2_problem_var;

typedef struct {
  int d;
  const int* m;        /* mode sizes m[k] = n[k] - 2 (d entries) */
  int* r;              /* ranks r[0..d], r[0] = r[d] = 1; read on input, written on output */
  double** cores;      /* d core pointers, core k: [r[k]][m[k]][r[k+1]] row-major */
  const size_t* cap;   /* d capacities in doubles */
  int loc;             /* t2s2_location */
} t2s2_tt;

typedef struct {
  double residual;     /* achieved ||b - A x||_F / ||b||_F on the collocation system */
  int sweeps;          /* alternating sweeps (the paper's AMEn "swaps") performed */
  int max_rank;        /* largest TT rank of the returned solution */
  int refinements;     /* outer FP64 refinement steps (mixed precision only) */
  long long local_iters; /* total Krylov iterations of the local solves */
} t2s2_solve_info;

/* Human-readable name of a status code; never NULL. */
const char* t2s2_strerror(t2s2_status s);

/* Number of usable devices (compute capability 10.3) or a negative status. */
int t2s2_device_count(void);

/*
 * Build the d-dimensional collocation operator (Overview (ii)-(iii)).
 * Per dimension, on the host in FP64: GLL nodes, superconsistent collocation
 * points eta (roots in (-1,1) of eps P_N' - beta_k P_N, dropping the root
 * nearest the outflow end when N of them fall inside, N = n-1; a reading of
 * Overview (ii), which does not print the rule), Lagrange matrices Rt = l_i(eta_j),
 * D, D2 on the interior nodes, Lt = beta_k D - eps D2, the interpolation
 * inverse and B_k = Rt^{-1} Lt.  The collocation operator is the rank-2
 * TT-matrix (eq. tt-matrix-format)
 *     A = sum_k Rt_1 x ... x Lt_k x ... x Rt_d,
 * and the collocated time derivative has mass matrix M = Rt_1 x ... x Rt_d.
 * Uploads the matrices to the current device and allocates the workspace.
 * Errors: T2S2_EINVAL for d outside [1, T2S2_MAX_D], n outside [3, T2S2_MAX_N],
 * eps <= 0, NULL pointers; T2S2_ENOMEM / T2S2_ECUDA for device failures.
 */
t2s2_status t2s2_build_operator(const t2s2_problem* prob, void* stream, t2s2_op* out);

/*
 * t2s2_build_operator with variable coefficients (t2s2_problem_var): at the
 * collocation point eta_j of dimension k the rows of the 1D derivative are
 * scaled by beta_k(eta_j) and rho_k(eta_j) Rt_k is added (rho0 Rt in the
 * first dimension), Lt_k = diag(beta_k(eta)) D - eps D2 + diag(rho_k(eta))
 * Rt_k: the same rank-2 TT-matrix, so every entry point that takes an
 * operator works unchanged.  A product reaction prod_k pi_k(x_k) adds the
 * Kronecker product (x)_k diag(pi_k(eta)) Rt_k, a rank-3 TT-matrix in all:
 * then t2s2_apply returns ranks 3 r_x (FP64 only), t2s2_residual includes
 * the term, and t2s2_solve (FP64 only; other precisions return
 * T2S2_ENOTIMPL) lags the reaction: each outer step solves, with the
 * alternating solver and from the current x, (c_mass M + c_op A + c_op
 * rho_bar M) x+ = b - c_op (P - rho_bar M) x (rho_bar: the product of the
 * factors' means over the collocation points, the part of the product term
 * the solver sees), until the residual of the full operator is at most tol;
 * the steps contract by ||(c_mass M + c_op (A + rho_bar M))^-1 c_op
 * (P - rho_bar M)||.  info->refinements counts the outer steps; the
 * residual is |b - A_full x| / |b| with its inner products in double-double.
 * With a product reaction t2s2_solve wants 2 (rmax + 8) <= 96 (T2S2_EINVAL
 * otherwise).
 * t2s2_cn_step and t2s2_be_step return T2S2_ENOTIMPL for such an operator.
 * The functions are called on the host during the build, n[k] - 2 times per
 * dimension.  Errors as t2s2_build_operator, and T2S2_EINVAL if a
 * coefficient value is not finite.
 */
t2s2_status t2s2_build_operator_var(const t2s2_problem_var* prob, void* stream, t2s2_op* out);

/*
 * Operator of the unified space-time form (Methods overview; Results,
 * "Global Accuracy"): time is one more collocated dimension, placed first,
 * with the time interval [0, t_len] mapped onto [-1, 1].  Dimension 0 has n_t
 * GLL nodes, n_t - 1 unknowns (every node but s = -1, which carries the
 * initial condition) and collocation at the n_t - 1 Gauss points (see
 * t2s2_dim_matrices, T2S2_DIM_TIME); its Lt is (2 / t_len) D.  Dimensions
 * 1..d are those of t2s2_build_operator(space).  The operator is the rank-2
 * TT-matrix Lt_t x M_x + Rt_t x A_x over d + 1 dimensions; solve it with
 * c_mass = 0, c_op = 1 and a right-hand side that carries the lifted initial
 * condition.  Errors as t2s2_build_operator, and T2S2_EINVAL for n_t outside
 * [3, T2S2_MAX_N], t_len <= 0 or space->d + 1 > T2S2_MAX_D.
 */
t2s2_status t2s2_build_spacetime_operator(const t2s2_problem* space, int n_t, double t_len, void* stream,
                                          t2s2_op* out);

/*
 * Right-hand side of a space-time solve with the initial condition lifted:
 *     out = round(b - L0 x (M_x u0) - R0 x (A_x u0), tol, rmax),
 * where b is the source on the space-time collocation grid (d + 1 cores,
 * time first), u0 the initial condition on the spatial interior GLL grid (d
 * cores), M_x and A_x the spatial mass matrix and operator, and L0, R0 the
 * columns of the time matrices at the initial node s = -1.  op must come from
 * t2s2_build_spacetime_operator.  Errors: T2S2_EINVAL for another operator or
 * mismatched shapes; T2S2_ENOMEM if out is too small.
 */
t2s2_status t2s2_spacetime_rhs(t2s2_op op, const t2s2_tt* b, const t2s2_tt* u0, t2s2_tt* out, double tol,
                               int rmax, void* stream);

/*
 * Non-zero Dirichlet data (eq. pblm:time:B, u = g on the boundary) by TT
 * lifting.  g is a TT on the FULL GLL grid of a spatial operator: mode sizes
 * n[k] (not n[k] - 2), cores [r[k]][n[k]][r[k+1]]; only its values at
 * boundary nodes matter (any extension inside gives the same solution).
 * With the full (n-2) x n 1D matrices Rf, Lf (every GLL node a column),
 *     out = round(b - (c_mass M_full + c_op A_full) g, tol, rmax),
 * the source of the zero-data system for the correction w = u - g:
 * (c_mass M + c_op A) w = out, after which u = w + g on the interior nodes.
 * b is the source on the collocation grid as for t2s2_solve; out has the
 * interior mode sizes.  Errors: T2S2_EINVAL for a g off the full grid, a
 * space-time operator or non-finite coefficients; T2S2_ENOMEM if out is too
 * small.
 */
t2s2_status t2s2_dirichlet_rhs(t2s2_op op, const t2s2_tt* b, const t2s2_tt* g, double c_mass, double c_op,
                               t2s2_tt* out, double tol, int rmax, void* stream);

/*
 * t2s2_solve with Dirichlet data g (a full-grid TT as in t2s2_dirichlet_rhs;
 * NULL means zero data and gives exactly t2s2_solve).  The lifted source is
 * rounded at tol / 100, the correction w solved from the initial guess in x
 * (any interior-grid TT, e.g. all ones), and x receives u = w + g on the
 * interior nodes as the exact TT sum, not recompressed (ranks of w plus those
 * of g, so x needs room for ranks up to rmax + T2S2_RANK_KICK + max rank of
 * g; recompressing it would lose the small directions of w next to g and the
 * operator would amplify that loss).
 * info->residual is the relative residual of the solved system,
 * ||b_g - (c_mass M + c_op A) w|| / ||b_g||, b_g the lifted source.
 */
t2s2_status t2s2_solve_dirichlet(t2s2_op op, const t2s2_tt* b, const t2s2_tt* g, t2s2_tt* x, double c_mass,
                                 double c_op, double tol, int rmax, int max_sweeps, t2s2_precision prec,
                                 void* stream, t2s2_solve_info* info);

/* Free an operator and its workspace.  NULL is accepted. */
t2s2_status t2s2_op_destroy(t2s2_op op);

/* Kinds of a dimension for t2s2_dim_matrices. */
#define T2S2_DIM_SPACE 0       /* both ends Dirichlet, superconsistent points */
#define T2S2_DIM_SPACE_PLAIN 1 /* both ends Dirichlet, interior GLL points (Plain-SC) */
#define T2S2_DIM_TIME 2        /* time of the space-time form: value given at s = -1 only */

/*
 * One dimension's 1D collocation matrices, computed on the host in FP64 with
 * no device involved (the per-dimension part of t2s2_build_operator).
 * n GLL nodes x_0 = -1 < ... < x_N = 1 (N = n-1, 3 <= n <= T2S2_MAX_N):
 *   space kinds: m = n-2 unknowns x_1..x_{N-1}; collocation points as in
 *                t2s2_build_operator (superconsistent, or interior GLL for
 *                T2S2_DIM_SPACE_PLAIN); boundary columns x_0 and x_N (nb = 2);
 *   T2S2_DIM_TIME: the unified space-time formulation (time mapped onto
 *                [-1, 1], the initial condition a boundary condition at
 *                s = -1, none at s = 1): m = n-1 unknowns x_1..x_N,
 *                collocation at the N zeros of P_N (the eps -> 0
 *                superconsistent points of transport with only the inflow
 *                end constrained; a reading, the paper prints no time
 *                nodes); boundary column x_0 (nb = 1).  Pass beta = 2/T for
 *                a time interval of length T and eps = 0.
 * Outputs (host arrays; any may be NULL): x (n), eta (m collocation
 * points), Rt and Lt (m x m, row-major, row = collocation point, column =
 * unknown node), Rb and Lb (m x nb, the boundary columns, for lifting
 * boundary or initial data), with R = l_i(eta_j) and L = beta l_i'(eta_j) -
 * eps l_i''(eta_j).
 * Errors: T2S2_EINVAL for n outside [3, T2S2_MAX_N], an unknown kind,
 * non-finite eps or beta, eps <= 0 on a space kind (as t2s2_build_operator)
 * or eps < 0 on the time kind.
 */
t2s2_status t2s2_dim_matrices(int n, double eps, double beta, int kind, double* x, double* eta, double* Rt,
                              double* Lt, double* Rb, double* Lb);

/* Copy dimension k's GLL nodes x (n values) and collocation points eta
 * (m values: n-2, or n-1 for the time dimension of a space-time operator)
 * into host arrays; either pointer may be NULL. */
t2s2_status t2s2_op_nodes(t2s2_op op, int k, double* x, double* eta);

/* Copy dimension k's matrices Rt and Lt (m^2 doubles each, m as above,
 * row-major, row = collocation point, column = unknown GLL node) to host
 * arrays; either pointer may be NULL. */
t2s2_status t2s2_op_matrices(t2s2_op op, int k, double* Rt, double* Lt);

/*
 * TT-matrix-by-TT product y = (c_mass M + c_op A) x (Methods: operations raise
 * TT ranks; this one doubles them).  Output ranks: r_y[k] = 2 r_x[k] for
 * 0 < k < d.  Core k of y is built from Rt_k X_k and Lt_k X_k (the mode-k
 * contractions) in the block pattern of the rank-2 TT-matrix:
 *     first [G_1 X, Rt_1 X], middle [[Rt X, 0], [G_k X, Rt X]], last [Rt X; G_d X],
 * G_k = c_op Lt_k (+ c_mass Rt_1 for k = 1).  x and y must not alias.
 * prec selects the contraction arithmetic (results always stored as FP64).
 */
t2s2_status t2s2_apply(t2s2_op op, const t2s2_tt* x, t2s2_tt* y, double c_mass,
                       double c_op, t2s2_precision prec, void* stream);

/*
 * Grouped apply: y_i = (c_mass M_i + c_op A_i) x_i for `count` independent
 * instances (each its own operator; uneven n and ranks allowed), every core
 * of every instance in ONE persistent launch (tensor cores for TF32 / BF16
 * when every m <= 64, else the FP64 kernel).  x and y must be device TTs;
 * y ranks are written as in t2s2_apply.  The launch shape (CTAs per SM) is
 * picked by timing the candidates on the first call for each shape class
 * (see t2s2_autotune_report).  Returns after the work is done.
 * Errors: as t2s2_apply for any instance; T2S2_ETIMEOUT if a tensor-core
 * wait gave up.  The paper applies one operator at a time.
 */
t2s2_status t2s2_apply_batched(const t2s2_op* ops, const t2s2_tt* x, t2s2_tt* y, int count,
                               double c_mass, double c_op, t2s2_precision prec, void* stream);

/* Text table of the launch shapes the grouped apply has tuned so far (one
 * line per shape class with each candidate's time); copies at most len-1
 * characters into buf (NUL-terminated, buf may be NULL) and returns the full
 * length. */
int t2s2_autotune_report(char* buf, int len);

/*
 * TT rounding rndg (Methods, "Tensor-train (TT) decomposition"): in place,
 * right-to-left orthogonalisation, then left-to-right truncated SVDs with
 * per-unfolding threshold tol ||x||_F / sqrt(d-1), then the cap rmax
 * (rmax <= 0: no cap).  Guarantees ||x - rndg(x)||_F <= tol ||x||_F when the
 * cap does not bind.  All arithmetic FP64.  Uses `op` for its workspace.
 */
t2s2_status t2s2_round(t2s2_op op, t2s2_tt* x, double tol, int rmax, void* stream);

/* The values of x along mode `mode` with the other indices fixed (eq.
 * TT-format:elementwise, the product of the core slices): out[t] =
 * x(idx[0], .., t, .., idx[d-1]) for t < m[mode]; idx has d entries (the one
 * at `mode` is ignored); out is a host array of m[mode] doubles.  Used to read
 * a solution along a grid line (the mid-axis lines of the stability map).
 * Synchronises.  Errors: T2S2_EINVAL for a mode or index out of range or
 * ranks above 8192. */
t2s2_status t2s2_tt_fibre(t2s2_op op, const t2s2_tt* x, int mode, const int* idx, double* out, void* stream);

/* ||x||_F (accurate: orthogonalise and take the norm of the first core). */
t2s2_status t2s2_norm(t2s2_op op, const t2s2_tt* x, double* out, void* stream);

/*
 * ||x||_F exactly as t2s2_norm computes it, but without allocating anything.
 * The paper has no counterpart; this entry point exists for callers that may
 * not allocate device memory at the time they need the norm: real-time or
 * embedded loops whose memory is fixed at start-up (a cudaMalloc there can
 * stall or fail), or hosts whose framework allocator already owns the device
 * memory.  It takes no operator handle (no workspace).  Every temporary
 * lives in one 32 MiB array that the library reserves as a static device
 * variable on each GPU that loads it, kept until the process exits.  x must
 * be device-resident (loc == T2S2_DEVICE) with ranks <= 96.  A train whose
 * temporaries would exceed the 32 MiB array is rejected with T2S2_ENOMEM
 * before any work is queued; if an error occurs after work was queued, the
 * call waits for that work before it returns.  The first call on a device
 * looks up that device's array address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the one array, so
 * calls whose GPU work overlaps race on it: serialise them.  The call
 * synchronises with `stream` and reads the result back into host memory
 * before it returns.
 */
t2s2_status t2s2_norm_noalloc(const t2s2_tt* x, double* out, void* stream);

/* ||x - y||_F for two TTs on the same grid, accurate to rounding level even
 * when x and y agree to many digits: the difference is formed as a TT
 * (ranks r_x + r_y), right-orthogonalised, and the norm of its first core
 * taken -- never sqrt(<x,x> - 2<x,y> + <y,y>), which cancels.  FP64.
 * Errors: T2S2_EINVAL for mismatched shapes. */
t2s2_status t2s2_diff_norm(t2s2_op op, const t2s2_tt* x, const t2s2_tt* y, double* out, void* stream);

/* ||b - (c_mass M + c_op A) x||_F / ||b||_F in FP64, accurate even where A x
 * agrees with b to many digits: z = b - A x is formed as a TT and <z, z> is
 * accumulated in double-double (error-free products and sums), ~1e-4 relative
 * at a residual of 1e-12; a result below 1e-13 is recomputed as the norm of the
 * right-orthogonalised z. */
t2s2_status t2s2_residual(t2s2_op op, const t2s2_tt* b, const t2s2_tt* x, double c_mass,
                          double c_op, double* out, void* stream);

/*
 * Solve (c_mass M + c_op A) x = b in TT format with the alternating solver
 * the paper uses (AMEn, Results "Superconsistent Stabilization", Fig. 6):
 * sweeps over the cores with local solves, local SVD truncation at
 * tol/sqrt(d), residual-based rank enrichment, until the true relative
 * residual ||b - (c_mass M + c_op A) x||_F / ||b||_F <= tol or max_sweeps.
 * b is the right-hand side sampled on the collocation grid; x holds the
 * initial guess on input and the solution on output (ranks <= rmax + T2S2_RANK_KICK).
 * Returns T2S2_ENOCONV (with x and info filled) if the sweep cap is hit, or
 * earlier once some TT rank of x sits at rmax + T2S2_RANK_KICK and the
 * residual has not halved over 8 sweeps (the rank cap, not the sweep count,
 * then limits the solution; environment variable T2S2_STALL sets the number
 * of sweeps, 0 turns this stop off).
 * The plain solve is c_mass = 0, c_op = 1.
 */
t2s2_status t2s2_solve(t2s2_op op, const t2s2_tt* b, t2s2_tt* x, double c_mass, double c_op,
                       double tol, int rmax, int max_sweeps, t2s2_precision prec,
                       void* stream, t2s2_solve_info* info);

/*
 * Batched form of t2s2_solve (c_mass = 0, c_op = 1): `count` independent
 * instances, instance i with operator ops[i] (distinct handles: each owns its
 * workspace), right-hand side b[i] and initial guess / solution x[i].
 * Instances run concurrently on `workers` host threads (<= 0: 8), each with
 * its own CUDA stream; every instance's cooperative local solves use at most
 * 152 / workers CTAs so that the workers share the GPU.  Per-instance
 * statuses go to statuses[i] and, if infos != NULL, details to infos[i].
 * Returns the first hard error, else T2S2_ENOCONV if any instance hit its
 * sweep cap, else T2S2_OK.  Errors: T2S2_EINVAL for NULL arrays or a repeated
 * operator handle.
 */
t2s2_status t2s2_solve_batched(const t2s2_op* ops, const t2s2_tt* b, t2s2_tt* x, int count, double tol,
                               int rmax, int max_sweeps, t2s2_precision prec, int workers,
                               t2s2_solve_info* infos, t2s2_status* statuses);

/*
 * One Crank-Nicolson step (eq. ttss-Crank-Nicolson) with the collocated time
 * derivative (mass matrix M):  rhs = rndg((M - dt/2 A) u), then solve
 * (M + dt/2 A) u+ = rhs from the initial guess u; u is overwritten by u+.
 */
t2s2_status t2s2_cn_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info);

/* One backward-Euler step (eq. ttss-backward-Euler): (M + dt A) u+ = M u. */
t2s2_status t2s2_be_step(t2s2_op op, t2s2_tt* u, double dt, double tol, int rmax,
                         t2s2_precision prec, void* stream, t2s2_solve_info* info);

/*
 * Strided-batched GEMM of the solver's core contractions, exported so that
 * those kernels can be checked and timed on their own (the paper has no such
 * call).  For b = 0 .. batch-1, with row-major FP64 device matrices,
 *     C_b = alpha op(A_b) op(B_b) + beta C_b,   op(X) = X (t = 0) or X^T (t = 1),
 * op(A_b) M x K at A + b sA (leading dimension lda), op(B_b) K x N at
 * B + b sB (ldb), C_b M x N at C + b sC (ldc).  prec T2S2_FP64 or
 * T2S2_FP32_REFINE: FP64 SIMT kernel; T2S2_TF32_REFINE / T2S2_BF16_REFINE:
 * tcgen05 kernel with operands rounded to TF32 / BF16 and FP32 accumulation.
 * Split-K workspace comes from the operator's arena.  Asynchronous on
 * `stream` except for the tensor-core status check, which synchronises it.
 * Errors: T2S2_EINVAL for negative sizes, null pointers or leading
 * dimensions shorter than a stored row; T2S2_ETIMEOUT if a device wait gave up.
 */
t2s2_status t2s2_gemm(t2s2_op op, int M, int N, int K, int tA, int tB, double alpha, const double* A,
                      long lda, long sA, const double* B, long ldb, long sB, double beta, double* C,
                      long ldc, long sC, int batch, t2s2_precision prec, void* stream);

/* ---- learned warm start -------------------------------------------------
 * A small network maps a problem's parameters p to the TT cores of an
 * initial guess X(p) for t2s2_solve (the paper's solver takes any initial
 * guess; the tolerance, and so the answer, does not depend on it).
 *     h1 = relu(W1 p + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
 * y = the cores of X(p): (1 x m_1 x r), (r x m_k x r) ..., (r x m_d x 1),
 * row-major, concatenated.  Training minimises the mean over a batch of
 * ||X(p) - U||^2 / ||U||^2 (U: a solution the solver produced), a loss that
 * does not depend on the TT gauge, with Adam (beta1 0.9, beta2 0.999, 1e-8).
 * The layer products run on tcgen05 tensor cores with BF16 operands and FP32
 * accumulation; parameters, gradients and Adam moments are FP32.  Parameter
 * order everywhere: W1 (hidden x in), b1, W2 (hidden x hidden), b2,
 * W3 (out x hidden), b3, each row-major.  The paper has no such network.
 */
typedef struct t2s2_mlp_s* t2s2_mlp;

/* Create a network for d >= 2 modes of sizes m[0..d-1] (<= 64), output rank
 * r (<= 16) and targets of rank <= ru (<= 32); He-normal weights from `seed`,
 * zero biases.  Errors: T2S2_EINVAL for sizes out of range, T2S2_ENOMEM. */
t2s2_status t2s2_mlp_create(int in_dim, int hidden, int d, const int* m, int r, int ru,
                            unsigned long long seed, t2s2_mlp* out);
t2s2_status t2s2_mlp_destroy(t2s2_mlp net);
/* Number of parameters and the length of y. */
t2s2_status t2s2_mlp_info(t2s2_mlp net, long long* nparams, int* out_dim);
/* Copy parameters and/or the last gradient (nparams floats each; host or
 * device pointers, either may be NULL) out of / into the network. */
t2s2_status t2s2_mlp_get_params(t2s2_mlp net, float* params, float* grads, void* stream);
t2s2_status t2s2_mlp_set_params(t2s2_mlp net, const float* params, void* stream);
/* Store the device TT u (ranks <= ru, mode sizes m) as a training target:
 * slot (device, d * ru * mmax * ru floats) receives its cores zero-padded to
 * ru x mmax x ru, uu (device, 1 float) its squared norm (FP64 TT norm). */
t2s2_status t2s2_mlp_pack_target(t2s2_mlp net, t2s2_op op, const t2s2_tt* u, float* slot, float* uu,
                                 void* stream);
/* Start the network's output at a representative solution u (a device or
 * host TT on the network's grid): the output bias takes the cores of u
 * rounded to the network's rank r (FP64 rounding with no tolerance, then
 * stored as FP32, zero-padded to the output's core shapes), the output
 * weights W3 are multiplied by weight_scale, and the log-scale bias is set to
 * zero.  X(p) then starts near u for every p and training learns the
 * deviations.  Uses op's workspace.  Synchronises.  Errors: T2S2_EINVAL for
 * a TT off the network's grid or a non-finite weight_scale. */
t2s2_status t2s2_mlp_init_output(t2s2_mlp net, t2s2_op op, const t2s2_tt* u, float weight_scale, void* stream);
/* Loss and gradient of a batch: P (device, batch x in_dim), targets and uu
 * (device, as packed above).  The gradient stays in the network (see
 * t2s2_mlp_get_params); *loss (may be NULL) receives the mean loss.
 * Synchronises the stream.  T2S2_ETIMEOUT if a tensor-core wait gave up. */
t2s2_status t2s2_mlp_loss_grad(t2s2_mlp net, const float* P, int batch, const float* targets,
                               const float* uu, float* loss, void* stream);
/* Output-scale calibration: evaluates the batch and adds 0.5 log(mean <U,U> /
 * mean <X,X>) to the bias of the log-scale output, so that X(p) starts at the
 * targets' size (normalised cores multiply to a TT whose norm shrinks with d
 * and r).  *shift (may be NULL) receives the change.  Synchronises. */
t2s2_status t2s2_mlp_calibrate_scale(t2s2_mlp net, const float* P, int batch, const float* targets,
                                     const float* uu, float* shift, void* stream);
/* As t2s2_mlp_loss_grad followed by one Adam update with learning rate lr. */
t2s2_status t2s2_mlp_train_step(t2s2_mlp net, const float* P, int batch, const float* targets,
                                const float* uu, float lr, float* loss, void* stream);
/* `steps` training steps over a resident training set of n samples (P: n x
 * in_dim, targets / uu as packed above, all device), minibatches of `batch`
 * consecutive samples cycling through the set, learning rate lr.  With
 * use_graph = 1 the launch sequence of a step is captured once per minibatch
 * as a CUDA graph (the first visit runs eagerly) and replayed afterwards;
 * the step count and learning rate live in device memory so a replay stays
 * valid.  *loss (may be NULL) receives the last step's mean loss.
 * Synchronises the stream at the end. */
t2s2_status t2s2_mlp_train(t2s2_mlp net, const float* P, int n, const float* targets, const float* uu,
                           int batch, int steps, float lr, int use_graph, float* loss, void* stream);
/* Warm start: the cores of X(p) (p: host or device, in_dim floats) as FP64
 * into x (device or host cores with room for them); x->r is set to the
 * network's ranks.  For a device x whose layers fit one CTA's shared memory
 * (in_dim + 2 hidden + outputs <= 24k floats) the prediction is a single
 * launch (layers with BF16 operands and FP32 sums, as the batched layers)
 * queued on `stream` without synchronising; otherwise the batched layers run
 * and the call synchronises. */
t2s2_status t2s2_mlp_predict(t2s2_mlp net, const float* p, t2s2_tt* x, void* stream);

/* The FP64 reciprocal square root and reciprocal that the small
 * factorisations use (binary32 hardware seed refined by two binary64 Newton
 * steps, y <- y (3 - x y^2) / 2 and y <- y (2 - x y); IEEE division and
 * square root for |x| outside (1e-36, 1e36)), applied elementwise to the
 * device array x (n doubles) so that they can be checked against correctly
 * rounded results.  rsqrt_out / rcp_out: device arrays of n doubles, either
 * may be NULL.  Synchronises.  The paper has no such call. */
t2s2_status t2s2_fastmath(const double* x, double* rsqrt_out, double* rcp_out, long n, void* stream);

/* ---- diagnostics ---------------------------------------------------------
 * Kernel families for tracing: 0 GEMM (SIMT contractions), 1 TT apply
 * (FP64), 2 local solve (Krylov team and its eigendecompositions), 3 small
 * factorisations (Cholesky, Jacobi SVD), 4 elementwise, 5 TT apply on tensor
 * cores (BF16/TF32), 6 GEMM on tensor cores (BF16/TF32), 7 warm-start network
 * (forward, backward, Adam), 8 fused CholeskyQR, 9 rank-1-right local solves
 * (Sylvester solver), 10 TT inner products (binary64 and double-double).
 */

/* Number of CUDA kernels this library has launched in this process. */
long long t2s2_kernel_launches(void);

/* Clear the per-family counters and turn event timing on (1) or off (0).
 * While on, every launch is bracketed by two CUDA events on its stream. */
t2s2_status t2s2_trace(int enable);

/* Average time (ms) of an empty kernel launched as the library launches its
 * kernels and bracketed by two CUDA events, over n launches on `stream`: the
 * share of a traced launch's event time that is not the kernel's work.
 * Synchronises. */
t2s2_status t2s2_trace_overhead(int n, void* stream, double* ms);

/* Totals since the last t2s2_trace call for one family: launches, summed
 * event time in ms, algorithmic FLOPs and algorithmic bytes (operands read
 * once, results written once).  Synchronises on the recorded events.
 * Errors: T2S2_EINVAL for an unknown family. */
t2s2_status t2s2_trace_read(int family, long long* launches, double* ms, double* flops,
                            double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* T2S2_H */
