/*
 * lqcd.h -- C ABI of the GB300 Wilson-clover / overlap fermion library.
 *
 * The operators are the ones whose GPU kernels the paper ports and measures
 * (Bi et al., "Lattice QCD package GWU-code and QUDA with HIP", Lattice
 * 2019): the Wilson and clover Dirac operators (Table 1, QUDA_DIRAC_WILSON
 * and QUDA_DIRAC_CLOVER), the D-slash kernel with SU(3) links compressed to
 * 12 reals (Table 2 and its caption), the Krylov inverter built on them, and
 * the overlap inverter of GWU-code (abstract, Sec. 3, Sec. 4).  The paper
 * prints no formula; each call states the standard definition it follows.
 *
 * Conventions shared by every call
 *   lattice   dims[4] = (L0, L1, L2, L3) = (x, y, z, t), every Lmu even
 *             and >= 2; lexicographic site s = x0 + L0 (x1 + L1 (x2 + L2 x3));
 *             parity (x0 + x1 + x2 + x3) mod 2, even = 0.  Periodic in x, y,
 *             z; in t periodic or antiperiodic (t_antiperiodic = 1: a hop
 *             across the t boundary carries a factor -1).
 *   gamma     DeGrand-Rossi chiral basis, gamma5 = diag(1, 1, -1, -1).
 *   hopping   (D psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
 *                                + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu).
 *   clover    A(x) = 1 - c_sw kappa sum_{mu<nu} sigma_munu F_munu(x),
 *             F_munu = [(Q - Q^dag)/(8i)] minus trace/3, Q the four
 *             plaquette leaves at x, sigma_munu = (i/2)[g_mu, g_nu].
 *   operator  M = A - kappa D;  Schur complement on odd sites
 *             Mhat = A_oo - kappa^2 D_oe A_ee^-1 D_eo,  Mhat^dag = g5 Mhat g5.
 *   canonical FP64 arrays, complex as (re, im) pairs, x fastest:
 *             links  [t][z][y][x][mu 4][row 3][col 3]       (36 complex/site)
 *             spinor [rhs][t][z][y][x][spin 4][colour 3]    (12 complex/site)
 *
 * Memory and ownership
 *   Pointers marked "host or device" are device pointers when on_device = 1
 *   (for example torch.Tensor.data_ptr() of a CUDA tensor) and host pointers
 *   otherwise; the library copies what it needs during the call, on the
 *   context's stream, and never keeps or frees a caller's pointer.  The
 *   library owns everything it allocates; lqcd_destroy releases it.
 *   Calls on one context are not thread-safe; different contexts are
 *   independent.  Every call is asynchronous on the context's stream unless
 *   it returns data to host memory or says otherwise.
 *
 * Errors
 *   Every call returns an lqcd_status; 0 is success.  Arguments are checked
 *   before any launch.  lqcd_last_error() returns a thread-local message for
 *   the most recent failure.  The library never calls exit() or abort() and
 *   never traps the GPU.
 */
#ifndef LQCD_H
#define LQCD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQCD_OK = 0,
  LQCD_ERR_ARG = -1,      /* invalid argument (NULL pointer, bad size, bad enum) */
  LQCD_ERR_CUDA = -2,     /* a CUDA runtime call or kernel launch failed */
  LQCD_ERR_OOM = -3,      /* device or pinned host allocation failed */
  LQCD_ERR_NOCONV = -4,   /* solver stopped without reaching the tolerance */
  LQCD_ERR_TIMEOUT = -5,  /* a bounded device-side wait ran out */
  LQCD_ERR_STATE = -6,    /* call needs state not set yet (gauge, kappa) */
  LQCD_ERR_NOT_SU3 = -7,  /* a loaded link is not unitary with det 1 */
  LQCD_ERR_SINGULAR = -8  /* a clover block has a zero pivot */
} lqcd_status;

/* Storage precision of a field.  Arithmetic is FP64 for LQCD_F64 and FP32
 * for F32, F16 and BF16; FP16 and BF16 spinors and clover terms carry one
 * FP32 scale per site, links are stored unscaled.  LQCD_DF64 ("double-float",
 * no counterpart in the paper) stores every real as two FP32 numbers hi + lo
 * (eight bytes, the FP64 layout) and computes on the FP32 pipes with
 * error-free transformations: a 48-bit significand (relative rounding about
 * 2^-47 per operation against FP64's 2^-53), the FP32 exponent range (values
 * below ~1e-30 in magnitude lose low-order bits, above ~3e38 overflow), and
 * several times the throughput of FP64 on a GPU whose FP64 rate is 1/64 of
 * its FP32 rate. */
typedef enum { LQCD_F64 = 0, LQCD_F32 = 1, LQCD_F16 = 2, LQCD_BF16 = 3, LQCD_DF64 = 4 } lqcd_prec;

/* Link storage: all 18 reals, or rows 0 and 1 only (12 reals) with row 2
 * rebuilt as conj(row0 x row1) in registers (Table 2's caption), or 8 reals
 * (FP32/FP16 operators, one right-hand side per thread; BF16 would keep the
 * two angles only to ~6e-3 rad and is refused): arg U00,
 * arg U20, U01, U02, U10, the rest rebuilt from unitarity and det U = 1
 * (|U00| and |U20| from the unit row 0 and column 0, U11 and U12 from a 2x2
 * linear system of determinant 1 - |U00|^2, row 2 as the cross product).
 * LQCD_ERR_ARG for the 8-real form on a field with a link of |U00| = 1 (unit
 * links, the free field), where that determinant vanishes. */
typedef enum { LQCD_RECON_18 = 18, LQCD_RECON_12 = 12, LQCD_RECON_8 = 8 } lqcd_recon;

/* Which sites a device-resident field holds. */
typedef enum { LQCD_EVEN = 0, LQCD_ODD = 1, LQCD_FULL = 2 } lqcd_subset;

typedef enum {
  LQCD_OP_M = 0,            /* full lattice: out = M in                               */
  LQCD_OP_MHAT = 1,         /* odd sites:    out_o = Mhat in_o                          */
  LQCD_OP_MHAT_DAG = 2,     /* odd sites:    out_o = Mhat^dag in_o                      */
  LQCD_OP_MHAT_NORMAL = 3,  /* odd sites:    out_o = Mhat^dag Mhat in_o                 */
  LQCD_OP_HOP_EO = 4,       /* even sites:   out_e = D_eo in_o                          */
  LQCD_OP_HOP_OE = 5,       /* odd sites:    out_o = D_oe in_e                          */
  LQCD_OP_HW = 6,           /* full lattice: out = g5 [(4 - rho) in - D in / 2]         */
  LQCD_OP_K2A = 7,          /* even sites:   out_e = A_ee^-1 D_eo in_o (c_sw = 0: D_eo) */
  LQCD_OP_M_DAG = 8,        /* full lattice: out = M^dag in = g5 M g5 in                */
  LQCD_OP_MHAT_SYM = 9,     /* odd sites:    out_o = A_oo^-1 Mhat in_o                  */
                            /*   = in_o - kappa^2 A_oo^-1 D_oe A_ee^-1 D_eo in_o         */
                            /*   (the symmetric Schur complement; c_sw = 0: Mhat)        */
  LQCD_OP_MHAT_SYM_DAG = 10 /* odd sites:    out_o = (A_oo^-1 Mhat)^dag in_o            */
                            /*   = in_o - kappa^2 g5 D_oe A_ee^-1 D_eo g5 A_oo^-1 in_o   */
} lqcd_op;

typedef struct lqcd_ctx lqcd_ctx;     /* one lattice geometry, gauge field and clover term */
typedef struct lqcd_field lqcd_field; /* a device-resident spinor field (one or more RHS) */

/* ---- context ---------------------------------------------------------- */

/* Create a context for one lattice.  dims: four even extents >= 2.
 * cuda_stream: a cudaStream_t to run on, or NULL for the legacy default
 * stream.  Errors: LQCD_ERR_ARG (bad dims, NULL ctx), LQCD_ERR_CUDA. */
lqcd_status lqcd_create(lqcd_ctx **ctx, const int dims[4], int t_antiperiodic, void *cuda_stream);

/* Release the context and everything the library allocated for it.
 * Fields created on it must be destroyed first.  NULL is accepted. */
lqcd_status lqcd_destroy(lqcd_ctx *ctx);

/* Replace the stream the context launches on (NULL: default stream). */
lqcd_status lqcd_set_stream(lqcd_ctx *ctx, void *cuda_stream);

/* Block until all work queued on the context's stream has finished. */
lqcd_status lqcd_synchronize(lqcd_ctx *ctx);

/* Thread-local message describing the last failure on this thread. */
const char *lqcd_last_error(void);

/* ---- gauge field and clover term -------------------------------------- */

/* Load the links U_mu(x) (canonical layout, host or device).  The library
 * keeps an FP64 copy and packs the site-blocked FP64/FP32/FP16/BF16 and
 * 18/12-real forms on first use.  Every link is checked: unitarity
 * max|U U^dag - 1| and |det U - 1| must be below 1e-10, else
 * LQCD_ERR_NOT_SU3 (12-real storage relies on det U = 1).  Loading a new
 * field drops the clover term.  Blocks until the check has finished. */
lqcd_status lqcd_load_gauge(lqcd_ctx *ctx, const double *U, int on_device);

/* Set kappa and c_sw and build the clover term A and A^-1 on the GPU in
 * FP64: clover-leaf field strength, two 6x6 Hermitian blocks per site (the
 * chiral basis makes sigma_munu block diagonal), inverted by an LDL^dag
 * factorisation.  c_sw = 0 selects the plain Wilson operator (A = 1, no
 * clover storage).  Needs a gauge field (else LQCD_ERR_STATE); a zero pivot
 * gives LQCD_ERR_SINGULAR.  Blocks until the build has finished. */
lqcd_status lqcd_clover(lqcd_ctx *ctx, double kappa, double c_sw);

/* Set rho of the overlap kernel H_W = g5 D_W(-rho), D_W(m) = 4 + m - D/2. */
lqcd_status lqcd_set_rho(lqcd_ctx *ctx, double rho);

/* ---- operator application on canonical arrays -------------------------- */

/* out = op(in) for nrhs right-hand sides stored back to back in canonical
 * order (host or device; both nrhs * V * 24 doubles).  The arithmetic runs
 * in `prec` with links in `recon` form: the input is converted to that
 * precision on the GPU, the result converted back to FP64.  Sites outside
 * the op's output subset are set to zero.  Needs the gauge field, and
 * kappa for every op but HOP_EO/HOP_OE/HW (rho for HW).  Host buffers are
 * read and written inside the call, which then blocks; for LQCD_OP_MHAT on
 * host buffers the call is pipelined over chunks of whole time slices (the
 * largest divisor of L3 between 4 and LQCD_HOST_CHUNKS, default 32; copies in
 * and out on two streams of the context while the context's stream computes;
 * the result is bit-identical to the device-buffer path).  Environment
 * LQCD_NO_PIPELINE=1 disables that. */
lqcd_status lqcd_dslash(lqcd_ctx *ctx, double *out, const double *in, int nrhs, lqcd_op op, lqcd_prec prec,
                        lqcd_recon recon, int on_device);

/* ---- device-resident fields -------------------------------------------- */

/* Allocate a spinor field of nrhs right-hand sides on `subset` in storage
 * precision `prec`, zero-filled (asynchronously, on the context's stream). */
lqcd_status lqcd_field_create(lqcd_ctx *ctx, lqcd_prec prec, lqcd_subset subset, int nrhs, lqcd_field **field);
lqcd_status lqcd_field_destroy(lqcd_field *field);

/* Convert canonical FP64 spinors (nrhs back to back, host or device) into
 * the field, taking the sites of the field's subset.  Export converts back
 * and writes only the sites of the field's subset. */
lqcd_status lqcd_field_import(lqcd_ctx *ctx, lqcd_field *field, const double *canon, int on_device);
lqcd_status lqcd_field_export(lqcd_ctx *ctx, const lqcd_field *field, double *canon, int on_device);

/* out = op(in) on device-resident fields of one precision (the arithmetic
 * precision follows the fields).  Subsets must match the op: EVEN/ODD
 * parities for the Schur and hopping ops, FULL for M, M_DAG and HW.  The
 * intermediate of MHAT-type ops lives in context-owned scratch.  Nothing is
 * copied to or from the host and nothing synchronises. */
lqcd_status lqcd_apply(lqcd_ctx *ctx, lqcd_op op, lqcd_recon recon, lqcd_field *out, const lqcd_field *in);

/* The second half of Mhat on its own: out_o = A_oo x_o - kappa^2 D_oe y_e
 * (dagger = 1: A_oo x_o - kappa^2 g5 D_oe y_e, the form used inside
 * Mhat^dag = g5 Mhat g5 once y_e was built from g5 x_o).  Together with
 * LQCD_OP_K2A this is one Mhat application split into its two kernels. */
lqcd_status lqcd_apply_schur(lqcd_ctx *ctx, lqcd_recon recon, int dagger, lqcd_field *out, const lqcd_field *x_odd,
                             const lqcd_field *y_even);

/* Sum over all sites and right-hand sides of |component|^2, reduced in FP64
 * in a fixed order (bitwise reproducible).  Blocks; result in host memory. */
lqcd_status lqcd_field_norm2(lqcd_ctx *ctx, const lqcd_field *field, double *result);

/* ---- solvers ----------------------------------------------------------- */

/* Krylov recursion of lqcd_solve.  CGLS (CG on the normal equations Mhat^dag
 * Mhat) is the paper's; BiCGStab (van der Vorst 1992) works on Mhat itself,
 * with the same plain / mixed-precision-with-reliable-updates structure (no
 * counterpart in the paper's text; QUDA's inverter family, which the paper
 * ports, includes it).  lqcd_solve_batch runs CGLS only. */
typedef enum { LQCD_SOLVER_CGLS = 0, LQCD_SOLVER_BICGSTAB = 1, LQCD_SOLVER_GCR = 2 } lqcd_solver;

/* Even-odd reduced operator the recursion works on.  Both solve the same
 * system M x = b (same x_o):
 *   LQCD_SCHUR_ASYM: Mhat x_o = bhat_o with Mhat = A_oo - kappa^2 D_oe A_ee^-1 D_eo
 *   LQCD_SCHUR_SYM:  A_oo^-1 Mhat x_o = A_oo^-1 bhat_o, i.e.
 *                    (1 - kappa^2 A_oo^-1 D_oe A_ee^-1 D_eo) x_o = A_oo^-1 bhat_o
 * The symmetric form has the better-conditioned operator on rough gauge fields
 * (fewer iterations); its application costs the same bytes as Mhat, its
 * adjoint one more site-local clover pass.  Its iterated residual is
 * A_oo^-1 (bhat - Mhat x), so the solver's targets are divided by a
 * Gershgorin bound of ||A_oo|| taken when the clover term is built: the
 * true residual still meets tol.  With c_sw = 0 the two forms coincide. */
typedef enum { LQCD_SCHUR_ASYM = 0, LQCD_SCHUR_SYM = 1 } lqcd_schur;

typedef struct {
  double tol;          /* target ||b - M x|| / ||b|| on the full lattice, > 0     */
  int max_iter;        /* cap on CG iterations (inner iterations when mixed)       */
  lqcd_prec inner;     /* LQCD_F64 / LQCD_DF64: plain CG in that precision; else  */
                       /* mixed with this storage (F32, F16, BF16)                */
  double delta;        /* reliable-update trigger: inner ||r|| < delta * ||r_0||   */
  int nrhs;            /* right-hand sides stored back to back in x and b          */
  int use_x0;          /* 1: x holds an initial guess on entry                     */
  lqcd_recon recon;    /* link storage of the FP64 operator                        */
  lqcd_recon inner_recon; /* link storage of the inner low-precision operator      */
  int check_every;     /* FP64 CG: iterations between host checks (0: 8); the     */
                       /* mixed solver checks every iteration on the device       */
  lqcd_prec outer;     /* mixed solver: precision of the reliable updates and of  */
                       /* the accumulated solution, LQCD_F64 (0, the default) or  */
                       /* LQCD_DF64; the final residual check is FP64 either way  */
  int solver;          /* lqcd_solver: LQCD_SOLVER_CGLS (0, the default: CG on    */
                       /* the normal equations), LQCD_SOLVER_BICGSTAB or          */
                       /* LQCD_SOLVER_GCR (restarted GCR(m) on the Schur         */
                       /* operator; mixed: each cycle in the inner precision on   */
                       /* the normalised residual, a reliable update after it,    */
                       /* a cycle ending after m steps or a delta drop)           */
  int schur;           /* lqcd_schur: LQCD_SCHUR_ASYM (0, the default) or         */
                       /* LQCD_SCHUR_SYM; any solver, plain, mixed and batched    */
  int gcr_nkrylov;     /* GCR: steps per cycle m, 1..64 (0: 8); 2m fields kept     */
} lqcd_solve_params;

typedef struct {
  int iters;              /* CG iterations done (the largest over right-hand sides) */
  int reliable_updates;   /* FP64 residual recomputations (mixed solver)            */
  int nrhs;
  double true_resid[64];  /* ||b - M x|| / ||b|| per RHS, recomputed in FP64 on GPU */
  double seconds;         /* wall time of the solve                                 */
  double mhat_applies;    /* Mhat (or Mhat^dag) applications, all precisions        */
} lqcd_solve_info;

/* Solve M x = b (canonical arrays, nrhs right-hand sides, host or device)
 * by even-odd preconditioning: bhat_o = b_o + kappa D_oe A_ee^-1 b_e,
 * CG on the normal equations of Mhat x_o = bhat_o (CGLS form, one
 * independent recursion per right-hand side), then
 * x_e = A_ee^-1 (b_e + kappa D_eo x_o).  With params->inner != LQCD_F64 the
 * CG runs with low-precision storage and FP32 arithmetic inside a CUDA graph
 * conditional WHILE loop that a device-side control kernel ends when an update
 * is due, and the solution is accumulated, and the residual recomputed, in
 * FP64 whenever the inner residual fell by `delta` (reliable updates).  Returns LQCD_OK only after
 * the FP64 full-lattice residual of every RHS is <= tol; LQCD_ERR_NOCONV
 * with info filled and x the last iterate otherwise.  Blocks. */
lqcd_status lqcd_solve(lqcd_ctx *ctx, double *x, const double *b, int on_device, const lqcd_solve_params *params,
                       lqcd_solve_info *info);

/* Solve several lattices at once (each its own context: geometry, gauge
 * field, clover term), nrhs right-hand sides each, with the mixed-precision
 * recursion of lqcd_solve (params->inner must not be LQCD_F64).  Every
 * lattice runs on a private stream for the duration of the call; the inner
 * iterations of all unfinished lattices form one CUDA graph with one
 * conditional WHILE node per lattice, whose loop runs on the GPU until that
 * lattice needs an FP64 reliable update; the host performs the updates
 * between launches and rebuilds the graph when a lattice finishes.  x[i], b[i]: canonical
 * arrays of lattice i (host or device, all alike); infos: nctx records or
 * NULL.  The result of each lattice equals lqcd_solve's for the same inputs.
 * Returns the first failure (LQCD_ERR_NOCONV if a lattice did not converge;
 * every lattice's x and info are written regardless).  Blocks. */
lqcd_status lqcd_solve_batch(lqcd_ctx *const *ctxs, int nctx, double *const *x, const double *const *b,
                             int on_device, const lqcd_solve_params *params, lqcd_solve_info *infos);

/* ---- overlap operator ---------------------------------------------------- */

/* The overlap operator of GWU-code's inverter (abstract; Sec. 3; the overlap
 * eigensystem run of Sec. 4), in its standard form
 *   D_ov(m) = (1 - m/(2 rho)) rho (1 + g5 eps(H_W)) + m,   H_W = g5 D_W(-rho),
 *   D_W(m') = 4 + m' - D/2 (plain Wilson kernel, no clover, full lattice),
 * with the sign function eps(H_W) computed as
 *   eps v = sum_i sign(lam_i) v_i <v_i, v> + H_W P(H_W^2) (v - sum_i v_i <v_i, v>)
 * from the n_low eigenpairs (lam_i, v_i) of H_W of smallest |lam| and the
 * Chebyshev interpolant P(y) of 1/sqrt(y) on [a, b], a = lam_{n_low+1}^2
 * (the largest unprojected-range lower bound found), b = (4 - rho + 4)^2. */
typedef struct {
  double rho;        /* kernel mass parameter, 0 < rho < 2 (1.5 in the workloads)        */
  double mass;       /* overlap quark mass m                                             */
  int n_low;         /* low modes of H_W treated exactly, 0..64                          */
  int max_degree;    /* cap on the Chebyshev degree                                      */
  double sign_tol;   /* target sup |x P(x^2) - sign x| on [sqrt a, sqrt b]               */
  double eig_tol;    /* target ||H_W v - lam v|| of every low mode (absolute, |v| = 1)   */
  int max_filter;    /* cap on subspace-iteration sweeps of the low-mode solver          */
  unsigned long long seed; /* seed of the random start block of the low-mode solver     */
  lqcd_prec high;    /* arithmetic of the FP64 parts (the low-mode filter once it leaves   */
                     /* FP32, the FP64 sign function and so D_ov, its CG and the mixed   */
                     /* CG's reliable updates): LQCD_F64 (0, the default) or LQCD_DF64;  */
                     /* fields stay FP64 either way; Gram matrices, rotations and the    */
                     /* sign function's low-mode projection accumulate in double-float  */
                     /* (~2^-44 relative) in both cases                                  */
  int eig_method;    /* low-mode solver on H_W^2: LQCD_EIG_SUBSPACE (0, the default:      */
                     /* block subspace iteration with a Chebyshev filter; max_filter caps */
                     /* its sweeps) or LQCD_EIG_LANCZOS (thick-restart Lanczos, one      */
                     /* vector at a time, double-float basis; max_filter caps its       */
                     /* restarts; 16^3x32: 16 s against 70 s).  Lanczos needs           */
                     /* far fewer H_W applications, but a single Krylov vector can reach */
                     /* a near-degenerate cluster late: on clustered spectra it may stop */
                     /* with converged pairs above a cluster it has not yet found, which */
                     /* the block method (40 random start vectors) guards against        */
} lqcd_overlap_params;

typedef enum { LQCD_EIG_SUBSPACE = 0, LQCD_EIG_LANCZOS = 1 } lqcd_eig_method;

typedef struct {
  int n_low;              /* low modes found                                           */
  double lambda[64];      /* their eigenvalues of H_W, sorted by |lambda|              */
  double resid[64];       /* ||H_W v - lambda v|| of each                              */
  double a, b;            /* interval of the Chebyshev interpolant (in H_W^2)          */
  int degree;             /* its degree                                                */
  double sign_error;      /* its sup error on [sqrt a, sqrt b]                         */
  int sweeps;             /* subspace-iteration sweeps (Lanczos: restart cycles) used  */
  double seconds;         /* wall time of the set-up                                   */
  int degree_inner;       /* degree of the FP32 sign function inside the mixed CG: the */
                          /* smallest reaching max(sign_tol, 1e-6), the FP32 rounding */
                          /* level (reliable updates use the full degree)             */
  double hw_applies;      /* H_W applications (one per vector) of the low-mode solver */
} lqcd_overlap_info;

typedef enum {
  LQCD_OV_APPLY = 0,      /* out = D_ov(m) in                                          */
  LQCD_OV_APPLY_DAG = 1,  /* out = D_ov(m)^dag in                                      */
  LQCD_OV_SIGN = 2,       /* out = eps(H_W) in                                         */
  LQCD_OV_SOLVE = 3,      /* out = D_ov(m)^-1 in by CG on the normal equations         */
  LQCD_OV_SOLVE_DEFLATED = 4  /* the same CG started from the exact part of the solution */
                          /* in the eigensystem of lqcd_overlap_eigen (deflation)      */
} lqcd_overlap_op;

/* Compute the low modes of H_W (block subspace iteration on H_W^2 with
 * Chebyshev filtering, or thick-restart Lanczos on H_W^2, per
 * params->eig_method; then Rayleigh-Ritz in H_W) and the Chebyshev
 * coefficients for the sign function, and keep them in the context.  Needs
 * the gauge field.  Blocks.  The tolerance holds for H_W itself: after the
 * final Rayleigh-Ritz step every returned mode's ||H_W v - lambda v|| is
 * checked against eig_tol, and while one exceeds it the H_W^2 target is
 * tightened and the block iteration continues (after the Lanczos method, on
 * its Ritz vectors padded to a full block).  LQCD_ERR_NOCONV if the modes do
 * not reach eig_tol within max_filter sweeps or restarts (info is filled
 * either way); the context then holds no usable overlap state
 * (lqcd_overlap and lqcd_overlap_lowmodes return LQCD_ERR_STATE until a
 * set-up succeeds).  LQCD_ERR_ARG for a lattice too small for the requested
 * modes. */
lqcd_status lqcd_overlap_setup(lqcd_ctx *ctx, const lqcd_overlap_params *params, lqcd_overlap_info *info);

/* Copy the n_low low-mode vectors (canonical, n_low fields back to back,
 * host or device) out of the context, in the order of info->lambda. */
lqcd_status lqcd_overlap_lowmodes(lqcd_ctx *ctx, double *vecs, int on_device);

/* Apply or invert the overlap operator set up by lqcd_overlap_setup on nrhs
 * canonical full-lattice spinors (host or device), in FP64.  For
 * LQCD_OV_SOLVE, cg->tol is the target ||b - D_ov x|| / ||b|| per right-hand
 * side and cg->max_iter caps the iterations; cg->inner selects the plain
 * FP64 CG (LQCD_F64) or the mixed one with an FP32 inner sign function
 * (LQCD_F32, reliable updates every cg->delta); the other fields of cg
 * (solver, schur, recon, outer, ...) belong to the Wilson-clover solves and
 * are ignored here.  info (may be NULL) receives the iteration count and the
 * final residuals.  Blocks. */
lqcd_status lqcd_overlap(lqcd_ctx *ctx, double *out, const double *in, int nrhs, int on_device, lqcd_overlap_op op,
                         const lqcd_solve_params *cg, lqcd_solve_info *info);

/* ---- the overlap eigensystem (Sec. 4: 200 pairs of the overlap eigensystem
 * of a 24^3 x 64 lattice) and the deflated overlap CG ---------------------
 *
 * D_ov(0) = rho (1 + g5 eps) is normal and g5-Hermitian, so D_ov(0)^dag D_ov(0)
 * commutes with g5 = diag(1, 1, -1, -1) (DeGrand-Rossi) and its eigenvectors
 * can be taken chiral.  On the chirality sector s (P_s = (1 + s g5) / 2) it is
 * H_s = 2 rho^2 P_s (1 + s eps) P_s, one sign-function application per vector.
 * An eigenvalue mu of H_s (0 < mu < 4 rho^2) belongs to the eigenvalue pair
 * lambda = mu / (2 rho) +- i sqrt(mu - mu^2 / (4 rho^2)) of D_ov(0), and its
 * vector chi has a partner eta = P_-s eps chi / |P_-s eps chi| of the other
 * sector with the same mu (chiral zero modes and mu = 4 rho^2 have none). */
#define LQCD_OV_MAX_EV 256

typedef struct {
  int n_ev;                 /* eigenpairs of H_s wanted, 1..LQCD_OV_MAX_EV                   */
  int sector;               /* s = +1 (spins 0, 1) or -1 (spins 2, 3)                        */
  double tol;               /* contract: ||H_s chi - mu chi|| <= tol for every pair (|chi|=1) */
  int basis;                /* Lanczos basis size; 0: min(max(3 n_ev, n_ev + 48), 511)        */
  int max_restarts;         /* cap on Lanczos restart cycles                                 */
  unsigned long long seed;  /* seed of the random start vector                               */
} lqcd_overlap_eigen_params;

typedef struct {
  int n_ev;                         /* pairs kept (= params->n_ev on success)                */
  int n_partners;                   /* of them with a partner in the other sector            */
  double mu[LQCD_OV_MAX_EV];        /* eigenvalues of D_ov(0)^dag D_ov(0), ascending         */
  double resid[LQCD_OV_MAX_EV];     /* ||H_s chi - mu chi||, recomputed after convergence    */
  double lambda_re[LQCD_OV_MAX_EV]; /* the D_ov(0) eigenvalue pair lambda_re +- i lambda_im */
  double lambda_im[LQCD_OV_MAX_EV];
  int restarts;                     /* Lanczos restart cycles                                */
  double sign_applies;              /* sign-function applications (one per vector)          */
  double seconds;                   /* wall time                                             */
} lqcd_overlap_eigen_info;

/* The n_ev lowest eigenpairs of H_s for the sign function of the current
 * lqcd_overlap_setup: thick-restart Lanczos on H_s (double-float basis,
 * FP64 or double-float sign function per the set-up's `high`), then every
 * pair's residual recomputed and its partner formed.  The context keeps the
 * n_ev vectors and their partners (replacing an earlier eigensystem; a new
 * lqcd_overlap_setup drops it) for LQCD_OV_SOLVE_DEFLATED.  LQCD_ERR_NOCONV if
 * Lanczos does not converge within max_restarts or a recomputed residual
 * exceeds tol (info filled either way; no eigensystem is kept);
 * LQCD_ERR_STATE without an overlap set-up; LQCD_ERR_ARG for bad parameters
 * or a lattice too small for the basis.  Blocks.  Device memory: the basis,
 * 2 x (basis + 1) double-float vectors, during the solve; 2 n_ev FP64 vectors
 * kept. */
lqcd_status lqcd_overlap_eigen(lqcd_ctx *ctx, const lqcd_overlap_eigen_params *params,
                               lqcd_overlap_eigen_info *info);

/* Copy the kept eigenvectors (canonical full-lattice spinors, back to back,
 * host or device): the n_ev sector vectors in the order of info->mu
 * (partners = 0), or the n_partners partners (partners = 1), in the order of
 * their sector vectors.  LQCD_ERR_STATE without an eigensystem. */
lqcd_status lqcd_overlap_eigvecs(lqcd_ctx *ctx, double *vecs, int partners, int on_device);

/* LQCD_OV_SOLVE_DEFLATED: the same mass serves every eigenvector, since
 * D_ov(m)^dag D_ov(m) = (a^2 + a m / rho) D_ov(0)^dag D_ov(0) + m^2 with
 * a = 1 - m / (2 rho).  With W the kept vectors and mu'_w their eigenvalues
 * of D_ov(m)^dag D_ov(m), x0 = sum_w w <w, D_ov(m)^dag b> / mu'_w is the exact
 * component of the solution in their span (D_ov maps each pair span{chi,
 * eta} into itself, so this needs only inner products with W); the CG then
 * solves D_ov(m) e = b - D_ov(m) x0 to the target ||b - D_ov(m) x|| <=
 * tol ||b|| and returns x = x0 + e (info->iters counts its iterations).  The
 * mixed CG (cg->inner = LQCD_F32) deflates again at each accepted reliable
 * update.  A massless zero mode (mu' = 0) is not deflated. */

/* ---- domain decomposition along t: building blocks -------------------- */

/* The paper's multi-GPU runs (Sec. 4: the clover solve on a 96^3 x 192 lattice
 * over 324 GPUs, the overlap eigensystem over 4 GPUs) split the lattice
 * between GPUs.  Here a domain is an ordinary context whose lattice is its
 * share of the time slices plus `halo` ghost slices on either side (created
 * with t_antiperiodic = 0: the global time boundary's sign travels with the
 * ghost data instead).  Since t is the slowest site index, time slice t of a
 * parity is a contiguous run of Vh / L3 sites in the global order, so these
 * calls move and compute whole slices; the exchange between domains (NCCL,
 * gloo, or copies between domains of one process) belongs to the caller
 * (paper_2001_05706_gb300/domain.py drives it). */

/* Copy time slices [t0, t1) of parity `parity` of field f (all its
 * right-hand sides) to (to_field = 0) or from (to_field = 1) the device buffer
 * buf, laid out [rhs][16-byte word][site of the slices], multiplying every
 * real by factor (+1 or -1, exact).  FP64, FP32 and DF64 fields; buf holds
 * nrhs * (24 * bytes per real / 16) * (t1 - t0) * Vh / L3 words of 16 bytes
 * and must be device memory (LQCD_ERR_ARG otherwise).  Asynchronous on the
 * context's stream. */
lqcd_status lqcd_field_slices(lqcd_ctx *ctx, lqcd_field *f, int parity, int t0, int t1, void *buf, int to_field,
                              double factor);

/* The two kernels of the Schur complement (Table 2's D-slash with the clover
 * term, see lqcd_apply_schur) on the output sites of time slices [t0, t1)
 * only: y_e = A_ee^-1 D_eo x_o (dagger: with g5 on x), and
 * z_o = A_oo x_o - kappa^2 D_oe y_e (dagger: g5 on the hop).  Sites outside
 * the slices are not written.  lqcd_k2b_slices writes ||z_o||^2 over those
 * slices per right-hand side to norm2 (host, nrhs doubles; NULL: none) and
 * then blocks; otherwise asynchronous. */
lqcd_status lqcd_k2a_slices(lqcd_ctx *ctx, lqcd_recon recon, int dagger, lqcd_field *y_even, const lqcd_field *x_odd,
                            int t0, int t1);
lqcd_status lqcd_k2b_slices(lqcd_ctx *ctx, lqcd_recon recon, int dagger, lqcd_field *z_odd, const lqcd_field *x_odd,
                            const lqcd_field *y_even, int t0, int t1, double *norm2);

/* y = a[k] x + b[k] y on right-hand side k (a, b host arrays of nrhs
 * doubles), fields of one context with the same precision (FP64 or FP32),
 * subset and nrhs (<= 128); blocks. */
lqcd_status lqcd_field_axpby(lqcd_ctx *ctx, lqcd_field *y, const double *a, const double *b, const lqcd_field *x);

/* out[k] = ||f_k||^2 (FP64 fixed-order sum over every site f holds) per
 * right-hand side, host array of nrhs doubles (nrhs <= 256); blocks. */
lqcd_status lqcd_field_norm2s(lqcd_ctx *ctx, const lqcd_field *f, double *out);

/* ---- adaptive multigrid: building blocks ------------------------------- */

/* The paper's clover inverter at scale is QUDA's 3-level multigrid (Sec. 4:
 * aggregation blocks (4,4,4,4) and then (2,2,2,2); Table 1: all parts a
 * clover multigrid needs).  The paper gives no steps; these calls are those
 * of standard adaptive aggregation multigrid, and the Krylov iteration and
 * cycle around them are the caller's (paper_2001_05706_gb300/multigrid.py).
 *
 * Every level is a nearest-neighbour stencil on a periodic lattice dims[4]
 * (x fastest, V sites), with n complex components per site (even, 2..64),
 * the first n/2 of chirality +1 and the last n/2 of chirality -1:
 *   D v(x) = X(x) v(x) + sum_mu F_mu(x) v(x + mu) + B_mu(x) v(x - mu).
 * Arrays are the caller's device memory of the current device, complex FP64
 * as interleaved (re, im) pairs, 16-byte aligned: fields (V, n), X (V, n, n),
 * F and B (4, V, n, n) row-major, the prolongator P (V, n, nc) with
 * nc = 2 nv coarse components per block.  A block of block[mu] sites per
 * direction (dividing dims) is one coarse site; the coarse lattice is
 * dims / block.  Errors: LQCD_ERR_ARG for NULL, misaligned or host pointers
 * and sizes out of range; LQCD_ERR_CUDA for launch failures.  Asynchronous on
 * the context's stream unless stated. */

/* X, F, B of M = A - kappa D_W on the context's lattice: X = the clover term
 * A (c_sw = 0: the identity), F_mu = -kappa (1 - gamma_mu) U_mu(x), B_mu =
 * -kappa (1 + gamma_mu) U_mu(x - mu)^dag, with -1 on hops across the t
 * boundary when the context is antiperiodic; n = 12 (index 3 spin + colour,
 * DeGrand-Rossi, gamma5 = diag(1, 1, -1, -1)).  X holds V 144 complex, F and
 * B 4 V 144.  LQCD_ERR_STATE without a gauge field or lqcd_clover. */
lqcd_status lqcd_mg_fine_stencil(lqcd_ctx *ctx, void *X, void *F, void *B);

/* out = D in for the stencil (X, F, B) on dims with n components; in and out
 * distinct. */
lqcd_status lqcd_mg_apply(lqcd_ctx *ctx, const int dims[4], int n, const void *X, const void *F, const void *B,
                          const void *in, void *out);

/* The prolongator P (V, n, 2 nv) of nv vectors vecs (nv, V, n): on each block
 * and chirality the vectors restricted there, orthonormalised in their order
 * by Gram-Schmidt (classical, applied twice; real positive diagonal), coarse
 * components [chirality +1: nv, chirality -1: nv]; entries across
 * chiralities zero.  nv <= 32 and <= the block's sites x n/2.  Blocks;
 * LQCD_ERR_SINGULAR when a vector is dependent (within 1e-12) on the earlier
 * ones on some block. */
lqcd_status lqcd_mg_orthonormalize(lqcd_ctx *ctx, const int dims[4], int n, const int block[4], int nv,
                                   const void *vecs, void *P);

/* out (V, n) = P w for a coarse field w (dims / block sites, nc components). */
lqcd_status lqcd_mg_prolong(lqcd_ctx *ctx, const int dims[4], int n, const int block[4], int nc, const void *P,
                            const void *w, void *out);

/* out (coarse sites, nc) = P^H v for a fine field v (V, n). */
lqcd_status lqcd_mg_restrict(lqcd_ctx *ctx, const int dims[4], int n, const int block[4], int nc, const void *P,
                             const void *v, void *out);

/* The coarse stencil (Xc, Fc, Bc) of P^H D P on dims / block with nc
 * components: hops inside a block go to Xc, hops across its forward and
 * backward face in mu to Fc[mu] and Bc[mu]; sums in a fixed order. */
lqcd_status lqcd_mg_coarsen(lqcd_ctx *ctx, const int dims[4], int n, const int block[4], int nc, const void *X,
                            const void *F, const void *B, const void *P, void *Xc, void *Fc, void *Bc);

/* out[j] = <X_j, y> = sum_i conj(X_j[i]) y[i] for the k <= 64 vectors X_j of
 * len complex numbers stored one after the other; out is a host array of k
 * complex (2 k doubles).  Fixed-order sums; blocks. */
lqcd_status lqcd_mg_dots(lqcd_ctx *ctx, long len, int k, const void *X, const void *y, double *out);

/* y += sum_j coef[j] X_j for k <= 64 vectors (coef: host, k complex). */
lqcd_status lqcd_mg_axpys(lqcd_ctx *ctx, long len, int k, const double *coef, const void *X, void *y);

/* y = a x + b y (a, b: host complex; x may be y). */
lqcd_status lqcd_mg_axpby(lqcd_ctx *ctx, long len, const double a[2], const void *x, const double b[2], void *y);

/* ---- allocation-free reduction ---------------------------------------- */

/* The paper has no counterpart of this call.  result[k] = sum_i x[k*n + i]^2
 * for k < nrhs: the FP64 fixed-order sum of squares of nrhs device vectors
 * of n doubles each (for example canonical spinors, n = 24 V), written to
 * the device array `result` on `cuda_stream` (NULL: default stream); the
 * call does not wait for it.  It allocates nothing, for callers that cannot
 * call cudaMalloc (device memory owned by another allocator, or
 * latency-critical loops where cudaMalloc/cudaFree would synchronise the
 * device): its scratch -- at most 1024 x 64 partial sums (512 KiB) and a
 * counter -- is a static array of the library that every GPU loading it
 * holds until the process exits.  The first call on a device (and on each
 * new CUDA context of it, for example after cudaDeviceReset) looks up that
 * array's device address, so make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (on
 * different streams, or from several threads) race and give wrong results.
 * nrhs > 64, n < 1 or n > 2^40, and x or result not device (or managed)
 * memory of the current device give LQCD_ERR_ARG; the sizes of the arrays
 * cannot be checked (x must hold n * nrhs doubles, result nrhs); no context
 * is needed. */
lqcd_status lqcd_norm2_noalloc(const double *x, long n, int nrhs, double *result, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
