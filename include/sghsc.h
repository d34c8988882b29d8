/*
 * sghsc.h -- C ABI of the GB300 stochastic Galerkin solver with the
 * hierarchical Schur complement (HSC) preconditioner.
 *
 * Method: B. Sousedik, R. G. Ghanem, E. T. Phipps, "Hierarchical Schur
 * complement preconditioner for the stochastic Galerkin finite element
 * methods" (arXiv 1205.1864).
 *
 * The system is eq. (global-system) of Sec. 2,
 *     sum_k  G_k (x) A_k  u = f,        k = 0..M,
 * with A_0..A_M the Karhunen-Loeve stiffness matrices (the paper's K_i) on one
 * shared sparsity pattern and (G_k)_{jl} = E[xi_k psi_j psi_l], G_0 = I, for
 * the normalised chaos basis of total degree <= p in M variables
 * (P = (M+p)!/(M! p!) polynomials, eq. (gPC-u)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout of a coefficient block: "n x P row-major" -- element (r, l) at
 *   offset r*P + l, r the spatial row (0..n-1), l the chaos index (0..P-1).
 *   In this layout the operator reads Y = sum_k A_k U G_k^T.
 * Chaos order: degrees ascending (graded, as Sec. 3 requires); inside one
 *   degree, descending lexicographic order of (alpha_1, ..., alpha_M). So
 *   l = 0 is the mean, l = 1..M are xi_1..xi_M. sg_chaos_table() exports it.
 * Memory: arguments named "host" are host pointers; every vector argument of
 *   an apply/solve call is a DEVICE pointer on the current CUDA device. The
 *   caller owns all buffers it passes; sg_setup copies what it needs and the
 *   handle owns its device copies and workspace until sg_destroy.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Work is enqueued on it; calls that report per-iteration results
 *   synchronise it. Calls on one handle must not overlap (the handle's
 *   workspace is shared by all its calls).
 * Errors: every call returns an sg_status; invalid arguments are rejected
 *   before any launch; sg_last_error() returns a thread-local message for the
 *   last failure. Nothing traps or aborts; device loops have iteration caps
 *   and report through the status.
 */
#ifndef SGHSC_H
#define SGHSC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_problem sg_problem;

typedef enum {
  SG_OK = 0,
  SG_ERR_INVALID_ARG = 1,     /* a pointer, size, pattern or option is invalid */
  SG_ERR_CUDA = 2,            /* a CUDA runtime call failed */
  SG_ERR_OOM = 3,             /* device allocation failed */
  SG_ERR_NOT_SPD = 4,         /* an inner solve met p^T A_0 p <= 0 */
  SG_ERR_BREAKDOWN = 5,       /* the outer solve met p^T A p <= 0 or a non-finite value */
  SG_ERR_NO_CONVERGENCE = 6,  /* the outer solve reached maxit */
  SG_ERR_UNSUPPORTED = 7      /* valid input outside what this build implements */
} sg_status;

enum { SG_F64 = 0, SG_F32 = 1 };                     /* element type of a block */
/* sg_level_apply only: X and Yout FP32, Yin FP64, products accumulated and
 * subtracted in FP64 (the level-p products of the mixed preconditioner with
 * top_level_f64, Algorithm 1), or in double-float arithmetic on the FP32
 * units (the same with sg_prec_opts.df64). */
enum { SG_F32_ACC64 = 2, SG_F32_ACCDF64 = 3 };
enum { SG_LEGENDRE = 0, SG_HERMITE = 1 };            /* chaos family */
enum { SG_PREC_NONE = 0, SG_PREC_MEAN = 1, SG_PREC_HSC = 2, SG_PREC_BGS = 3 };

/* Uniform grid of ne_x x ne_y bilinear (Q1) elements on the unit square with
 * Dirichlet nodes eliminated: n = (ne_x-1)(ne_y-1) interior nodes, numbered
 * lexicographically with x fastest (Sec. 6 discretisation). The inner solves
 * need it (and the 9-point pattern of the Q1 stencil); the multigrid inner
 * preconditioner also needs ne_x == ne_y, a power of two. */
typedef struct { int ne_x, ne_y; } sg_mesh;

/* Options of one preconditioner application (Algorithm 1, Sec. 4; inner
 * loops of Sec. 5). */
typedef struct {
  int precision;          /* SG_F32: inner solves and level products in FP32 (mixed);
                             SG_F64: everything in FP64 */
  int top_level_f64;      /* with SG_F32: the level-p off-diagonal products of
                             Algorithm 1 are computed in FP64 */
  double inner_tol;       /* per-column relative residual of the inner PCG on A_0 */
  int inner_maxit;        /* cap on inner iterations (status bit set when reached) */
  int inner_fixed_iters;  /* > 0: run exactly this many inner iterations, no tolerance test */
  int nu;                 /* V-cycle: weighted-Jacobi sweeps before and after */
  double omega;           /* V-cycle: Jacobi damping */
  int m0;                 /* mean-value preconditioner M_0 of the inner PCG (Sec. 5 leaves it
                             open): SG_M0_VCYCLE one multigrid V-cycle (needs a power-of-two
                             square mesh), SG_M0_DIAG the diagonal of A_0 (any mesh given to
                             sg_setup whose pattern is the 9-point Q1 stencil) */
  double level_tol;       /* gPC coefficient (sg_setup_gpc) only: D_l is not block diagonal
                             (Sec. 6, lognormal case), so D_l^{-1} is a nested flexible CG on
                             the level block, preconditioned by the inner PCG on A_0 per
                             column, to this relative residual */
  int level_maxit;        /* cap on the iterations of that nested CG */
  int md_m0;              /* variants of eq. (general-prec), Sec. 5: bit 0 replaces M_D^1 (the
                             D_l^{-1} of the pre-correction) and bit 1 replaces M_D^2 = M_D^3
                             (the D_l^{-1} of the post-correction, applied to r_l - C_l u) by
                             the mean-value preconditioner M_0 alone (one V-cycle or the
                             diagonal, per m0) instead of the inner PCG; 0 is Algorithm 1.
                             Linear KL expansion only (the D_l of a gPC coefficient is not
                             I (x) A_0). */
  int df64;               /* with precision SG_F32: 1 runs the FP64-accurate products that read
                             the FP32 preconditioner's output -- the level-p products of
                             Algorithm 1 (top_level_f64) and, in sg_solve, the outer SG product
                             q = A p -- in double-float arithmetic (pairs of FP32 numbers, a
                             48-bit significand; products and sums by error-free
                             transformations) on the FP32 units, whose multiply-add rate on this
                             GPU is about 70 times the FP64 one; each output is finished in
                             FP64. 0: FP64 arithmetic. */
} sg_prec_opts;

enum { SG_M0_VCYCLE = 0, SG_M0_DIAG = 1 };

/* Options of the outer flexible CG (Sec. 5-6). */
typedef struct {
  int precond;            /* SG_PREC_NONE, SG_PREC_MEAN (I (x) A_0^{-1}, Sec. 6), SG_PREC_HSC
                             (Algorithm 1) or SG_PREC_BGS (block symmetric Gauss-Seidel, Sec. 6) */
  sg_prec_opts prec;
  double tol;             /* stop at ||r||_2 <= tol ||f||_2 (recursive residual) */
  int maxit;
  int flexible;           /* 1: beta = z_{k+1}^T (r_{k+1}-r_k)/(z_k^T r_k); 0: standard CG */
  int use_x0;             /* 1: U holds the initial guess on entry */
  int check_true_residual;/* 1: recompute ||f - A u|| / ||f|| in FP64 after the loop
                             (one more SG product) into stats->true_rel_res */
  int schur_reduced;      /* 1: iterate on the Schur-reduced system of Sec. 5,
                             eq. (global-Schur-system): S_{p-1} u_{p-1} = g_{p-1} with
                             S_{p-1} = A_{p-1} - B_p D_p^{-1} C_p, g_{p-1} = f^{p-1} - B_p D_p^{-1} f^p,
                             the preconditioner on levels 0..p-1 only, then
                             u^p = D_p^{-1} (f^p - C_p u_{p-1}). Needs p >= 1 and use_x0 = 0;
                             tol, iterations, rel_res and kappa_est refer to the reduced system,
                             true_rel_res to the full one. */
  double schur_inner_tol; /* relative tolerance of the FP64 inner solves that apply D_p^{-1}
                             inside S_{p-1} (the reduction assumes exact solves, Sec. 5) */
} sg_solve_opts;

#define SG_MAX_HIST 1024

typedef struct {
  int status;             /* sg_status of the solve */
  int iterations;         /* outer operator applications */
  double rel_res;         /* final recursive relative residual */
  double true_rel_res;    /* ||f - A u|| / ||f|| recomputed in FP64 at the end
                             (-1 when check_true_residual is 0) */
  double kappa_est;       /* Lanczos estimate from the CG coefficients (Sec. 6) */
  long long inner_iters_total;   /* sum over all inner column solves */
  int inner_iters_max;    /* largest inner iteration count of one column */
  double solve_ms;        /* host wall time of the call */
  int n_hist;             /* entries of res_hist (iterations + 1) */
  double res_hist[SG_MAX_HIST + 1];
  double alpha[SG_MAX_HIST];
  double beta[SG_MAX_HIST];
} sg_solve_stats;

/* sg_default_prec_opts, sg_default_solve_opts -- fill an options struct with
 * the library defaults (host memory; a NULL pointer is ignored; no device
 * call). Preconditioner: precision SG_F32, top_level_f64 1, inner_tol 1e-2,
 * inner_maxit 200, inner_fixed_iters 0, nu 2, omega 0.8, m0 SG_M0_VCYCLE,
 * level_tol 1e-8, level_maxit 500, md_m0 0 (Algorithm 1 itself), df64 0.
 * Solve: precond SG_PREC_HSC, prec as above, tol 1e-8 (the stopping test of
 * Sec. 6), maxit 500, flexible 1, use_x0 0, check_true_residual 1,
 * schur_reduced 0, schur_inner_tol 1e-11. */
void sg_default_prec_opts(sg_prec_opts* o);
void sg_default_solve_opts(sg_solve_opts* o);

/* sg_setup -- build a problem handle (Sec. 2, eq. (global-system); Sec. 3).
 * mesh      host, may be NULL: needed for the multigrid inner solves.
 * M, p      number of random variables and total chaos degree (M >= 0, p >= 0).
 * family    SG_LEGENDRE (xi ~ U(-sqrt3, sqrt3)) or SG_HERMITE (xi ~ N(0,1)).
 * n, nnz    spatial size and nonzeros of the shared CSR pattern.
 * rowptr    host int[n+1], colidx host int[nnz] (sorted, in range).
 * vals      host double[nnz][M+1]: entry e of A_k at vals[e*(M+1) + k].
 * mass_vals host double[nnz] or NULL: consistent mass matrix on the same
 *           pattern (needed by sg_qoi / sg_qoi_grad).
 * out       receives the handle. The chaos tables (multi-indices, the sparse
 *           G_k) and the multigrid hierarchy are built here.
 * Returns SG_ERR_INVALID_ARG for a malformed pattern or sizes (checked on
 * the host before any device call), SG_ERR_OOM if device memory runs out,
 * SG_ERR_CUDA without a usable CUDA device (there is no CPU fallback); on any
 * error *out is NULL. */
int sg_setup(const sg_mesh* mesh, int M, int p, int family, int n, int nnz,
             const int* rowptr, const int* colidx, const double* vals,
             const double* mass_vals, sg_problem** out);

/* sg_setup_gpc -- a handle for a coefficient given by its generalised
 * polynomial chaos expansion k = sum_i k_i(x) psi_i(xi) (Remark K-L of Sec. 2;
 * Sec. 6, the lognormal case): vals host double[nnz][nterm] holds the
 * stiffness matrices of the nterm = C(M+q, M) coefficient terms k_i, in the
 * graded chaos order (term 0 the mean, whose matrix is A_0), and the
 * operator is sum_i G_i (x) A_i with (G_i)_{jl} = E[psi_i psi_j psi_l]
 * (the paper expands the lognormal coefficient to q = 2p). Only Hermite
 * chaos (family SG_HERMITE, xi ~ N(0,1)); q <= 16, nterm <= 4096. The
 * coupling is block dense: B_l and C_l reach every lower degree, D_l is not
 * block diagonal (hsc_precond_apply solves with it by a nested CG,
 * sg_prec_opts.level_tol; FP64 only; bgs_precond_apply and the
 * Schur-reduced system return SG_ERR_UNSUPPORTED). Other arguments and
 * errors as sg_setup; SG_ERR_UNSUPPORTED for another family. */
int sg_setup_gpc(const sg_mesh* mesh, int M, int p, int q, int family, int n, int nnz, const int* rowptr,
                 const int* colidx, const double* vals, const double* mass_vals, sg_problem** out);

/* Value terms per nonzero of a handle (M+1, or C(M+q, M) for sg_setup_gpc)
 * and its coefficient degree q (-1 for the linear KL expansion). */
int sg_problem_terms(const sg_problem* h, int* nterm, int* q);

void sg_destroy(sg_problem* h);

/* sg_set_scales -- A_k := scale[k] * A_k(as given to sg_setup), k = 0..M, for
 * parameterised KL matrices (A_0 = a_mean L_h, A_k = sigma s_k Phi_k): one
 * handle then serves every parameter set. scale: host double[M+1] (one per
 * value term: nterm for sg_setup_gpc), finite,
 * scale[0] > 0 when the multigrid hierarchy exists (it is rescaled too).
 * Synchronises the device. */
int sg_set_scales(sg_problem* h, const double* scale);

/* Sizes of a handle (host outputs, any may be NULL). */
int sg_problem_dims(const sg_problem* h, int* n, int* P, int* M, int* p, int* nnz);

/* The chaos order: alpha host int[P*M] (row l is the multi-index of psi_l)
 * and level_offsets host int[p+2] (degree d occupies [off[d], off[d+1])). */
int sg_chaos_table(const sg_problem* h, int* alpha, int* level_offsets);

/* sg_apply -- MAT-VEC of eq. (global-system) (the remark after
 * eq. (global-matrix-block)): Y = sum_k A_k U G_k^T.
 * U, Y: device n x P row-major of element type dtype (SG_F64 or SG_F32);
 * or dtype SG_F32_ACCDF64: U FP32, Y FP64, the sums in double-float
 * arithmetic (FP32 pairs: within about m 2^-46 of the sum of the magnitudes
 * of the m terms of an entry) -- the product the mixed solver applies to the
 * FP32 output of its preconditioner. Y must not alias U. */
int sg_apply(sg_problem* h, const void* U, void* Y, int dtype, void* stream);

/* sg_level_apply -- one off-diagonal block product of the hierarchy
 * (eq. (global-matrix-hierarchy)): Yout = Yin - sum_k A_k X G_k[out, in]^T
 * with out, in two adjacent degree levels (|lvl_out - lvl_in| = 1): the
 * pre-correction product B_l (out = l-1, in = l) and the post-correction
 * product C_l (out = l, in = l-1) of Algorithm 1.
 * X: device n x w_in packed; Yin, Yout: device n x w_out packed (may alias);
 * w_d = number of chaos polynomials of degree d. dtype SG_F64 or SG_F32 for
 * all three blocks, or SG_F32_ACC64 / SG_F32_ACCDF64: X and Yout FP32, Yin
 * FP64 (required, not aliasing Yout), the sum accumulated in FP64 or in
 * double-float arithmetic. */
int sg_level_apply(sg_problem* h, int lvl_out, int lvl_in, const void* X, const void* Yin,
                   void* Yout, int dtype, void* stream);

/* sg_vcycle_apply -- one multigrid V-cycle with zero initial guess for A_0
 * applied independently to the w columns of B (the mean-value
 * preconditioner M_0 of Sec. 4-5). B, X: device n x w packed, w <= 1024. */
int sg_vcycle_apply(sg_problem* h, const void* B, void* X, int w, int dtype,
                    const sg_prec_opts* opts, void* stream);

/* sg_vcycle_apply_static -- sg_vcycle_apply without allocating device memory.
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not call cudaMalloc while they run (code inside a CUDA stream
 * capture, allocator or memory-pool hooks, processes whose device memory is
 * budgeted and already handed out). The V-cycle's level buffers live in a
 * fixed 32 MiB array inside the library, which every GPU that loads the
 * library keeps until the process exits. Arguments and results are those of
 * sg_vcycle_apply (B, X: device n x w packed, w <= 1024, dtype SG_F64 or
 * SG_F32); the handle must come from sg_setup as usual. The scratch of one
 * call is, in elements of dtype, 3 n_0 wp + 3 (n_1 + n_2 + ...) wp plus wp
 * ints, each of these 1 + 3 G blocks rounded up to 256 bytes, where n_g is
 * the node count of multigrid grid g (n_0 = n, n_1 ~ n/4, ...) and wp is w
 * rounded up to the vector width (4 columns in FP32, 2 in FP64). A batch whose
 * scratch exceeds the 32 MiB is rejected with SG_ERR_INVALID_ARG. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current), so make that first call before any stream
 * capture; a lookup that fails is retried by the next call. All calls on a
 * device share the array and it keeps the last call's contents: calls whose
 * GPU work overlaps race. */
int sg_vcycle_apply_static(sg_problem* h, const void* B, void* X, int w, int dtype,
                           const sg_prec_opts* opts, void* stream);

/* sg_inner_solve -- the batched inner PCG on A_0 (Sec. 5: independent
 * Krylov loops for the diagonal blocks of D_l), V-cycle preconditioned,
 * per-column convergence: column s stops once ||r_s|| <= inner_tol ||b_s||;
 * zero columns are done at entry with x = 0. B, X: device n x w packed,
 * w <= 1024. iters: host int[w] or NULL (per-column iteration counts;
 * synchronises the stream). */
int sg_inner_solve(sg_problem* h, const void* B, void* X, int w, int dtype,
                   const sg_prec_opts* opts, int* iters, void* stream);

/* sg_inner_cluster -- 1 when the FP32 inner solves of h (sg_inner_solve, and
 * the D_l and A_0 solves inside hsc_precond_apply, mean_precond_apply and
 * sg_solve) run on the cluster-resident solver: one launch per solve, the
 * multigrid hierarchy of each group of 4 columns held in the shared memory of
 * a cluster of 8 thread blocks. 0 when they run on the stand-alone kernels:
 * FP64 solves always do, and so does a grid hierarchy too large for one
 * block's shared memory (finest grids above 127 x 127 nodes), a device that
 * cannot hold such a cluster, or a handle created while the environment
 * variable SGHSC_NO_CLUSTER was 1. A batch of w columns uses the cluster
 * solver only when its ceil(w/4) clusters are all resident at once (on a
 * GB300, up to 60 columns); wider batches take the stand-alone kernels. Both
 * solvers compute the same method; their results differ by FP32 rounding
 * (summation order). h NULL: 0. */
int sg_inner_cluster(const sg_problem* h);

/* sg_inner_path -- which solver a batched inner solve of w columns of element
 * type dtype takes on h: 0 the stand-alone kernels, 1 the cluster solver with
 * the whole multigrid hierarchy in shared memory (ceil(w/4) clusters of 8
 * blocks, all resident at once), 3 the same with clusters of 16 blocks (half
 * the rows per block; taken first when all ceil(w/4) of them are resident),
 * 2 the cluster solver with the finest grid in global memory and the coarse
 * grids in shared memory (two blocks per SM, for batches too wide for 1).
 * After sg_autotune, the solver it timed fastest for that width (one of those
 * eligible); else the first eligible of 3, 1, 2, then 0.
 * h NULL or w <= 0: 0. */
int sg_inner_path(const sg_problem* h, int w, int dtype);

/* hsc_precond_apply -- Algorithm 1 (Sec. 4): Z = M_P R with the D_l^{-1}
 * and A_0^{-1} actions replaced by the batched inner PCG.
 * R, Z: device n x P row-major FP64; must not alias. */
int hsc_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts,
                      void* stream);

/* bgs_precond_apply -- block symmetric Gauss-Seidel with zero initial guess
 * (M_bGS, the comparison preconditioner of Sec. 6): a forward and a backward
 * sweep over the chaos blocks K^(j,l) = sum_k c_kjl A_k of eq. (global-matrix)
 * in the graded chaos order, each diagonal block (A_0) solved by the batched
 * inner PCG. Blocks of one degree do not couple, so each sweep runs level by
 * level, a level's columns in one batch; the top level is solved once (its
 * backward step equals its forward one). Precision options as for
 * hsc_precond_apply (top_level_f64: the level-p forward product in FP64).
 * R, Z: device n x P row-major FP64; must not alias. */
int bgs_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts, void* stream);

/* mean_precond_apply -- mean-based preconditioner I (x) A_0^{-1} (Sec. 6,
 * Powell-Elman) with the same inner PCG. R, Z: device n x P FP64. */
int mean_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts,
                       void* stream);

/* sg_solve -- flexible CG on eq. (global-system) preconditioned by
 * opts->precond (Sec. 5-6), outer iteration in FP64.
 * F: device n x P FP64 right-hand side; U: device n x P FP64 solution (initial
 * guess on entry when opts->use_x0). stats: host, may be NULL.
 * Returns SG_ERR_NO_CONVERGENCE if maxit is reached (U holds the last
 * iterate), SG_ERR_BREAKDOWN / SG_ERR_NOT_SPD on loss of definiteness. */
int sg_solve(sg_problem* h, const double* F, double* U, const sg_solve_opts* opts,
             sg_solve_stats* stats, void* stream);

/* sg_solve_host -- sg_solve with the right-hand side and the solution in host
 * memory: F_host (n x P FP64, read) and U_host (n x P FP64, written; read as
 * the initial guess when opts->use_x0), both owned by the caller, row-major.
 * Page-locked buffers (cudaHostAlloc, cudaHostRegister; torch pin_memory)
 * are read and written by the library's kernels through their device mapping,
 * over the host link; other host memory goes through cudaMemcpyAsync. Returns
 * when U_host holds the result (the call synchronises the stream). Errors as
 * sg_solve. No counterpart in the paper (the end-to-end entry). */
int sg_solve_host(sg_problem* h, const double* F_host, double* U_host, const sg_solve_opts* opts,
                  sg_solve_stats* stats, void* stream);

/* sg_autotune -- time the candidate block sizes (64 to 1024 threads) of the
 * full SG product in FP64 and FP32, and separately of the outer solver's fused
 * product (SG product + CG update + p.q, in FP64 and in its double-float
 * variant, sg_prec_opts.df64), each in two forms, on this problem
 * and keep the fastest for all later calls (products that take a fixed-shape
 * kernel -- the FP32 row kernel, the staged double-float kernel -- are not
 * timed). The forms: the pair form sums each distinct (k, j) of the couplings
 * once per row and keeps those sums in shared memory (fewer multiply-adds);
 * the gather form sums per coupling (no extra shared memory). Where several
 * inner solvers can run a degree level's FP32 batch (grids up to 127 x 127:
 * the stand-alone kernels, the 8- and 16-CTA cluster solvers, the wide one),
 * each is timed on a batch of that width (two fixed PCG iterations) and the
 * fastest is kept (sg_inner_path reports it). Allocates temporary blocks and,
 * if absent, the outer solve buffers; invalidates the handle's cached solve
 * graphs. */
int sg_autotune(sg_problem* h, void* stream);
/* Results are cached per problem class (device, n, nnz, M, p, family, the
 * longest row of the pattern and the coefficient degree): a later handle of a
 * class already tuned in this process takes the cached choices without timing
 * anything. */
/* Block sizes chosen by sg_autotune (0: not tuned, the built-in choice). */
int sg_autotune_result(const sg_problem* h, int* threads_f64, int* threads_f32);
/* Block size chosen for the outer solver's fused product (0: the built-in 256). */
int sg_autotune_outer_result(const sg_problem* h, int* threads_outer);
/* sg_autotune_set -- pin the shapes sg_autotune would choose, without timing:
 * block sizes of the full SG product in FP64 and FP32 and of the outer fused
 * product (0: the built-in choice; otherwise whole warps, 32..1024 threads,
 * at most 8 outputs per thread, 4 above 256 threads), and the pair (1) or
 * gather (0) form of each (the outer shape applies to its FP64 and its
 * double-float variant). SG_ERR_INVALID_ARG for an unusable block size.
 * Invalidates the handle's cached solve graphs. */
int sg_autotune_set(sg_problem* h, int threads_f64, int threads_f32, int threads_outer, int pairs_f64,
                    int pairs_f32, int pairs_outer);
/* Forms chosen by sg_autotune: 1 the pair form, 0 the gather form, for the
 * full SG product in FP64 and FP32 and for the outer fused product (all 1
 * before tuning). Any pointer may be NULL. */
int sg_autotune_forms(const sg_problem* h, int* pairs_f64, int* pairs_f32, int* pairs_outer);

/* Batched solves of many independent systems (uneven n, M, p): one graph
 * launch runs every system's whole solve (its outer flexible CG and nested
 * inner loops) as an independent branch. The handles stay owned by the
 * caller and must outlive the batch; a handle may belong to one batch. */
typedef struct sg_batch sg_batch;
/* problems: host array of count >= 1 distinct, non-NULL handles. *out is the
 * batch, or NULL on any error (SG_ERR_INVALID_ARG for a NULL or repeated
 * handle, SG_ERR_CUDA if its streams cannot be created). */
int sg_batch_create(int count, sg_problem* const* problems, sg_batch** out);
/* F, U: host arrays of count device pointers (n_i x P_i FP64 each);
 * stats: host array of count entries or NULL. Returns SG_OK when every system
 * converged, else the first failure (per-system status in stats). */
int sg_batch_solve(sg_batch* b, const double* const* F, double* const* U, const sg_solve_opts* opts,
                   sg_solve_stats* stats, void* stream);
/* sg_batch_solve_host -- sg_batch_solve with host blocks F_host[i], U_host[i]
 * (moved as by sg_solve_host: page-locked ones by the library's kernels). */
int sg_batch_solve_host(sg_batch* b, const double* const* F_host, double* const* U_host,
                        const sg_solve_opts* opts, sg_solve_stats* stats, void* stream);
void sg_batch_destroy(sg_batch* b);

/* sg_qoi -- Q = sum_j u_j^T M_h u_j = E[int u^2] for the orthonormal chaos
 * basis; also writes dQ/dU = 2 M_h U to dQdU when not NULL.
 * U, dQdU: device n x P FP64; q_out: device double[1]. Needs mass_vals. */
int sg_qoi(sg_problem* h, const double* U, double* dQdU, double* q_out, void* stream);

/* sg_qoi_grad -- adjoint gradient contraction: with h_k = <Lam, A_k U G_k^T>_F,
 * grad[t] = sum_k W[t*(M+1) + k] h_k for t = 0..nparam-1 (W host, for
 * A_k(theta) = theta-scaled KL matrices W = -d log A_k / d theta).
 * U, Lam: device n x P FP64; grad: device double[nparam]; hk_out: device
 * double[M+1] or NULL. */
int sg_qoi_grad(sg_problem* h, const double* U, const double* Lam, int nparam, const double* W,
                double* grad, double* hk_out, void* stream);

/* sg_measure_alu_peak -- measured multiply-add rate of the current device in
 * FP64 (dtype SG_F64) or FP32 (SG_F32): one warm-up and one timed launch of a
 * kernel made of independent FMA chains (8 per thread, every SM filled),
 * timed with CUDA events on `stream` (synchronised). iters: chain steps per
 * thread / 8 (for example 4096 in FP64, 131072 in FP32, about 0.1 s each on a
 * GB300). flops_per_s: host, receives 2 x FMAs / second. The paper has no
 * counterpart: this is the roofline denominator of the ALU-bound products,
 * measured instead of derived from unit counts and clocks. */
int sg_measure_alu_peak(int dtype, int iters, double* flops_per_s, void* stream);

/* The gradient workload's parameterisation (the paper has no gradient): the
 * handle holds the KL matrices with unit parameters (A_0 = L_h, A_k = Phi_k,
 * i.e. assembled with a_mean = 1, sigma = 1, s_k = 1) and
 * theta = (a_mean, sigma, s_1..s_M), host double[M+2], finite and nonzero,
 * a_mean > 0, makes A_0 = a_mean L_h and A_k = sigma s_k Phi_k.
 * sg_kl_set_theta -- sg_set_scales with those factors (synchronises).
 * sg_kl_qoi_grad -- dQ/dtheta, device double[M+2], from the forward solution
 * U and the adjoint solution Lam (device n x P FP64) of the current theta:
 * dQ/dtheta_t = -sum_k (d log scale_k / d theta_t) <Lam, A_k U G_k^T>_F
 * (sg_qoi_grad with those weights); hk_out as there. */
int sg_kl_set_theta(sg_problem* h, const double* theta);
int sg_kl_qoi_grad(sg_problem* h, const double* U, const double* Lam, const double* theta, double* grad,
                   double* hk_out, void* stream);

/* Thread-local message of the last failure ("" if none). */
const char* sg_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (a monotone counter for measurement). */
long long sg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* SGHSC_H */
