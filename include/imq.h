/*
 * imq.h -- C ABI of the GB300 library for the fast inverse-multiquadric (IMQ)
 * matrix-vector product and the interpolation solve built on it.
 *
 * Method: De Marchi, Egidi, Giacomini, Maponi, Perticarini, "Computational
 * issues by interpolating with inverse multiquadrics: a solution",
 * arXiv 2205.04194.
 *
 *   Section 2, Eq. (4)-(5):  A_ij = phi(|x_i - x_j|) = 1 / sqrt(|x_i - x_j|^2 + c^2)
 *     (the paper names the shape parameter t; it is c here, c > 0).
 *   Section 2.2, Eq. (11)-(13) and Algorithm 1: each entry is the Laplace Green's
 *     function 1/|X - Y| between X = (x_i, +c/2) and Y = (x_j, -c/2), expanded in
 *     spherical harmonics about quadtree box centres to truncation order p, so
 *     that only adjacent ("not well separated") boxes are summed directly.
 *
 * Conventions for every entry point:
 *   - Arrays are dense and row-major.  A point set is double[N][2] (x, y).  A
 *     block of vectors is [nrhs][N] (vector r at offset r*N).
 *   - "Host or device" pointers are classified with cudaPointerGetAttributes:
 *     device (and managed) memory is used in place; pageable or pinned host
 *     memory is copied to the device and results are copied back, inside the
 *     call, on `stream`.  Results written to host memory are complete when the
 *     call returns (the call synchronises `stream`); results written to device
 *     memory are complete when `stream` reaches the end of the enqueued work.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All GPU
 *     work of a call is enqueued on it.
 *   - The caller owns every buffer it passes; no pointer is retained after the
 *     call returns.  A plan owns its own device memory until imq_plan_destroy.
 *   - Every call returns an imq_status; no C++ exception crosses the ABI.  On
 *     error the output buffers hold unspecified values, and imq_last_error()
 *     returns a message (thread-local, valid until the next call on the thread).
 *   - The library requires a CUDA device of compute capability 10.3 (sm_103a)
 *     and fails with IMQ_UNSUPPORTED elsewhere; there is no CPU fallback.
 */
#ifndef IMQ_H
#define IMQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum imq_status {
    IMQ_OK = 0,
    IMQ_INVALID_ARG = 1,       /* bad size, pointer, c <= 0, NaN/Inf coordinates ...   */
    IMQ_DUPLICATE_POINTS = 2,  /* two points are exactly equal (Section 2 needs distinct sites) */
    IMQ_CUDA_ERROR = 3,        /* a CUDA runtime call failed                              */
    IMQ_OOM = 4,               /* device allocation failed                                */
    IMQ_NOT_CONVERGED = 5,     /* iteration cap reached; best iterate returned            */
    IMQ_NUMERICAL = 6,         /* NaN/Inf met inside an iteration                         */
    IMQ_UNSUPPORTED = 7,       /* p outside [1, IMQ_MAX_P], wrong GPU, option not built    */
    IMQ_TIMEOUT = 8            /* a device-side bounded wait gave up                      */
} imq_status;

typedef enum imq_dtype {
    IMQ_F32 = 0,   /* the expansion path in FP32 (P2P, P2M ... L2P; FP32 rsqrt)     */
    IMQ_F64 = 1    /* every kernel of the product in FP64                          */
} imq_dtype;

#define IMQ_MAX_P 18
#define IMQ_MAX_LEVEL 16

/* Opaque plan: the tree, its interaction lists and the translation operators
 * for one point set, one shape c and one truncation order p. */
typedef struct imq_plan_s *imq_plan_t;

/* Optional plan settings.  Zero-initialise, set struct_size = sizeof(imq_options). */
typedef struct imq_options {
    int32_t struct_size;
    int32_t has_domain;        /* 1: use (x0, y0, side) as the square D (Section 2.2) */
    double x0, y0, side;       /*    otherwise D is the exact bounding square          */
    int32_t check_duplicates;  /* 1: imq_plan fails with IMQ_DUPLICATE_POINTS on equal points */
    int32_t m2l_kernel;        /* imq_m2l_kernel: how the FP32 product runs M2L             */
    int32_t algorithm;         /* imq_algorithm: the fast multipole form (default) or the
                                  paper's treecode, Algorithm 1                              */
    int32_t levels;            /* IMQ_ALG_TREECODE: the paper's L (1..15): blocks of the
                                  finest level are 2^(L+1) x 2^(L+1); `leaf` is ignored      */
    int32_t translations;      /* imq_translations: precision of M2M / M2L / L2L in the FP32
                                  product (IMQ_ALG_FMM, p <= 16)                             */
    /* Tile shapes of the FP32 product (0: the default; imq_autotune measures them):        */
    int32_t p2p_warps;         /* target leaves (warps) per P2P CTA: 2, 4 (default) or 8    */
    int32_t p2p_chunk;         /* targets per P2P register tile: 8, 16 (default) or 32      */
    int32_t m2l_stages;        /* tensor-core M2L pipeline stages: 2..6 (default: as many as
                                  fit in shared memory; more than fit, or fewer than 4, are
                                  clamped)                                                   */
    int32_t m2l_split;         /* tensor-core M2L: CTAs sharing one 128-box tile's offset
                                  classes, 1..4 (default: by the tile count)                  */
    /* Optional allocator of the plan's own device buffers (tree, lists, operators,
     * expansions, solver work arrays), e.g. a framework's caching allocator.  Both
     * NULL: cudaMalloc / cudaFree.  alloc returns device memory of at least `bytes`
     * (16-byte aligned) or NULL (the call then fails with IMQ_OOM); free receives
     * each such block once, when the plan is destroyed or the buffer is replaced,
     * after the device has finished with it.  Per-call temporaries stay
     * stream-ordered (cudaMallocAsync).  Read only when struct_size covers them. */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *ctx);
    void *alloc_ctx;
} imq_options;

/* How imq_matvec evaluates the product.
 *   FMM      : adaptive quadtree (split while a box holds more than `leaf`
 *              points); multipoles translated to local expansions (M2L, L2L)
 *              and evaluated once per target; the paper's M2P only on the
 *              W lists of the adaptive tree.
 *   TREECODE : Algorithm 1 of Section 2.2 on a uniform partition: levels
 *              l = 1..L of 2^(l+1) x 2^(l+1) blocks, the moments of every block
 *              (here P2M at the finest level and M2M upward, equal to the
 *              per-level moments up to rounding), the far-field sum of
 *              Eq. (13) at every target for the blocks of S_p at every level
 *              (M2P over the union of the V lists of the target block's
 *              ancestors), and the direct sum over NS_p at level L (U lists). */
typedef enum imq_algorithm { IMQ_ALG_FMM = 0, IMQ_ALG_TREECODE = 1 } imq_algorithm;

/* Precision of the translations (M2M, M2L, L2L) inside the FP32 product of
 * imq_matvec and of the CG inner iterations.  P2M, P2L, P2P, M2P and L2P stay
 * FP32 either way.
 *   FP32 : every kernel in FP32, M2L on the tensor cores (fastest).
 *   FP64 : the multipoles are widened after P2M and translated in FP64, the
 *          locals narrowed before L2P.  When the data make the far-field sums
 *          cancel (oscillating vectors, flat shapes), the FP32 rounding of the
 *          translated coefficients sets the error floor of the product
 *          (relative 2-norm error ~1e-6 at c ~ 0.15-0.2 on trig-sum vectors);
 *          FP64 translations remove that term at the cost of FP64 M2L.
 *   MIXED: M2M and L2L in FP64 (latency-bound levels, cheap on the FP64
 *          units), M2L on the tensor cores from the narrowed multipoles (FP32
 *          in and out): between the two in cost and error. */
typedef enum imq_translations { IMQ_TRANS_FP32 = 0, IMQ_TRANS_FP64 = 1, IMQ_TRANS_MIXED = 2 } imq_translations;

/* M2L kernel of the FP32 product.  AUTO takes the tensor cores when the
 * expansion fits them (K, K_out <= 256 reals), else the CUDA cores.
 * TENSOR fails the plan with IMQ_UNSUPPORTED when it does not fit. */
typedef enum imq_m2l_kernel {
    IMQ_M2L_AUTO = 0,
    IMQ_M2L_CUDA_CORES = 1,    /* register-tiled FP32 FMA                          */
    IMQ_M2L_TENSOR = 2         /* tcgen05 kind::f16, fp16 hi/lo split, TMEM accumulator */
} imq_m2l_kernel;

/* ------------------------------------------------------------------------- *
 * imq_plan -- build the quadtree, its interaction lists and the operators.
 *
 *   Section 2.2: the square D containing the points is partitioned into
 *   2^l x 2^l blocks; the adaptive tree here splits a block while it holds
 *   more than `leaf` points (and its depth is below IMQ_MAX_LEVEL).  The
 *   well-separated sets S_p become the V/W/X lists and the not-well-separated
 *   sets NS_p the U list.
 *
 *   points : double[N][2], host or device; read during the call only.
 *   N      : number of points, N >= 1.
 *   c      : shape parameter, c > 0 (finite).
 *   p      : truncation order of the expansions (the paper's M), 1 <= p <= IMQ_MAX_P.
 *   leaf   : maximum points per leaf box, leaf >= 1.
 *   opt    : may be NULL.
 *   out    : receives the plan (NULL on failure).
 *
 *   Synchronises `stream` (box counts are read back once per level).
 *   Errors: IMQ_INVALID_ARG, IMQ_DUPLICATE_POINTS, IMQ_UNSUPPORTED, IMQ_OOM,
 *   IMQ_CUDA_ERROR.
 * ------------------------------------------------------------------------- */
imq_status imq_plan(const double *points, int64_t N, double c, int p, int leaf,
                    const imq_options *opt, void *stream, imq_plan_t *out);

/* ------------------------------------------------------------------------- *
 * imq_plan_eval -- a plan for evaluating the interpolant of Eq. (2),
 * P(t) = sum_j coef_j phi(|t - x_j|), at off-node targets.  The tree is built
 * over nodes and targets together (node i is point i, target k is point
 * n_nodes + k), so the same fast product serves evaluation, its transpose and
 * the c-derivative (imq_evaluate*).  Arguments as imq_plan; targets may
 * coincide with nodes (check_duplicates must be 0).
 * ------------------------------------------------------------------------- */
imq_status imq_plan_eval(const double *nodes, int64_t n_nodes, const double *targets, int64_t n_targets,
                         double c, int p, int leaf, const imq_options *opt, void *stream,
                         imq_plan_t *out);

/* ------------------------------------------------------------------------- *
 * imq_plan_batched -- one plan for nprob independent problems (their own
 * points and shape c, one order p and leaf size), merged into one flattened
 * tree so that every phase of imq_matvec / imq_cg_solve is one launch over
 * all problems.  Problem b owns points [offsets[b], offsets[b+1]) of
 * `points` (double[N][2], host or device); offsets (int64[nprob+1], host,
 * offsets[0] = 0, strictly increasing) and cvals (double[nprob], host).
 * Vectors of the batched plan are [nrhs][N] in the same concatenated order;
 * the product is block diagonal (no interaction between problems).  The
 * problems share the square D (opt->has_domain, else the bounding square of
 * all points).  imq_matvec_dc and evaluation are not available on batched
 * plans (IMQ_UNSUPPORTED).  Errors as imq_plan.
 * ------------------------------------------------------------------------- */
imq_status imq_plan_batched(const double *points, const int64_t *offsets, int nprob, const double *cvals,
                            int p, int leaf, const imq_options *opt, void *stream, imq_plan_t *out);

/* Release every device allocation of the plan (after synchronising its work). */
void imq_plan_destroy(imq_plan_t plan);

/* ------------------------------------------------------------------------- *
 * imq_matvec -- b = A v by the fast method (Algorithm 1, generalised to the
 * translations of the fast multipole method; see the paper's Section 2.2).
 *
 *   v   : [nrhs][N] of dtype, host or device, in the caller's point order.
 *   out : [nrhs][N] of dtype, host or device, in the caller's point order.
 *   dt  : IMQ_F32 -- every kernel in FP32 except the FP64 operator set-up;
 *         IMQ_F64 -- every kernel in FP64.
 *   Streams: with device buffers the call only enqueues work.  The FP32
 *   product forks from `stream` onto two streams the plan owns (the far-field
 *   chain at the highest priority, P2L / P2P / M2P at the lowest) and joins
 *   them back into `stream` before its last kernel, so later work on `stream`
 *   is ordered after the product.  A plan serves one call at a time: calls on
 *   the same plan from several host threads, or on streams that overlap, must
 *   be serialised by the caller.  With host buffers the call synchronises.
 *   A kernel's bounded wait that ran out is reported by the next call that
 *   synchronises, or by imq_sync_check.
 *   Errors: IMQ_INVALID_ARG (nrhs < 1, NULL pointers), IMQ_OOM, IMQ_CUDA_ERROR,
 *   IMQ_TIMEOUT (host buffers only, see above).
 * ------------------------------------------------------------------------- */
imq_status imq_matvec(imq_plan_t plan, const void *v, void *out, int nrhs,
                      imq_dtype dt, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_matvec_dc -- b = (dA/dc) v, dA_ij/dc = -c / (|x_i - x_j|^2 + c^2)^{3/2}
 * (derivative of Eq. (5) in the shape parameter).  Under the lift of Eq. (11)
 * this is the vertical derivative of the Green's function at the targets, so
 * the same multipoles and tree serve (odd-parity locals, see dz.cu).
 * Arguments, layout and errors as imq_matvec.
 * ------------------------------------------------------------------------- */
imq_status imq_matvec_dc(imq_plan_t plan, const void *v, void *out, int nrhs,
                         imq_dtype dt, void *stream);

/* ------------------------------------------------------------------------- *
 * Evaluation on a plan from imq_plan_eval (Eq. (2)), E_kj = phi(|t_k - x_j|):
 *   imq_evaluate           out[r][k] = sum_j E_kj coef[r][j]      coef: [nrhs][n_nodes], out: [nrhs][n_targets]
 *   imq_evaluate_transpose out[r][j] = sum_k E_kj v[r][k]         v: [nrhs][n_targets],  out: [nrhs][n_nodes]
 *   imq_evaluate_dc        out[r][k] = sum_j dE_kj/dc coef[r][j]
 * Host or device buffers; errors as imq_matvec, and IMQ_INVALID_ARG for a plan
 * not made by imq_plan_eval.
 * ------------------------------------------------------------------------- */
imq_status imq_evaluate(imq_plan_t eplan, const void *coef, void *out, int nrhs, imq_dtype dt, void *stream);
imq_status imq_evaluate_transpose(imq_plan_t eplan, const void *v, void *out, int nrhs, imq_dtype dt,
                                  void *stream);
imq_status imq_evaluate_dc(imq_plan_t eplan, const void *coef, void *out, int nrhs, imq_dtype dt, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_matvec_timed -- imq_matvec with the kernels of each phase bracketed by
 * CUDA events recorded on `stream` (for benchmarks).  Synchronises `stream`.
 *
 *   phase_ms[k] (k < n_phases, host) receives the summed event time of phase k:
 *     0 gather  1 P2M  2 M2M  3 M2L  4 P2L  5 L2L  6 L2P+M2P  7 P2P  8 scatter.
 *   launches (host, may be NULL) receives the number of kernels launched.
 * ------------------------------------------------------------------------- */
#define IMQ_NUM_PHASES 9
imq_status imq_matvec_timed(imq_plan_t plan, const void *v, void *out, int nrhs,
                            imq_dtype dt, void *stream, float *phase_ms, int n_phases,
                            int32_t *launches);

/* ------------------------------------------------------------------------- *
 * imq_cg_solve -- solve A coef = f (Section 2, Eq. (3)-(4): the interpolant
 * reproduces the data at the nodes) by preconditioned conjugate gradients on
 * the fast product.  The paper names iterative methods as the solver whose
 * cost is the matrix-vector product (Section 2) and leaves the solver and a
 * preconditioner to future work (Section 4).
 *
 *   f    : double[nrhs][N], host or device, caller's point order.
 *   coef : double[nrhs][N], host or device; initial guess on entry when
 *          opt->x0_given, solution on exit (also on IMQ_NOT_CONVERGED: the
 *          iterate with the smallest recursive residual of the last pass).
 *   opt  : NULL for imq_cg_default_options().
 *   info : may be NULL; receives iterations, outer steps, the true relative
 *          residual ||f - A coef||_2 / ||f||_2 of each right-hand side
 *          (computed with the FP64 product selected by opt->residual), time.
 *
 *   Inner iterations run the FP32 fast product with FP64 vectors, dots and
 *   scalars, captured into a CUDA graph with a device-side convergence test.
 *   With refine_steps > 0 an outer loop recomputes r = f - A coef in FP64 and
 *   solves A d = r (iterative refinement).  Synchronises `stream`.
 *   Errors: IMQ_INVALID_ARG, IMQ_NOT_CONVERGED (tolerance not reached within
 *   maxit / refine_steps), IMQ_NUMERICAL (NaN/Inf or breakdown), IMQ_OOM,
 *   IMQ_CUDA_ERROR.
 * ------------------------------------------------------------------------- */
/* Preconditioners.  SCHWARZ: symmetric additive Schwarz over leaf neighbourhood
 * patches (each patch factored once, FP32 patches applied through their
 * explicit inverse).  SCHWARZ_2L: the same plus a Galerkin coarse space, one
 * indicator vector per coarse box (the largest tree boxes holding at most
 * coarse_points points), E = Z^T A Z assembled exactly over every pair and
 * inverted in FP64 once; applied in the deflated form z = y + Q (r - A y),
 * y the patch solves, Q = Z E^{-1} Z^T, each inner pass started from Q r.
 * One extra FP32 fast product per iteration; at most 16384 coarse boxes.  On a
 * batched plan the coarse boxes are each problem's own (E is block diagonal)
 * and the two-level preconditioner runs with GMRES only.  (Section 4 leaves the preconditioner to future work;
 * Section 1 cites preconditioned iterations.) */
typedef enum imq_precond { IMQ_PRECOND_NONE = 0, IMQ_PRECOND_SCHWARZ = 1, IMQ_PRECOND_SCHWARZ_2L = 2 } imq_precond;
typedef enum imq_operator {
    IMQ_OPERATOR_FAST_F32 = 0,   /* inner iterations on the FP32 fast product (default)   */
    IMQ_OPERATOR_FAST_F64 = 1,   /* inner iterations on the FP64 fast product              */
    IMQ_OPERATOR_DENSE_F64 = 2   /* inner iterations on the dense FP64 product (O(N^2))    */
} imq_operator;
typedef enum imq_residual {
    IMQ_RESIDUAL_PLAN_F64 = 0,   /* the fast product in FP64 (opt->residual_plan if given, else plan) */
    IMQ_RESIDUAL_DENSE_F64 = 1   /* the dense FP64 product (exact up to rounding, O(N^2))          */
} imq_residual;
/* Inner Krylov method.  CG: preconditioned conjugate gradients, graph-captured
 * (A is symmetric positive definite, Micchelli; the paper's Section 2 names
 * iterative solvers).  GMRES: right-preconditioned restarted GMRES(m) on the
 * same operator and preconditioner (Arnoldi vectors, Gram-Schmidt applied
 * twice and all dots in FP64; the small least-squares problem on the host).
 * GMRES minimises the residual norm over each cycle, so it keeps converging
 * where A is positive definite in exact arithmetic but not numerically (flat
 * shapes, c many times the point spacing), where CG's p.Ap or r.z loses its
 * sign and the pass ends.  Each cycle is one refinement pass.  On a batched
 * plan every problem has its own Arnoldi scalars, Hessenberg matrix and
 * convergence test; the vectors and the fast product are shared. */
typedef enum imq_krylov { IMQ_KRYLOV_CG = 0, IMQ_KRYLOV_GMRES = 1 } imq_krylov;
#define IMQ_CG_MAX_RHS_INFO 16

typedef struct imq_cg_options {
    int32_t struct_size;
    double rtol;             /* target of the true relative residual                         */
    int32_t maxit;           /* cap on the total number of inner iterations                   */
    int32_t precond;         /* imq_precond                                                    */
    int32_t schwarz_nmax;    /* max points per Schwarz patch, 1..224 (0: 224; 160 with FP64)   */
    double schwarz_shift;    /* patch diagonal shift, relative to A_ii = 1/c (FP32 patches: at
                                least 1e-6)                                                    */
    int32_t refine_steps;    /* outer refinement steps (0: one pass, then the true residual)   */
    double inner_rtol;       /* lower bound of the inner relative tolerance when refining      */
    int32_t residual;        /* imq_residual                                                   */
    int32_t x0_given;        /* 1: coef holds the initial guess                                */
    imq_plan_t residual_plan;/* optional plan on the same points (e.g. larger p), or NULL      */
    int32_t inner_operator;  /* imq_operator                                                   */
    int32_t schwarz_fp64;    /* 1: factor and apply the Schwarz patches in FP64 (nmax <= 160)   */
    int32_t coarse_points;   /* SCHWARZ_2L: max points per coarse box, 1..1024 (0: the leaf size) */
    int32_t coarse_gram;     /* SCHWARZ_2L: pairs of E = Z^T A Z in 0: FP64 if N^2 <= 4e10, else
                                FP32 with FP64 partial sums; 1: FP64; 2: FP32                   */
    int32_t krylov;          /* imq_krylov (batched plans: one Hessenberg matrix per problem)  */
    int32_t gmres_m;         /* GMRES restart length, 1..200 (0: 40); (m + 1) N doubles of basis */
    int32_t reserved[2];
} imq_cg_options;

typedef struct imq_cg_info {
    int32_t iterations;      /* inner iterations, summed over right-hand sides and outer steps */
    int32_t outer_steps;
    imq_status status;
    double max_rel_residual; /* max over right-hand sides of the true relative residual       */
    double seconds;          /* wall time of the solve (after preconditioner set-up)           */
    double rel_residual[IMQ_CG_MAX_RHS_INFO];
} imq_cg_info;

void imq_cg_default_options(imq_cg_options *opt);
imq_status imq_cg_solve(imq_plan_t plan, const double *f, double *coef, int nrhs,
                        const imq_cg_options *opt, imq_cg_info *info, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_cg_solve_batched -- imq_cg_solve on a plan from imq_plan_batched: the
 * nprob systems A_b coef_b = f_b (Section 2, Eq. (3)-(4), one per problem)
 * are solved together, one fast product over all problems per iteration,
 * with per-problem Krylov scalars (CG, or GMRES with opt->krylov) and
 * convergence tests.  imq_cg_solve on a batched plan does the same without
 * the per-problem outputs.
 *
 *   f, coef      : double[nrhs][N_total], problems in the plan's order.
 *   rel_residual : host double[nrhs][nprob] or NULL: true relative residual
 *                  ||f_b - A_b coef_b|| / ||f_b|| of each problem, computed with
 *                  the FP64 product opt->residual selects (the plan's fast
 *                  product, or the dense product of each problem with itself).
 *   iterations   : host int32[nrhs][nprob] or NULL: inner iterations of each
 *                  problem.
 *   info         : iterations = sum over right-hand sides of the largest
 *                  per-problem count; rel_residual[r] and max_rel_residual
 *                  are maxima over the problems.
 *   The dense inner operator and the dense residual are block diagonal: each
 *   problem's points only with each other (O(sum N_b^2) FP64 work).
 *   Errors: as imq_cg_solve; IMQ_INVALID_ARG if the plan is not batched;
 *   IMQ_UNSUPPORTED for residual_plan.
 * ------------------------------------------------------------------------- */
imq_status imq_cg_solve_batched(imq_plan_t plan, const double *f, double *coef, int nrhs,
                                const imq_cg_options *opt, imq_cg_info *info, double *rel_residual,
                                int32_t *iterations, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_interp_loss_grad -- validation loss of the interpolant (Eq. (2)) and its
 * gradient in the shape c and the data values f (adjoint method).
 *   coef = A^{-1} f (CG on `train`), P = E coef on `eval` (a plan from
 *   imq_plan_eval with the training points as nodes and the validation points
 *   as targets, same c), L = mean (P - y)^2, g = (2/N_v)(P - y),
 *   lambda = A^{-1} E^T g, dL/df = lambda, dL/dc = g.(dE/dc coef) - lambda.(dA/dc coef).
 *   f: double[N]; y: double[N_v]; host or device.  loss, dloss_dc: host scalars.
 *   dloss_df, coef_out: double[N] (host or device) or NULL.  dt selects the
 *   precision of the evaluation and derivative products; opt configures both
 *   solves.  info (may be NULL) sums both solves.  Errors: those of
 *   imq_cg_solve and imq_evaluate, IMQ_INVALID_ARG for mismatched plans.  On
 *   IMQ_NOT_CONVERGED every output is still written, from the best iterates.
 * ------------------------------------------------------------------------- */
imq_status imq_interp_loss_grad(imq_plan_t train, imq_plan_t eval, const double *f, const double *y,
                                const imq_cg_options *opt, imq_dtype dt, double *loss,
                                double *dloss_dc, double *dloss_df, double *coef_out,
                                imq_cg_info *info, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_dense_matvec -- the plain ("standard row-column") product of Section 3:
 * b_i = sum_j v_j / sqrt(|x_i - x_j|^2 + c^2) over all N^2 pairs, matrix-free.
 *
 *   points : double[N][2]; v, out : [nrhs][N] of dtype; all host or device.
 *   IMQ_F32: FP32 coordinates (cast from FP64), FP32 rsqrt, FP32 partial sums
 *            over source tiles accumulated in FP64.  IMQ_F64: all FP64.
 *   Errors: IMQ_INVALID_ARG, IMQ_OOM, IMQ_CUDA_ERROR.
 * ------------------------------------------------------------------------- */
imq_status imq_dense_matvec(const double *points, int64_t N, double c, const void *v,
                            void *out, int nrhs, imq_dtype dt, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_dense_matvec_noalloc -- the FP32 dense product of imq_dense_matvec for
 * callers that cannot allocate device memory.  (The paper has no counterpart:
 * this is an interface for such callers.)
 *
 *   Some callers cannot let a library call cudaMalloc or cudaMallocAsync:
 *   code running under a memory manager that owns all device memory and
 *   forbids allocations behind its back, or latency-critical loops that
 *   cannot afford an allocation's possible implicit synchronisation.  This
 *   entry point allocates nothing: its scratch (the packed source records and
 *   one error word) lives in a fixed device array of IMQ_NOALLOC_MAX_N + 1
 *   16-byte records (4 MiB + 16 B) inside the library, which every GPU that
 *   loads the library keeps until the process exits.
 *
 *   points : double[N][2]; v, out : float[N]; all DEVICE memory (host pointers
 *            are rejected, since staging them would need an allocation).
 *   N      : 1 <= N <= IMQ_NOALLOC_MAX_N; larger N fails with IMQ_INVALID_ARG.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and clears its error word; make that first call
 *   before any stream capture.  All calls share the one array, which keeps the
 *   previous call's contents (each call rewrites the records it uses): calls
 *   that overlap on the GPU race and must be serialised by the caller, e.g. on
 *   one stream.  Work is enqueued on `stream`; the call does not wait.
 *   A tile wait in the kernel is bounded; one that runs out sets the array's
 *   error word, which stays set until imq_sync_check reads and clears it
 *   (IMQ_TIMEOUT, `out` of the affected calls invalid).  imq_sync_check
 *   allocates nothing either.
 *   Errors: IMQ_INVALID_ARG, IMQ_UNSUPPORTED, IMQ_CUDA_ERROR.
 * ------------------------------------------------------------------------- */
#define IMQ_NOALLOC_MAX_N 262144
imq_status imq_dense_matvec_noalloc(const double *points, int64_t N, double c, const float *v,
                                    float *out, void *stream);

/* ------------------------------------------------------------------------- *
 * imq_autotune -- choose the truncation order p, the leaf size, the precision
 * of the translations and the tile shapes of the FP32 product.
 *
 *   The paper fixes M (= p) from the a-priori bound of Theorem 2.1 (worked
 *   example, Section 2.2) and the number of levels L by balancing the far-
 *   and near-field multiplication counts (Section 2.3).  Here everything is
 *   measured:
 *     1. for each leaf size in leaf_cand, the smallest p in p_cand whose FP32
 *        fast product meets `target` (relative 2-norm error on sampled rows,
 *        worst over problems and right-hand sides), then the fastest of those;
 *     2. if no candidate meets the target with FP32 translations, step 1 again
 *        with IMQ_TRANS_MIXED and then with IMQ_TRANS_FP64, whose error floors
 *        are lower;
 *     3. on the chosen (p, leaf, translations), the P2P tile shape (p2p_warps x
 *        p2p_chunk in {2, 4, 8} x {8, 16, 32}), then the tensor-core M2L
 *        pipeline depth (m2l_stages 4..6, as far as they fit) and the number
 *        of CTAs sharing an M2L tile (m2l_split 1..4): the fastest shape whose
 *        error still meets the target (else whose error does not grow by more
 *        than 1 %).
 *   If no candidate meets the target, the most accurate one is returned and
 *   met = 0.
 *
 *   points  : double[N][2], host or device, N = offsets[nprob].
 *   offsets : HOST int64[nprob + 1], offsets[0] = 0 (problem q owns points
 *             [offsets[q], offsets[q+1])); nprob = 1 tunes imq_plan, nprob > 1
 *             tunes imq_plan_batched.
 *   cvals   : HOST double[nprob], the shapes c.
 *   target  : > 0, e.g. 1e-6.
 *   p_cand  : HOST int32[n_p], 1 <= n_p <= 16, each in [1, IMQ_MAX_P].
 *   leaf_cand : HOST int32[n_leaf], 1 <= n_leaf <= 16, each >= 1.
 *   nrhs    : right-hand sides of the timed product, 1..16.
 *   opt     : plan options (domain, M2L kernel), may be NULL; its translations
 *             and tile fields are ignored (they are what is tuned).
 *   out     : HOST result; out->tried lists every configuration measured.
 *
 *   Sample: 2048 rows (single problem) or 32 rows per problem, evenly spaced
 *   in the caller's order; the test vectors are SplitMix64 values in [-1, 1)
 *   (imq_autotune_v: the caller's own);
 *   exact rows are FP64 direct sums.  The time of a configuration is the best
 *   of 3 products after one warm-up (CUDA events on `stream`).  Builds and
 *   frees one plan per configuration; synchronises `stream`.
 *   Errors: IMQ_INVALID_ARG, those of imq_plan / imq_plan_batched /
 *   imq_matvec.
 * ------------------------------------------------------------------------- */
#define IMQ_TUNE_MAX_TRIED 64
typedef struct imq_tune_entry {
    int32_t p, leaf;
    double rel_err;          /* sampled relative 2-norm error of the FP32 product */
    float matvec_ms;         /* best of the timed products                         */
    int32_t translations;    /* imq_translations                                   */
    int32_t p2p_warps, p2p_chunk, m2l_stages, m2l_split;   /* tile shape (0: default) */
} imq_tune_entry;

typedef struct imq_tune_result {
    int32_t p, leaf;         /* the choice                                         */
    double rel_err;
    float matvec_ms;
    int32_t met;             /* 1 if rel_err <= target                             */
    int32_t n_tried;
    int32_t sampled_rows;
    int32_t translations;    /* the choice's imq_translations                      */
    int32_t p2p_warps, p2p_chunk, m2l_stages, m2l_split;   /* the choice's tile shape */
    int32_t reserved;
    imq_tune_entry tried[IMQ_TUNE_MAX_TRIED];
} imq_tune_result;

imq_status imq_autotune(const double *points, const int64_t *offsets, int nprob, const double *cvals,
                        double target, const int32_t *p_cand, int n_p, const int32_t *leaf_cand,
                        int n_leaf, int nrhs, const imq_options *opt, void *stream,
                        imq_tune_result *out);

/* imq_autotune_v -- imq_autotune with the caller's test vectors instead of
 * SplitMix64 values: v is float[nrhs][N] in the caller's point order, host or
 * device.  Data whose far-field sums cancel (oscillating right-hand sides, flat
 * shapes) have a larger relative error than random vectors at the same p and
 * translations; tuning on representative vectors makes `met` hold for them.
 * Errors: as imq_autotune; IMQ_INVALID_ARG for v == NULL.  (Section 2.3 as for
 * imq_autotune.) */
imq_status imq_autotune_v(const double *points, const int64_t *offsets, int nprob, const double *cvals,
                          double target, const int32_t *p_cand, int n_p, const int32_t *leaf_cand,
                          int n_leaf, int nrhs, const float *v, const imq_options *opt, void *stream,
                          imq_tune_result *out);

/* ------------------------------------------------------------------------- *
 * imq_sync_check -- synchronise `stream` and report a failed bounded wait.
 *
 *   The kernels that wait on shared-memory barriers (the tensor-core M2L
 *   pipeline, the P2P source staging, the M2M/L2L operator copy, the Schwarz
 *   patches' factor copy, the dense product's source tiles) give up after a
 *   bounded number of polls or 0.5 s
 *   instead of hanging, and record that in a per-device error word (the
 *   allocation-free dense product in the word of its own scratch array).
 *   Calls that synchronise anyway (host output buffers, imq_matvec_timed,
 *   imq_cg_solve, imq_dense_matvec) check it themselves; after asynchronous
 *   imq_matvec or imq_dense_matvec_noalloc calls on device buffers, call this
 *   before using the results.  Reads and clears both words; allocates no
 *   device memory.  (Not an operation of the paper.)
 *   Errors: IMQ_TIMEOUT (a wait ran out since the last check: the results of
 *   the products in between are invalid), IMQ_CUDA_ERROR.
 * ------------------------------------------------------------------------- */
imq_status imq_sync_check(void *stream);

/* imq_selftest_wait_timeout -- exercise the bounded-wait path: one kernel waits
 * on a shared-memory barrier that nothing ever completes, gives up after the
 * wait limit (0.5 s), records the timeout in the error word, and this call
 * reads it back (as imq_sync_check does).  Returns IMQ_TIMEOUT when the path
 * works; the context stays usable.  (Not an operation of the paper.) */
imq_status imq_selftest_wait_timeout(void *stream);

/* ------------------------------------------------------------------------- *
 * Introspection of a plan, for tests and benchmarks.
 * ------------------------------------------------------------------------- */
typedef struct imq_plan_info {
    int64_t n_points;
    int64_t n_nodes;                     /* evaluation plans: nodes among n_points (else 0) */
    int32_t n_problems;                  /* batched plans: independent problems (else 1)     */
    int32_t algorithm;                   /* imq_algorithm of the plan                        */
    int32_t n_boxes, n_leaves, max_level, p, leaf, k_real;  /* k_real: reals per expansion */
    double x0, y0, side, c;
    int64_t n_u, n_v, n_w, n_x;          /* total entries of each interaction list */
    int64_t p2p_pairs;                   /* sum over leaves of n_target * n_source in U */
    int64_t m2l_pairs;                   /* V-list entries on levels >= 2 */
    int64_t device_bytes;                /* device memory owned by the plan */
} imq_plan_info;

imq_status imq_plan_get_info(imq_plan_t plan, imq_plan_info *info);

/* Copy the tree to HOST buffers (each may be NULL to skip it):
 *   codes[N]   uint32 Morton codes in sorted order;  perm[N] int64 sorted->input index;
 *   level, prefix, begin, end, parent : [n_boxes];   child : [n_boxes][4] (-1 absent). */
imq_status imq_plan_export_tree(imq_plan_t plan, uint32_t *codes, int64_t *perm,
                                int32_t *level, uint32_t *prefix, int64_t *begin,
                                int64_t *end, int32_t *parent, int32_t *child);

/* Copy one interaction list in CSR form to HOST buffers.
 *   which  : 'U', 'V', 'W' or 'X'.
 *   offsets: int32[n_boxes + 1]; items: int32[offsets[n_boxes]] (box numbers, sorted
 *            ascending within each box).  Either may be NULL. */
imq_status imq_plan_export_list(imq_plan_t plan, char which, int32_t *offsets, int32_t *items);

/* Human-readable name of a status code (static string). */
const char *imq_status_string(imq_status s);

/* Message of the last failing call on this thread ("" if none). */
const char *imq_last_error(void);

/* Library version string. */
const char *imq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IMQ_H */
