/*
 * csl.h -- C ABI of the GB300 solver for complex-shifted Laplacian systems
 *
 *     (K + lambda I) z = f,   lambda = alpha + i beta            (Eq. 1)
 *
 * where K is the conservative finite-difference discretisation of
 * -div(a grad .) on the unit square (5-point) or cube (7-point) with
 * homogeneous Dirichlet boundary values and n_d interior points per axis
 * (h_d = 1/(n_d+1)).  The solve is preconditioned MINRES on the equivalent
 * 2x2 block real system (Eq. 2)
 *
 *     A = [[beta I, K + alpha I], [K + alpha I, -beta I]],  A [z1; z2] = [Im f; Re f],
 *
 * with z = z1 + i z2, and the absolute-value preconditioner of Eq. 4
 *
 *     P = blkdiag(sqrt((gamma L + alpha I)^2 + beta^2 I), same),  gamma = sqrt(a_min a_max),
 *
 * applied through the sine transform that diagonalises the constant-coefficient
 * Laplacian L (Section 2.3).  When a is constant, P is |A| (Eq. 3).
 *
 * Conventions shared by every entry point
 *  - Grids: dim = 2 or 3; n[0], n[1], n[2] are the interior point counts along
 *    x, y, z (n[2] ignored for dim = 2).  Every n[d] + 1 must be a power of two
 *    between 4 and 1024; 2D grids may reach 16384 in FP64 and 4096 in the
 *    FP32 / BF16 precisions, the sizes of the paper's larger tables (else
 *    CSL_UNSUPPORTED_SIZE).
 *  - Grid vectors are C-order arrays with x fastest: point (ix, iy[, iz]) at
 *    index ix + n[0]*(iy + n[1]*iz).  "complex128" vectors hold interleaved
 *    (re, im) doubles; "block-pair" vectors hold (block-1, block-2) doubles of
 *    the block system interleaved the same way.
 *  - Coefficient samples: coef_faces[0] are the x-faces, shape
 *    ([n2,] n1, n0+1), entry i along x being the face between grid indices
 *    i-1 and i (at x = (i + 1/2) h_x); coef_faces[1] the y-faces
 *    ([n2,] n1+1, n0); coef_faces[2] the z-faces (n2+1, n1, n0).  All > 0.
 *  - Pointers are DEVICE pointers owned by the caller unless the name ends in
 *    _host.  A plan owns its own workspace and copies the coefficients; the
 *    caller may free them after csl_plan_create returns.
 *  - All work runs on the plan's CUDA stream (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  Calls that return a csl_solve_info
 *    synchronise that stream; the others are stream-ordered and asynchronous.
 *  - Nothing throws across the ABI: every call returns a csl_status.
 */
#ifndef CSL_H
#define CSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum csl_status {
  CSL_OK = 0,
  CSL_INVALID_ARG = 1,       /* null pointer, dim not 2/3, n < 1, non-finite shift, coefficient <= 0;
                                FP32 / BF16 forms: per-mode scales of P^-1 outside the FP32 range */
  CSL_UNSUPPORTED_SIZE = 2,  /* n[d] + 1 not a power of two in the ranges above */
  CSL_SINGULAR_PRECOND = 3,  /* some (gamma mu_k + alpha)^2 + beta^2 == 0 (only possible when beta == 0) */
  CSL_BREAKDOWN = 4,         /* non-finite or negative <P^{-1} v, v> in the Lanczos process */
  CSL_NOT_CONVERGED = 5,     /* maxit reached; z holds the last iterate, info is filled */
  CSL_TIMEOUT = 6,           /* a bounded device wait expired */
  CSL_CUDA_ERROR = 7,        /* a CUDA runtime call failed */
  CSL_OUT_OF_MEMORY = 8
} csl_status;

typedef enum csl_precision {
  CSL_PREC_FP64 = 0,  /* every step in FP64 (the plain method)                          */
  CSL_PREC_FP32 = 1,  /* sine transforms and per-mode scale of P^{-1} in FP32; the
                         per-point vector work (stencil, Lanczos step, w/x update) in
                         float-pair arithmetic (about 2^-47 relative); Lanczos and Givens
                         scalars, reductions and the true-residual check in FP64; the
                         solution is returned in FP64 */
  CSL_PREC_BF16X3 = 2, /* as CSL_PREC_FP32, but the transforms along y and z (lines of
                          n+1 = 32, 64 or 128 points) run on the tensor cores as GEMMs with
                          the sine matrix of Section 2.3: operands split into two bf16 terms,
                          3 products accumulated in FP32 (relative error about 1e-5).
                          The paper has no such form (it ran FP64 throughout). */
  CSL_PREC_BF16X6 = 3, /* as CSL_PREC_BF16X3 with three bf16 terms and 6 products
                          (about FP32 accuracy) */
  CSL_PREC_FP32_PRECOND = 4 /* FP32 only inside P^{-1} (sine transforms and per-mode
                          scale); the stencil (matvec), the Lanczos vectors and step,
                          the w/x update, the Givens rotations, the reductions and the
                          true-residual check in FP64, as in CSL_PREC_FP64.  z = P^{-1} v
                          is kept in FP32, the precision it is computed in */
} csl_precision;

typedef struct csl_plan_options {
  int precision;          /* csl_precision, default CSL_PREC_FP64                          */
  double gamma_override;  /* > 0: use this gamma in P; otherwise sqrt(min a * max a) (Eq. 4) */
  int lines_per_cta;      /* sine-transform lines per CTA for the strided passes; 0 = tuned */
  int use_graph;          /* 1 (default): the iteration loop runs as a CUDA graph with a
                             device-controlled WHILE node; 0: host-driven loop              */
  int autotune;           /* 1 (default): time the candidate CTA shapes and transform
                             variants of each pass at plan creation and keep the fastest
                             (cached per shape for the process); 0: built-in defaults      */
  int programmatic_launch; /* 1 (default): the iteration's kernels are launched with
                             programmatic dependent launch, so each may start (tables,
                             set-up) while its predecessor drains; 0: plain launches       */
  int float_pair_stencil;  /* FP32 / BF16X3 / BF16X6 only. 1 (default): the stencil forms
                             (K + alpha I) z in float-pair arithmetic in difference form
                             (used while every face a/h^2, alpha and beta lie in
                             [2^-60, 2^60]); 0: FP64 arithmetic, direct form               */
  int update_mode;         /* where the MINRES w/x update of an iteration runs: 0 (default) or
                             1: its own kernel on a side branch beside the inverse x transform;
                             2: fused into the inverse x transform; 3: its own kernel after
                             the inverse x transform (batches always fuse)                  */
  int body_iters;          /* MINRES iterations per body of the CUDA graph's WHILE loop: 0
                             (default) = 2, else 2, 4 or 8 (more amortise the loop's
                             per-body cost; up to body_iters - 1 iterations after
                             convergence then exit at entry)                              */
  int warm_start;          /* 1: csl_solve / csl_adjoint / csl_solve_host read their output
                             vector z (y) on entry as the initial guess x_0 and run MINRES on
                             the correction (r_0 = f - (K + lambda I) x_0); the stopping
                             test stays relative to ||f||.  0 (default): x_0 = 0.  Single
                             plans only (csl_batch_create refuses it)                     */
  int history;             /* > 0: record the MINRES residual estimate |eta_j| / |eta_0|
                             (P^{-1}-norm, non-increasing) of up to `history` iterations;
                             read with csl_solve_history.  0 (default): none             */
  int reserved[1];
} csl_plan_options;

typedef struct csl_solve_info {
  int iters;          /* MINRES iterations = products with A in the loop ("Iter", Section 3) */
  int status;         /* csl_status of the solve                                             */
  double relres;      /* true ||f - (K + lambda I) z||_2 / ||f||_2 of the returned z          */
  double pnorm;       /* |eta|: the P^{-1}-norm residual estimate of MINRES at exit           */
  double gamma;       /* gamma used by P                                                      */
  int checks;         /* explicit true-residual evaluations performed                         */
  int launches;       /* kernels this library launched for the solve                           */
  int reserved[6];
} csl_solve_info;

typedef struct csl_plan csl_plan;

/* Library version string and status names (static storage, never NULL). */
const char* csl_version(void);
const char* csl_status_string(csl_status s);

/* Description of the last CUDA failure seen by this thread ("" if none). */
const char* csl_last_error(void);

/* Fill *opt with the defaults above. */
csl_status csl_plan_options_init(csl_plan_options* opt);

/*
 * Build a plan for one grid, one coefficient field and one shift
 * (Eq. 1, Eq. 4, Section 2.3): scales and copies the face samples, forms the
 * stencil diagonal, gamma = sqrt(a_min a_max), the per-axis Laplacian
 * eigenvalues mu_k = (4/h^2) sin^2(k pi / (2(n+1))), the per-mode scale of
 * P^{-1}, the FFT twiddles, and allocates the MINRES workspace
 * (about 10 vectors of 16 bytes per grid point).
 * coef_faces: `dim` device pointers (layout above).  opt may be NULL.
 * On success *out owns device memory until csl_plan_destroy.
 */
csl_status csl_plan_create(csl_plan** out, int dim, const int64_t n[3],
                           const double* const coef_faces[3], double alpha, double beta,
                           const csl_plan_options* opt, void* stream);
void csl_plan_destroy(csl_plan* plan);

/* Change the stream later calls run on. */
csl_status csl_plan_set_stream(csl_plan* plan, void* stream);

/*
 * All-at-once time solve (the setting Section 1 gives for the shifted
 * systems; a growth row of this library, not an algorithm of the paper).
 * Backward Euler for u' + K u = g on L steps of size tau,
 *     (B kron I + I kron K) U = F,  B = (I - S)/tau (S: ones on the subdiagonal),
 *     F_0 = g_0 + u0/tau,  F_n = g_n,
 * solved by preconditioned Richardson U <- U + P_a^{-1} (F - A U), U_0 = 0,
 * with the alpha-circulant P_a = C_a kron I + I kron K, C_a = (I - S_a)/tau
 * (S with a in its top-right corner).  P_a^{-1} is a DFT in time of the
 * slices scaled by a^{j/L}, the L complex-shifted solves
 * (d_k I + K) Z_k = R_k, d_k = (1 - a^{1/L} e^{-2 pi i k/L}) / tau, in one
 * batch (csl_batch_*), and the inverse DFT scaled by a^{-j/L}.  The sweep
 * count falls roughly like a^s.
 *
 * L must be a power of two in [2, 1024] (else CSL_UNSUPPORTED_SIZE), 0 < a < 1,
 * tau > 0.  Slices are stored slice-major (slice j of point p at j*M + p),
 * complex128, DEVICE pointers: u0 has M entries, g and u have L*M.  opt (may
 * be NULL) applies to the L shifted solves.  Stream-ordered on `stream`; the
 * solve synchronises it once per sweep (to read the residual norm).
 */
typedef struct csl_paradiag csl_paradiag;
typedef struct csl_paradiag_info {
  int sweeps;           /* P_a^{-1} applications                                     */
  int status;           /* CSL_OK when relres <= tol, else CSL_NOT_CONVERGED / error */
  double relres;        /* ||F - A U||_2 / ||F||_2 of the returned U                  */
  int inner_iters_max;  /* largest MINRES iteration count among the shifted solves    */
  int reserved[5];
} csl_paradiag_info;

csl_status csl_paradiag_create(csl_paradiag** out, int dim, const int64_t n[3], const double* const coef_faces[3],
                               int L, double tau, double a, const csl_plan_options* opt, void* stream);
csl_status csl_paradiag_solve(csl_paradiag* pd, const double* u0, const double* g, double* u, double tol,
                              int maxit, double inner_tol, int inner_maxit, csl_paradiag_info* info);
void csl_paradiag_destroy(csl_paradiag* pd);

/*
 * The shifted system as a preconditioner (Section 1: the complex-shifted
 * Laplacian was introduced as the "shifted Laplace" preconditioner of
 * Helmholtz problems; a growth row of this library, not an algorithm of the
 * paper).  Restarted flexible GMRES for (K + lam_A I) u = f (e.g. lam_A = -k^2),
 * right-preconditioned by z = M^{-1} v with M = K + lam_M I (e.g.
 * lam_M = -k^2 (1 - 0.5 i)), each application one csl_solve to the relative
 * residual inner_tol (inexact solves are allowed: the flexible variant keeps
 * the preconditioned vectors).  restart in [1, 200]; lam_M must give a
 * nonsingular P (as csl_plan_create).  f, u: complex128 DEVICE vectors of M
 * entries.  Stops when ||f - (K + lam_A I) u|| <= tol ||f|| (true residual,
 * checked at every restart) or after maxit Arnoldi steps; u = 0 initially.
 * Synchronises the stream at every Arnoldi step.
 */
typedef struct csl_helmholtz csl_helmholtz;
typedef struct csl_helmholtz_info {
  int iters;              /* Arnoldi steps (preconditioner applications)      */
  int status;             /* CSL_OK when relres <= tol, else NOT_CONVERGED / error */
  double relres;          /* true ||f - (K + lam_A I) u|| / ||f|| of the result */
  int inner_iters_total;  /* MINRES iterations summed over the inner solves    */
  int restarts;
  int reserved[4];
} csl_helmholtz_info;

csl_status csl_helmholtz_create(csl_helmholtz** out, int dim, const int64_t n[3], const double* const coef_faces[3],
                                double lam_re, double lam_im, double shift_re, double shift_im, int restart,
                                const csl_plan_options* opt, void* stream);
csl_status csl_helmholtz_solve(csl_helmholtz* h, const double* f, double* u, double tol, int maxit,
                               double inner_tol, int inner_maxit, csl_helmholtz_info* info);
void csl_helmholtz_destroy(csl_helmholtz* h);

/* Device bytes owned by the plan. */
size_t csl_plan_workspace_bytes(const csl_plan* plan);

/* Human-readable launch configuration the plan chose (autotuned or default). */
const char* csl_plan_config(const csl_plan* plan);

/*
 * The autotuner's cache (not part of the method).  Plans tune each sine-
 * transform pass by timing its candidate shapes and keep the result per
 * process.  csl_tune_cache_save writes every shape tuned so far to the text
 * file `path`; csl_tune_cache_load merges the shapes of such a file into the
 * cache, so that plans created later in this process take them without
 * timing (e.g. a profiled process runs the shapes a benchmark chose).
 * Loading checks every entry and loads nothing from a malformed file.
 * Returns CSL_INVALID_ARG (message in csl_last_error()) when the file cannot
 * be opened, written or parsed.
 */
csl_status csl_tune_cache_save(const char* path);
csl_status csl_tune_cache_load(const char* path);

/* gamma actually used by P (Eq. 4). */
double csl_plan_gamma(const csl_plan* plan);

/*
 * out = (K + lambda I) z for complex128 z, out (M entries each); Eq. 1's
 * operator, evaluated by the same stencil kernel the solver uses.  z and out
 * must not overlap.
 */
csl_status csl_apply(csl_plan* plan, const double* z, double* out);

/*
 * out = P^{-1} v for block-pair vectors (Eq. 4 via Section 2.3): each of the
 * two interleaved blocks goes through the sine transform, the per-mode scale
 * 1/sqrt((gamma mu + alpha)^2 + beta^2) and the inverse transform, in the
 * plan's precision.  Because P acts identically on both blocks, a complex128
 * vector may be passed as well.  v and out may be the same buffer.
 */
csl_status csl_precondition(csl_plan* plan, const double* v, double* out);

/*
 * Solve (K + lambda I) z = f (Eq. 1) by preconditioned MINRES on Eq. 2 with P
 * (Eq. 4), zero initial guess (or z's contents with the warm_start option),
 * until the true relative residual is <= tol or maxit iterations.  f, z: complex128, M entries, may not overlap.  info may
 * be NULL.  Returns CSL_OK, CSL_NOT_CONVERGED (z = last iterate),
 * CSL_BREAKDOWN, or an argument/CUDA error.  Synchronises the plan's stream.
 */
csl_status csl_solve(csl_plan* plan, const double* f, double* z, double tol, int maxit,
                     csl_solve_info* info);

/*
 * The residual history of the plan's last solve (plan option `history`):
 * copies min(iterations, history, cap) values |eta_j| / |eta_0| (j = 1, 2,
 * ...) to out_host and their number to *count.  Synchronises the stream.
 * CSL_INVALID_ARG when the plan records no history.
 */
csl_status csl_solve_history(csl_plan* plan, double* out_host, int cap, int* count);

/*
 * The same solve with HOST buffers: f_host is copied to the device, solved,
 * and z copied back to z_host (pinned host memory gives full copy speed).
 */
csl_status csl_solve_host(csl_plan* plan, const double* f_host, double* z_host, double tol,
                          int maxit, csl_solve_info* info);

/*
 * Adjoint solve (K + conj(lambda) I) y = g: the same preconditioned MINRES on
 * the block system with beta -> -beta (A is symmetric, so this is the
 * transposed system of Eq. 2 expressed in complex form; P is unchanged).
 * With g = dL/dRe z + i dL/dIm z this gives y = dL/dRe f + i dL/dIm f.
 */
csl_status csl_adjoint(csl_plan* plan, const double* g, double* y, double tol, int maxit,
                       csl_solve_info* info);

/*
 * Gradient of a loss with respect to the coefficient samples, given the
 * solution z and the adjoint y (both complex128):
 *   dL/da_e = -h_d^{-2} Re(conj(y_p - y_q) (z_p - z_q))
 * for the face e between grid points p and q along axis d (values outside the
 * grid are 0).  grad_faces[d] has the layout of coef_faces[d].  Derived from
 * Eq. 2 by differentiating A x = r (the paper has no gradient).
 */
csl_status csl_coef_grad(csl_plan* plan, const double* z, const double* y,
                         double* const grad_faces[3]);

/*
 * Batched solves (many shifts lambda_k, e.g. from an alpha-circulant time
 * discretisation, and grids of different sizes): one plan per system, all
 * systems of one grid size advanced together by the same kernels (a device
 * array of per-system arguments per launch), the size groups on parallel
 * branches of one CUDA graph whose WHILE node is closed once every system
 * has met its own stopping test.  Converged systems stop costing work.
 */
typedef struct csl_system_desc {
  int dim;                           /* 2 or 3 (the same for all systems of a batch) */
  int64_t n[3];                      /* grid, as for csl_plan_create                 */
  const double* coef_faces[3];       /* device pointers, as for csl_plan_create       */
  double alpha, beta;                /* lambda = alpha + i beta                        */
} csl_system_desc;

typedef struct csl_batch csl_batch;

/* Build a batch of nsys systems (opt applies to all; opt may be NULL). */
csl_status csl_batch_create(csl_batch** out, int nsys, const csl_system_desc* sys,
                            const csl_plan_options* opt, void* stream);

/*
 * Solve every system: f[i], z[i] are device complex128 pointers (host arrays
 * of nsys pointers).  infos (nsys entries) may be NULL.  Returns CSL_OK if
 * every system converged, else the first non-OK system status.  Synchronises
 * the batch's stream.
 */
csl_status csl_batch_solve(csl_batch* batch, const double* const* f, double* const* z, double tol, int maxit,
                           csl_solve_info* infos);
void csl_batch_destroy(csl_batch* batch);
size_t csl_batch_workspace_bytes(const csl_batch* batch);

/*
 * Allocation-free P^{-1} v (the paper has no counterpart; a deployment
 * convenience).  Same result as csl_precondition on a plan built with the
 * same grid, gamma, alpha, beta and precision, but without a plan and without
 * allocating device memory: for callers that cannot call cudaMalloc, such as
 * a runtime whose memory pool owns all device memory or a fixed-budget
 * embedded service.
 *   dim, n[3]   grid (n[d] + 1 a power of two in [4, 1024]); at most 262144
 *               grid points (e.g. 511 x 511, 63 x 63 x 63), else
 *               CSL_UNSUPPORTED_SIZE with a message in csl_last_error()
 *   gamma       the averaged coefficient, as csl_plan_create computes it (> 0);
 *               alpha, beta: lambda
 *   precision   CSL_PREC_FP64 or CSL_PREC_FP32 (as csl_plan_options.precision)
 *   v, out      device block-pair (or complex128) vectors of the grid; may alias
 *   stream      cudaStream_t as void*; the call is stream-ordered, asynchronous
 * Returns CSL_SINGULAR_PRECOND when (gamma mu + alpha)^2 + beta^2 vanishes
 * for some mode (to within rounding; only possible for beta = 0) and, for
 * CSL_PREC_FP32, CSL_INVALID_ARG when the per-mode scales leave the FP32
 * range, as csl_plan_create does; both are decided on the host before any
 * launch.  Scratch (about 6 MiB) lives in static device arrays of the
 * library, held by every GPU that loads it until the process exits and
 * shared by all calls: calls that overlap on the GPU race and must be
 * serialised by the caller.  Every call rewrites all the scratch it reads.
 * The first call on a device performs a one-time set-up: it looks up the
 * arrays' device addresses (cudaGetSymbolAddress) with that device current.
 */
csl_status csl_precondition_static(int dim, const int64_t n[3], double gamma, double alpha, double beta,
                                   int precision, const double* v, double* out, void* stream);

/*
 * Measurement hook (not part of the method): time each kernel of the MINRES
 * iteration with CUDA events on the plan's stream.  The iteration's kernel
 * sequence runs `reps` (1..1000) times in a row, after one untimed
 * iteration, with an event between consecutive kernels (the w/x update
 * after the inverse x transform), so that each kernel is timed after its
 * real predecessor with the caches as the iteration leaves them.  The
 * kernels run on a scratch copy of the solver state and the vectors the last
 * call left (run a solve first); the solver's own state is untouched.  On
 * return ms[i] is the mean duration of kernel i and names[i] its name, for
 * i < *count (<= 8).  Synchronises the stream.
 */
csl_status csl_time_kernels(csl_plan* plan, int reps, double ms[8], const char* names[8], int* count);

#ifdef __cplusplus
}
#endif
#endif /* CSL_H */
