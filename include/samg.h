/*
 * samg.h -- C ABI of the GB300 (sm_103a) solver for a few extremal singular
 * triplets of a sparse rectangular matrix, or eigenpairs of an SPD matrix, by
 * the self-learning algebraic multigrid method of H. De Sterck,
 * "A Self-learning Algebraic Multigrid Method for Extremal Singular Triplets
 * and Eigenpairs" (arXiv:1102.0919).
 *
 * The library runs the multiplicative setup phase (Sec. 3) and the additive
 * solve phase -- V-cycles with fixed interpolation (Secs. 4.1-4.2) plus the
 * Ritz step (Sec. 4.3) -- on one GPU.  All arithmetic of the solve phase runs
 * in the library's CUDA kernels; there is no CPU fallback: every entry point
 * that computes returns SAMG_E_CUDA when no usable sm_103a device is present.
 * Argument checks come first (SAMG_E_INVALID on any machine), and the entry
 * points marked "host only" below (setup steps, schedule analysis, hierarchy
 * files) need no GPU.
 *
 * Conventions for every entry point:
 *  - Host matrices are 0-based CSR with int64 row pointers, int32 sorted
 *    column indices and float64 values.  The library copies what it needs;
 *    the caller keeps ownership of every pointer it passes.
 *  - Host vector blocks are row-major: entry i of vector j of an m-row block
 *    is X[i * n_b + j] (a C-contiguous numpy array of shape (m, n_b)).
 *  - Device pointers appear only where an argument says "device".
 *  - A context is used by one host thread at a time.  All GPU work runs on
 *    the CUDA stream passed at creation (NULL = the legacy default stream).
 *  - No C++ exception crosses this interface.  A failing call returns a
 *    status; samg_last_error(ctx) then holds a message.  After SAMG_E_TIMEOUT
 *    or SAMG_E_CUDA the context is poisoned: only samg_destroy is valid.
 */
#ifndef SAMG_H
#define SAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct samg_ctx samg_ctx; /* opaque; owns all device memory it uses */

typedef enum {
    SAMG_OK = 0,
    SAMG_E_INVALID = 1,       /* bad argument, malformed CSR, sizes out of range */
    SAMG_E_NOMEM = 2,         /* device or host allocation failed */
    SAMG_E_CUDA = 3,          /* CUDA error or no sm_103a device */
    SAMG_E_NT_TOO_SMALL = 4,  /* too few test vectors for the LS fits (Sec. 3.8) */
    SAMG_E_NOT_CONVERGED = 5, /* max_outer reached before the tolerance */
    SAMG_E_TIMEOUT = 6        /* a device-side wait gave up (bounded spin) */
} samg_status;

/* dominant: largest singular values (Secs. 3-4); minimal: smallest (Sec. 5.3) */
typedef enum { SAMG_DOMINANT = 0, SAMG_MINIMAL = 1 } samg_target;

/* SVD of a rectangular A, or eigenpairs of an SPD A (Sec. 5.2: operators A, B, P) */
typedef enum { SAMG_SVD = 0, SAMG_SPD_EIG = 1 } samg_kind;

/* Arithmetic of the V-cycle.  FP64: everything in float64.  FP32: relaxation,
 * residual, transfers and coarse levels in float32 on the defect (error)
 * equation, with the finest-level residual, the correction, the coarsest
 * solve and the Ritz step in float64.  BF16_STORE (a variant, not in the
 * paper): as FP32, but the V-cycle's vector blocks are stored in HBM as
 * bfloat16 (8-bit mantissa) and converted to float32 on load; matrix
 * coefficients and all arithmetic stay float32, and the float64 residual and
 * Ritz step of every outer iteration recover the accuracy. */
typedef enum { SAMG_FP64 = 0, SAMG_FP32 = 1, SAMG_BF16_STORE = 2 } samg_precision;

typedef struct {
    int32_t m, n;            /* rows, columns */
    int64_t nnz;
    const int64_t *row_ptr;  /* host, m + 1 entries, row_ptr[0] = 0 */
    const int32_t *col;      /* host, nnz entries, sorted within each row */
    const double *val;       /* host, nnz entries */
} samg_csr;

typedef struct {
    int32_t n_t;          /* random test vectors (Sec. 3.3); <= 16 */
    double theta;         /* strength parameter, Eq. strength */
    int32_t mu_t, mu_b;   /* relaxations of test / boot vectors per level */
    int32_t mu_tJ, mu_bJ; /* inner weighted-Jacobi steps (dominant); 1 */
    double omega_J;       /* Jacobi weight; 0.7 */
    int32_t n_mult;       /* multiplicative (setup) cycles */
    int32_t coarsest_max; /* coarsest level when max(m_l, n_l) <= this */
    int32_t max_levels;
    uint64_t seed;        /* SplitMix64 seed of the random test vectors */
    samg_precision prec;  /* arithmetic of the solve-phase V-cycle */
    int32_t n_conv;       /* triplets that must meet samg_solve's tolerance:
                             the first n_conv (0 = all n_b); the others are
                             guards that keep the block complete past a small
                             gap (not in the paper) */
    int32_t coarse_pinv;  /* coarsest additive solve (Sec. 4.2):
                             0 = the paper's form, the SVD pseudo-inverse of
                               X_L - s_j Y_L without its smallest singular
                               value;
                             1 = a variant (not in the paper): with the
                               generalized eigenpairs X_L w_k = lam_k Y_L w_k,
                               W^t Y_L W = I (once per hierarchy),
                               z = sum over k != k* of w_k (w_k^t r) /
                               (lam_k - s_j), k* the lam_k nearest s_j (ties:
                               the lowest k).  It equals form 0 when Y_L = I
                               and costs two passes over W per cycle, so it
                               suits large coarsest levels. */
    int32_t row_form;     /* minimal SVD kind with m >= n (Sec. 3.7):
                             0 = rows coarsened directly from A (a reading of
                               the option Sec. 3.7 leaves open): P_0 = A Q_0,
                               P_l = Q_l below level 0, and the Ritz step of
                               Sec. 4.3 takes the left basis A V_b;
                             1 = the paper's form: rows coarsened on A A^t
                               with their own LS-fitted P, two-sided Ritz
                               on span(U_b) x span(V_b).  On the gradient
                               workloads form 1 collapses onto the
                               null(A^t) zero modes of Thm genSVD.
                             Ignored by the other kinds. */
    int32_t relax_order;  /* order of the solve phase's Kaczmarz sweeps
                             (minimal target; Sec. 5.3, R3):
                             0 = the paper's natural row order, run exactly
                               (dependency levels, bands, cross-band waits);
                             1 = a coloured variant (not in the paper): each
                               sweep's rows greedily coloured in natural
                               order (rows of one colour share no updated
                               column) and visited colour by colour, one
                               fully parallel pass per colour.  It changes
                               the iteration, so its cycle convergence
                               factor differs from form 0's.
                             The setup phase always sweeps in natural order. */
    int32_t square_form;  /* square SVD kind (m = n; Sec. 5.1):
                             0 = as any SVD kind (rows and columns coarsened
                               on A A^t and A^t A, or row_form 0's rows from
                               A for the minimal target);
                             1 = the C/F splitting and the sparsity patterns
                               of both P and Q from the strength graph of A
                               itself, every level square (the setting of the
                               paper's square nonsymmetric example), P fitted
                               to the u vectors and Q to the v vectors;
                             2 = as 1 with one operator P = Q fitted to both
                               sets of vectors, so that B_c = C_c.
                             The Ritz step is two-sided in forms 1 and 2.
                             Ignored by non-square or SPD problems. */
    double redo_tol;      /* Sec. 6.3 redo of the interpolation for lagging
                             triplets: 0 = off; > 0: samg_solve redetermines
                             P and Q (samg_redo_interpolation) each time the
                             number of triplets with rho_j <= redo_tol grows
                             while some are still above it.  Makes samg_setup
                             keep its fine test vectors on the device
                             ((m + n) x n_t doubles, padded). */
} samg_params;

/* Defaults: n_t 8, theta 0.06, mu_t 8, mu_b 4, mu_tJ = mu_bJ = 1,
 * omega_J 0.7, n_mult 10, coarsest_max 100, max_levels 30,
 * seed 20110204, prec SAMG_FP32, n_conv 0 (all), coarse_pinv 0, row_form 0,
 * relax_order 0, square_form 0, redo_tol 0. */
void samg_default_params(samg_params *p);

/* ---------------------------------------------------------------- setup --
 * samg_setup: multiplicative phase (Sec. 3.3): n_mult bootstrap V-cycles
 * with test-vector relaxation (Secs. 3.4, 5.3), boot relaxation with
 * Rayleigh-quotient updates (Sec. 3.5), Ruge-Stueben coarsening on the
 * strength graph of Eq. strength (Sec. 3.7, Algorithm coarsening), weighted
 * LS interpolation (Sec. 3.8, Eq. LS), Galerkin operators (Eq. coarseOp) on
 * the GPU, a direct generalized SVD on the coarsest level (Sec. 3.6) and a
 * Ritz step per cycle.  A is m x n (SVD) or n x n symmetric (SPD_EIG).
 * n_b in [1, 16], n_b <= min(m, n).  Returns SAMG_E_INVALID for malformed
 * input (CSR: row_ptr from 0 to nnz and non-decreasing, columns in range and
 * strictly increasing within a row, finite values), SAMG_E_NT_TOO_SMALL if
 * n_t + n_b < 2; these checks run on the host before any device call, so
 * they report the same status on a machine without a GPU. */
samg_status samg_setup(const samg_csr *A, int n_b, samg_target target, samg_kind kind,
                       const samg_params *params, void *cuda_stream, samg_ctx **out);

/* samg_import: build a context from an existing hierarchy instead of running
 * the setup: the finest A, the interpolation operators P_l (m_l x m_{l+1})
 * and, for SAMG_SVD, Q_l (n_l x n_{l+1}) for l = 0 .. n_levels-2 (Q is
 * ignored for SPD_EIG), and the boot triplets (sigma: n_b values, U: m x n_b,
 * V: n x n_b, V ignored for SPD_EIG).  The library forms the Galerkin
 * operators A_{l+1} = P^t A_l Q, B_{l+1} = P^t B_l P, C_{l+1} = Q^t C_l Q
 * (Eq. coarseOp; B_0 = I, C_0 = I) on the GPU.  Every matrix is checked as
 * in samg_setup, and the row counts of P_l, Q_l against the level above,
 * before any device call. */
samg_status samg_import(const samg_csr *A, int n_levels, const samg_csr *P, const samg_csr *Q,
                        int n_b, samg_target target, samg_kind kind, const samg_params *params,
                        const double *sigma, const double *U, const double *V, void *cuda_stream,
                        samg_ctx **out);

/* Many independent problems with the same n_b, target, kind and parameters
 * (the batched workload of uneven sizes; the paper treats one problem at a
 * time).  Each problem gets its own hierarchy, context and CUDA stream.
 * Fusing problems into shared launches or one captured graph is not built.
 *  - samg_setup_batched: every problem's arguments are checked before any
 *    device call (SAMG_E_INVALID names the problem); then the setups run in
 *    order on the given stream, and a failure destroys the contexts made so
 *    far.  After its setup each context moves to a non-blocking stream the
 *    batch creates and owns (destroyed by samg_batch_destroy).
 *  - samg_solve_batched: rounds of one outer iteration per unconverged
 *    problem, each on its problem's stream, so that the problems overlap on
 *    the device; between rounds the host reads every problem's residuals
 *    and Ritz status (pinned copies).  It starts after the work queued on
 *    the setup's stream and queues that stream behind the problems' work.
 *    With redo_tol > 0 the problems are solved one after another instead.
 *    outer_done (count entries, may be NULL) receives each problem's
 *    iterations.  It returns SAMG_E_NOT_CONVERGED when some problem reached
 *    max_outer (the others are still solved), or the first other error,
 *    which stops every problem.
 *  - samg_batch_problem: the problem's context, owned by the batch (valid
 *    until samg_batch_destroy), for samg_get_triplets and the other
 *    per-context calls, which run on the problem's stream.
 *  - samg_batch_last_error(NULL) reports a failed samg_setup_batched. */
typedef struct samg_batch samg_batch;
samg_status samg_setup_batched(const samg_csr *const *A, int count, int n_b, samg_target target,
                               samg_kind kind, const samg_params *params, void *cuda_stream,
                               samg_batch **out);
samg_status samg_solve_batched(samg_batch *b, double tol, int max_outer, int *outer_done);
samg_status samg_batch_problem(samg_batch *b, int problem, samg_ctx **ctx);
int samg_batch_size(const samg_batch *b);
const char *samg_batch_last_error(const samg_batch *b);
void samg_batch_destroy(samg_batch *b);

/* A hierarchy and its boot triplets in one binary file.  The paper has no
 * file format; the file keeps the solve phase's inputs.
 *  - samg_export writes the context's finest A, its P_l and Q_l as the solve
 *    uses them (minimal SVD kind: P_0 = A Q_0, P_l = Q_l below), and the
 *    current boot triplets.
 *  - samg_write_hierarchy writes the same file from host arrays given as to
 *    samg_import (host only, no GPU needed).
 *  - samg_import_file builds a context from such a file as samg_import does
 *    (the Galerkin operators are rebuilt from P and Q).
 * Layout, little-endian: "SAMGHIER", u32 version (1), u32 kind, u32 target,
 * u32 n_b, u32 n_levels; csr A; for each level below the coarsest csr P_l,
 * then csr Q_l (SVD kind only); f64 sigma[n_b], U[rows_u][n_b], V[n][n_b]
 * (SVD kind only; rows_u = m, or n for SPD_EIG); u64 FNV-1a hash of every
 * byte before it.  csr = i32 m, i32 n, i64 nnz, i64 row_ptr[m + 1],
 * i32 col[nnz], f64 val[nnz].  A missing, truncated, corrupted or
 * other-version file, or malformed matrices, give SAMG_E_INVALID before any
 * device call. */
samg_status samg_export(samg_ctx *ctx, const char *path);
samg_status samg_write_hierarchy(const char *path, const samg_csr *A, int n_levels,
                                 const samg_csr *P, const samg_csr *Q, int n_b, samg_target target,
                                 samg_kind kind, const double *sigma, const double *U,
                                 const double *V);
samg_status samg_import_file(const char *path, const samg_params *params, void *cuda_stream,
                             samg_ctx **out);

void samg_destroy(samg_ctx *ctx);
const char *samg_last_error(const samg_ctx *ctx);

/* ---------------------------------------------------------------- solve --
 * samg_solve: additive phase (Sec. 4): per outer iteration one V-cycle for
 * every boot triplet with sigma_j fixed (V(mu_b, mu_b), Kaczmarz block
 * Gauss-Seidel for minimal, weighted Jacobi block Gauss-Seidel for dominant,
 * pseudo-inverse of X - sigma_j Y without its smallest singular value on the
 * coarsest level), then a Ritz step on the finest level (Sec. 4.3), until
 * max_j rho_j <= tol with rho_j = sqrt(|A v_j - s_j u_j|^2 +
 * |A^t u_j - s_j v_j|^2) / s_j (SPD: |A x_j - l_j x_j| / l_j).  The state
 * (sigma, U, V) stays on the device.  *outer_done = iterations run.
 * Returns SAMG_E_NOT_CONVERGED when max_outer is reached first. */
samg_status samg_solve(samg_ctx *ctx, double tol, int max_outer, int *outer_done);

/* Sec. 6.3: redetermines the interpolation operators by one downward sweep
 * of the multiplicative phase from the setup's fine test vectors and copies
 * of the current boot triplets, with the LS weights of the test vectors and
 * of the triplets marked converged (converged[j] != 0, n_b host ints) divided
 * by 1000; the coarse levels, their schedules and the coarsest
 * pseudo-inverse are rebuilt, and (sigma, U, V) is unchanged.  SAMG_E_INVALID
 * when the context kept no setup state (redo_tol was 0 at samg_setup, or an
 * imported hierarchy) or converged is NULL. */
samg_status samg_redo_interpolation(samg_ctx *ctx, const int32_t *converged);

/* Replace / read the boot triplets (host buffers; V ignored for SPD_EIG).
 * resid (n_b values, may be NULL) receives rho_j of the current triplets. */
samg_status samg_set_triplets(samg_ctx *ctx, const double *sigma, const double *U,
                              const double *V);
samg_status samg_get_triplets(samg_ctx *ctx, double *sigma, double *U, double *V,
                              double *resid);

/* As samg_set_triplets with device pointers (row-major n_b columns; V
 * ignored for SPD_EIG); copies are ordered on the context's stream. */
samg_status samg_set_triplets_device(samg_ctx *ctx, const double *sigma, const double *U,
                                     const double *V);

samg_status samg_set_precision(samg_ctx *ctx, samg_precision prec);

/* Selects the form of the coarsest additive solve of this context, as
 * samg_params.coarse_pinv (0 the paper's SVD pseudo-inverse, 1 the
 * generalized-eigen variant); SAMG_E_INVALID for any other value.  The
 * hierarchy is unchanged. */
samg_status samg_set_coarse_pinv(samg_ctx *ctx, int form);

/* Selects the order of this context's solve-phase sweeps, as
 * samg_params.relax_order (0 the paper's natural order, 1 the coloured
 * variant); SAMG_E_INVALID for any other value.  The hierarchy is
 * unchanged; each order's sweep programs are built on first use. */
samg_status samg_set_relax_order(samg_ctx *ctx, int order);

/* Banding of the exact-order sweep programs of the smoothing phases (a
 * tuning of the parallel schedule; the sweeps' results do not depend on it
 * beyond rounding order inside a row): a band of rows grows until it has
 * about band_rows rows per dependency level (1..4096 on every level; 0, the
 * default, takes 32 on the finest level and, on a coarser level of m x n,
 * max(m, n) / 65536 rounded to a power of two within [2, 32], the
 * fastest measured) or its live columns fill the shared-memory window;
 * per-level settings are cleared.  float_windows = 1 gives float32 and
 * bfloat16 launches programs banded with float32-only windows, 0 (default)
 * shares the float64 programs.  The programs are rebuilt on first use.
 * SAMG_E_INVALID for values out of range. */
samg_status samg_set_sweep_banding(samg_ctx *ctx, int band_rows, int float_windows);

/* The same for one level (band_rows 0: back to the context's setting). */
samg_status samg_set_sweep_banding_level(samg_ctx *ctx, int level, int band_rows);

/* Kernel timing: with profiling on, every launch of the solve phase is
 * bracketed by CUDA events on the context's stream.  samg_profile_read
 * returns, for one kernel class (0 Kaczmarz sweep, 1 block SpMM pass
 * (residual, restriction, interpolation, right-hand sides), 2 Jacobi step,
 * 3 coarsest solve, 4 Ritz step), the number of launches, their total device
 * time in ms and their algorithmic bytes (what the method must move: matrix
 * values and indices, right-hand sides read, iterates read and written),
 * accumulated since the last reset (reset != 0 clears after reading). */
samg_status samg_profile(samg_ctx *ctx, int enable);
/* Number of kernel launches the library has issued in this process. */
uint64_t samg_launch_count(void);
samg_status samg_profile_read(samg_ctx *ctx, int kernel_class, int reset, int64_t *launches,
                              double *total_ms, double *alg_bytes);

/* Wall-clock seconds the last samg_setup spent in each stage of the
 * multiplicative phase (Sec. 3), summed over its cycles and levels; the
 * stream is synchronised at every stage boundary, so GPU work is charged to
 * the stage that launched it.  Stages (index into seconds[]):
 *   0 strength graphs and C/F splittings (Eq. strength, Alg. coarsening; host)
 *   1 relaxation of the test vectors (Sec. 3.3)
 *   2 relaxation of the boot vectors with Rayleigh-quotient updates, down and
 *     up, and their interpolation (Sec. 3.4)
 *   3 Rayleigh quotients and least-squares interpolation fits (Sec. 3.8; host)
 *   4 Galerkin operators and transposes (Sec. 2)
 *   5 level preparation: row norms, sweep schedules, precision copies
 *   6 coarsest direct solve for the boot triplets (Sec. 3.6)
 *   7 Ritz steps (Sec. 4.3)
 *   8 completion of the solve-phase hierarchy
 *   9 the rest (test-vector draw, injections, uploads)
 * A samg_redo_interpolation (or a redo inside samg_solve) adds its
 * downward sweep's time to the same stages.  Writes min(count,
 * SAMG_SETUP_STAGES) values.  SAMG_E_INVALID: ctx or seconds NULL, or
 * count < 0. */
#define SAMG_SETUP_STAGES 10
samg_status samg_setup_times(const samg_ctx *ctx, double *seconds, int32_t count);

/* Hierarchy description: levels, and per level m_l, n_l, nnz(A_l) (arrays of
 * n_levels entries; pass NULL to query n_levels only). */
samg_status samg_get_hierarchy_info(const samg_ctx *ctx, int *n_levels, int32_t *m, int32_t *n,
                                    int64_t *nnz_A);

/* Copy one operator of level l to host CSR buffers.  which: 0 A_l, 1 B_l,
 * 2 C_l, 3 P_l, 4 Q_l.  With row_ptr == NULL only *rows, *cols, *nnz are set. */
samg_status samg_get_level_matrix(const samg_ctx *ctx, int level, int which, int32_t *rows,
                                  int32_t *cols, int64_t *nnz, int64_t *row_ptr, int32_t *col,
                                  double *val);

/* --------------------------------------------- single steps (host buffers) --
 * One step of the V-cycle on level l in the context's current precision;
 * used to compare the GPU path step by step with a reference.  U, V, kappa,
 * tau, Uc, Vc have m_l / n_l / m_{l+1} / n_{l+1} rows and n_b columns. */

/* count block Gauss-Seidel relaxations of A v - s B u = kappa,
 * A^t u - s C v = tau (Eqs. genSVDresid1-2, add), in place on U, V.  For the
 * minimal target the count relaxations run as one exact-order sweep program
 * (the same row updates in the same order as count sequential relaxations,
 * up to the rounding order inside a row); the first call for a given count
 * builds its schedule. */
samg_status samg_relax(samg_ctx *ctx, int level, int count, const double *sigma, double *U,
                       double *V, const double *kappa, const double *tau);

/* r = kappa - (A v - s B u), s = tau - (A^t u - s C v) (Eq. add), then
 * kappa_c = P^t r, tau_c = Q^t s (Eq. addCoarse). */
samg_status samg_residual_restrict(samg_ctx *ctx, int level, const double *sigma,
                                   const double *U, const double *V, const double *kappa,
                                   const double *tau, double *kappa_c, double *tau_c);

/* U += P Uc, V += Q Vc (Eq. corrAdd). */
samg_status samg_interpolate(samg_ctx *ctx, int level, double *U, double *V, const double *Uc,
                             const double *Vc);

/* [U; V] = (X_L - s_j Y_L)^+ [kappa; tau] on the coarsest level with the
 * smallest singular value left out (Sec. 4.2). */
samg_status samg_coarsest_solve(samg_ctx *ctx, const double *sigma, const double *kappa,
                                const double *tau, double *U, double *V);

/* One additive V-cycle on the finest level for all columns with sigma fixed
 * (Sec. 4.2), in place on U, V. */
samg_status samg_vcycle(samg_ctx *ctx, const double *sigma, double *U, double *V);

/* Ritz step (Sec. 4.3) on host buffers: in/out sigma, U, V; resid = rho_j. */
samg_status samg_ritz(samg_ctx *ctx, double *sigma, double *U, double *V, double *resid);

/* Host-only steps of the setup phase (no GPU needed), as samg_setup runs
 * them on each level:
 *  - samg_host_coarsen: strength of connection on the square N (Eq. strength,
 *    sums over all columns including the diagonal) and one-pass
 *    Ruge-Stueben coarsening (Algorithm coarsening, ties to the lowest index);
 *    cf[i] = 1 for C points, 0 for F points (n entries, host).
 *  - samg_host_ls_interp: interpolation P (n x n_c, n_c = number of C points)
 *    from that strength graph and cf: C rows carry a single 1 at the coarse
 *    index (increasing fine index), F rows the weighted LS weights of Eq. LS
 *    over the at most nf - 1 strongest C-point influences, fitting yF[i] by
 *    the yC values of those points with weights w (w multiplies the squared
 *    residuals).  yF, yC: n x nf row-major; w: nf.  Call with row_ptr = NULL
 *    to get *nnz, then with row_ptr (n + 1), col and val (nnz) to fill P.
 * Both return SAMG_E_INVALID for malformed input. */
samg_status samg_host_coarsen(const samg_csr *N, double theta, int8_t *cf);
samg_status samg_host_ls_interp(const samg_csr *N, double theta, const int8_t *cf, int nf,
                                const double *yF, const double *yC, const double *w,
                                int64_t *nnz, int64_t *row_ptr, int32_t *col, double *val);

/* Host-only strength graph of a product (no GPU needed): the strong
 * influences (Eq. strength, sums over all columns including the diagonal)
 * of N = A A^t, computed row by row from A without forming N, as samg_setup
 * does for A_l A_l^t and A_l^t A_l of the dominant SVD kind (pass A^t for
 * A^t A).  Row i of the output S (m x m) holds the j != i with
 * |n_ij| >= theta * sum_k |n_ik|, columns increasing, values |n_ij|.  Call
 * with row_ptr = NULL to get *nnz, then with row_ptr (m + 1), col and val
 * (nnz) to fill S.  Returns SAMG_E_INVALID for malformed input. */
samg_status samg_host_strength_product(const samg_csr *A, double theta, int64_t *nnz,
                                       int64_t *row_ptr, int32_t *col, double *val);

/* Host-only analysis of the exact-order Kaczmarz schedule (no GPU needed):
 * the dependency level of every row of a sweep program in natural order
 * (1 + the level of the latest earlier row sharing a column; rows of one
 * level share no column and are updated in parallel, Sec. 5.3), the program's
 * depth (levels in sequence) and its number of bands.  fused_count = 0: one
 * sweep over the rows of A (m rows); fused_count = k >= 1: k block
 * Gauss-Seidel relaxations of the minimal SVD kind on level 0 as one program
 * (per relaxation the m rows of A over [v; u], then the n rows of A^t;
 * k (m + n) rows).  row_level (host, may be NULL) receives the levels when
 * capacity is large enough.  Returns SAMG_E_INVALID for a malformed CSR or a
 * short row_level. */
samg_status samg_sweep_plan(const samg_csr *A, int fused_count, int32_t *row_level,
                            int64_t capacity, int *depth, int *nbands);

/* Host only: the greedy row colouring the coloured sweep variant
 * (relax_order = 1) uses, for tests that compare it with a reference (the
 * paper has no counterpart).  Rows are taken in natural order; row i gets the
 * smallest colour that no earlier row sharing a column with it has.
 * colour: m entries; *ncolour: the number of colours.  SAMG_E_INVALID for a
 * malformed CSR. */
samg_status samg_row_colours(const samg_csr *A, int32_t *colour, int32_t *ncolour);

/* Host-only export of an exact-order sweep schedule, for tests that replay
 * it on the CPU (the paper has no counterpart): the schedule the kernels
 * receive, with float64 coefficients, for one sweep over the rows of A
 * (fused_count = 0, spd = 0), for the fused program of fused_count
 * minimal-SVD relaxations with the level's B (m x m) and C (n x n)
 * (spd = 0), or for max(1, fused_count) stacked sweeps over the rows of
 * A - lambda_j B of the SPD kind (spd = 1, A square; mode 1: norms formed
 * per column).  B, C may be NULL (identity, as on the finest level).
 * resident_slots = 0 gives the solve's schedule.  resident_slots in
 * [1, 4095] builds, when the program keeps at most that many columns live,
 * one band with every column resident in the window (a mode the solve does
 * not use yet).  band_rows: rows per level a band grows to (0: 32, the
 * solve's default).  slot_cap: live columns per band, at most 4095 (0: 512;
 * the solve uses the largest window its launch holds).  Call with buf = NULL (capacity 0) to get *size,
 * then with a buffer of that many bytes.  Layout, little-endian:
 *   i32 rows, cols, nbands, nlevels, nchunks, max_slots, mode, shifted;
 *   i64 nreq, image_bytes;
 *   i32 band_chunk[nbands + 1];
 *   per chunk: i32 L0, nl, nr, ne, nx, nq, bytes, 0; i64 offset;
 *   per level: i32 first requirement, requirement count, publish, 0;
 *   per requirement: i32 band, levels that band must have completed;
 *   the chunk images (float64 coefficients);
 *   i32 order[nbands]: the band each ticket claims (every band's required
 *   bands at earlier tickets).
 * A chunk image holds, at 16-byte aligned offsets: per level {first row,
 * rows, lanes log2, flags: 1 has requirements | 2 publish after it}
 * (4 x i32); per level {first requirement in the image's list, count}
 * (2 x i32; a count c < 0 means the level's -c - 1 requirements are read
 * from the global list at that first index); per row {right-hand-side row,
 * first entry | entries << 16} (2 x i32); per row 1 / |a_r|^2 (f64); per
 * entry {column, flags} (2 x i32: 1 first touch in the band, 2 last touch,
 * 4 staged, window slot + 1 in bits 3-14, staged index from bit 15); per
 * entry a (f64); per entry b (f64, shifted programs only); per staged value
 * its column (i32); per carried requirement {band, levels that band must
 * have completed} (2 x i32, nq of them).  Returns SAMG_E_INVALID for a
 * malformed CSR or a short buffer.  The schedule is built on up
 * to SAMG_HOST_THREADS host threads (environment variable; default: the
 * hardware's, at most 16), as every schedule the library builds, and does
 * not depend on their number. */
samg_status samg_sweep_schedule(const samg_csr *A, const samg_csr *B, const samg_csr *C,
                                int fused_count, int spd, int resident_slots, int band_rows,
                                int slot_cap, unsigned char *buf,
                                int64_t capacity, int64_t *size);

/* Test hook for the bounded device waits (the paper has no counterpart):
 * from now on band `band` of the Kaczmarz schedules of level `level`
 * (which: 0 the single sweep over the rows of A, 1 over the rows of A^t,
 * 2 every fused relaxation program built so far) never publishes its
 * progress, so a
 * later band that needs it gives up after its 2 s bounded wait; the sweep
 * then returns SAMG_E_TIMEOUT and the context is poisoned (only
 * samg_destroy is valid).  band = -1 restores publishing.  Returns
 * SAMG_E_INVALID for a level, operator or band out of range. */
samg_status samg_debug_mute_band(samg_ctx *ctx, int level, int which, int band);

/* ------------------------------------------- device-level building blocks --
 * G = X^t Y for two row-major device blocks X, Y (rows x ld, first nb
 * columns used), G row-major nb x nb on the device; float64.  Uses a
 * device workspace of (ceil(rows / 2048) * nb * nb) doubles that it
 * allocates and frees.  stream: CUDA stream or NULL. */
samg_status samg_block_gram(const double *X, const double *Y, int64_t rows, int nb, int ld,
                            double *G, void *cuda_stream);

/* G = X^t Y exactly as samg_block_gram (same kernels, same summation order,
 * bitwise the same result), but allocating nothing: no cudaMalloc, cudaFree
 * or allocating library routine.  The paper has no counterpart to this entry
 * point; it is a service for callers that cannot allocate device memory
 * here -- a caller whose memory pool already owns the free HBM (a new
 * cudaMalloc would fail or fragment it), or a caller on a latency-critical
 * stream that cannot afford cudaFree, which waits for all work on the
 * device.  It also does not synchronize the stream.
 *
 * The partial sums live in one fixed device array of 131072 doubles
 * (1 MiB): calls with ceil(rows / 2048) * nb * nb > 131072 are rejected with
 * SAMG_E_INVALID and a message (e.g. rows <= 4,194,304 at nb = 8, rows <=
 * 1,048,576 at nb = 16).  The array is shared by all callers in the process
 * on a device: calls whose GPU work overlaps (other streams, other host
 * threads) race on it and give wrong results; serialize them.  The first
 * call in each CUDA context (each device's primary context, and again after
 * a cudaDeviceReset has replaced it) looks the array's address up with
 * cudaGetSymbolAddress (that device current) and caches it under the
 * context's unique id; make that first call before any stream capture
 * begins on that device.  Arguments as for
 * samg_block_gram; X, Y and G are device pointers, stream NULL = legacy
 * default stream; the call returns when the work is enqueued. */
samg_status samg_block_gram_noalloc(const double *X, const double *Y, int64_t rows, int nb,
                                    int ld, double *G, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SAMG_H */
