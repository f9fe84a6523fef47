/*
 * ldupcg.h -- C interface of libldupcg: Jacobi-preconditioned conjugate
 * gradients, plain and pipelined, for symmetric finite-volume systems stored
 * in OpenFOAM LDU face addressing, on one GB300 GPU (sm_103a).
 *
 * The operation (Sec. 2, Eq. 9): solve A x = b, A square, symmetric and
 * positive definite, one row per mesh cell.  A arrives in the lduMatrix
 * layout the paper names (Sec. 5): diag[n]; for each internal face f an
 * owner cell owner[f] and a neighbour cell neighbour[f] with owner < neighbour,
 * upper[f] = A[owner, neighbour] and lower[f] = A[neighbour, owner].  The
 * number of non-zeros is n + 2*nFaces (Sec. 4.2, the n_i + 2 o_i of Eq. 2).
 *
 * Conventions for every entry point:
 *  - Pointers named in the argument list as "device" must point to memory of
 *    the GPU that was current when the matrix handle was created; "host"
 *    pointers to ordinary host memory.  The caller owns every buffer it
 *    passes; the library keeps no pointer to caller memory after a call
 *    returns.  A handle owns its own device allocations (repacked matrix,
 *    work vectors) until ldu_destroy.
 *  - Work is queued on `stream` (a cudaStream_t; NULL = the legacy default
 *    stream).  Entry points that return host results (iteration counts,
 *    residuals, statuses) synchronise that stream before returning; the
 *    others return once the work is queued.
 *  - The return value is a status (ldu_status).  0 is success, 1 means the
 *    iteration cap was reached (outputs hold the last iterate), negative
 *    values are errors; no C++ exception crosses this interface.  On an
 *    error, outputs are unspecified but buffers stay valid.
 *  - A handle must not be used by two calls that may run concurrently: the
 *    solves and the double product of one handle share its work vectors.
 */
#ifndef LDUPCG_H
#define LDUPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldu_matrix ldu_matrix;       /* opaque handle */
typedef struct CUstream_st *ldu_stream_t;   /* identical to cudaStream_t */

typedef enum ldu_status {
    LDU_OK = 0,
    LDU_NOT_CONVERGED = 1,          /* iteration cap reached */
    LDU_ERR_BAD_ARG = -1,           /* null pointer, negative size, bad option */
    LDU_ERR_BAD_ADDRESSING = -2,    /* owner >= neighbour or an index outside [0, n) */
    LDU_ERR_NOT_SPD = -3,           /* non-positive diagonal or CG breakdown (p^T A p <= 0) */
    LDU_ERR_CUDA = -4,              /* a CUDA runtime call failed */
    LDU_ERR_BARRIER_TIMEOUT = -5,   /* a grid barrier of a persistent kernel timed out */
    LDU_ERR_OOM = -6,               /* device allocation failed */
    LDU_ERR_UNSUPPORTED = -7        /* size beyond what the layout can index */
} ldu_status;

typedef enum ldu_precision {
    LDU_FP64 = 0,      /* everything in double */
    LDU_FP32 = 1,      /* ldu_spmv only: float values and vectors */
    LDU_MIXED = 2      /* float pipelined recurrences, double residual and solution */
} ldu_precision;

/* Layout options of the repacked matrix and launch shape of its kernels.
 * A zeroed struct (or NULL) selects the defaults. */
typedef struct ldu_opts {
    int slice_rows;     /* rows per sliced-ELL slice: 32, 64 or 128 (default 128) */
    int block_threads;  /* threads per block of the persistent solve kernels:
                           128 or 256 (default 256) */
    int blocks_per_sm;  /* resident blocks per SM for the persistent kernels;
                           0 = as many as fit.  The mixed solve also has
                           builds with fewer registers per thread for 3
                           (slice_rows 32 or 64) and 4 (slice_rows 32)
                           blocks per SM, chosen by this field */
    int staging;        /* float sweeps of the mixed solve: 0 = stage each
                           warp's next matrix slice into shared memory with
                           bulk copies when it fits (default), -1 = read the
                           matrix with plain loads */
    int min_slices;     /* single-system solves launch at most one block per
                           min_slices slices, so that a small system is not
                           spread over more blocks than it can keep busy
                           (every block joins every grid barrier); 0 = the
                           default (8: measured 15-20 % faster on 32^3 and
                           48^3 systems, neutral from 64^3 up), -1 = no
                           limit */
} ldu_opts;

/* Options of pipecg_solve (and pcg_solve_batched).  NULL or zeroed selects
 * the defaults given here. */
typedef struct pcg_opts {
    int rr_period;          /* iterations between residual replacements:
                               LDU_FP64 default 0 (replace only when the
                               recursive residual reaches tol);
                               LDU_MIXED: when rr_period and tau are both 0,
                               16 with tau 0.3 (FP64 replacement) */
    double tau;             /* LDU_MIXED: also replace when (r, M^-1 r) has
                               dropped by tau^2 since the last replacement;
                               0 = off (0.3 when rr_period is 0 too) */
    int restart;            /* LDU_MIXED: 1 = every replacement restarts the
                               search (classic defect correction with inner
                               tolerance tau); 0 = keep the search directions
                               (default) */
    double barrier_timeout_s;  /* grid-barrier spin limit, default 10 s */
    int fault_inject;       /* testing only: 1 = block 0 of the persistent kernel
                               returns before its first barrier, so the others
                               time out and the call returns
                               LDU_ERR_BARRIER_TIMEOUT; 0 otherwise */
    int deflate;            /* LDU_MIXED: 1 = deflate the constant vector (deflated
                               CG, Saad et al. 2000): removes the near-null mode of
                               pure-Neumann systems with a reference cell, which
                               float recurrences cannot resolve; 0 = off (default) */
} pcg_opts;

/* Counters of the last solve on a handle. */
typedef struct ldu_solve_stats {
    int status;
    int iters;              /* A*p products of the loop (float ones for LDU_MIXED) */
    int replacements;       /* true-residual evaluations, initial one included */
    double relres;          /* ||b - A x||_2 / ||b||_2 at exit: the residual formed
                               in FP64 (LDU_MIXED: its norm summed from its float
                               rounding, relative accuracy about 1e-7) */
    double bnorm;           /* ||b||_2 */
    int grid_blocks;        /* blocks of the persistent launch */
    int block_threads;
    int staged;             /* 1 when the float sweeps staged the matrix in
                               shared memory, 0 for plain loads */
} ldu_solve_stats;

/* Facts about a handle's device layout. */
typedef struct ldu_info {
    int64_t n, n_faces;
    int64_t n_padded;       /* rows rounded up to whole slices */
    int64_t nnz_padded;     /* stored off-diagonal slots incl. padding */
    int slice_rows;
    int64_t n_slices;
    int max_row_entries;    /* widest slice */
    int64_t device_bytes;   /* bytes the handle holds on the device */
    int col16;              /* 1: the handle also stores each slot's column as a
                               16-bit offset from its row (every offset fits),
                               which the staged float sweeps read instead of
                               the int32 columns */
} ldu_info;

/* Create a handle from an LDU matrix (Sec. 5, lduMatrix; Eq. 9's A).
 *   n, nFaces           cells and internal faces (n >= 0, nFaces >= 0)
 *   owner, neighbour    device int32[nFaces]: owner[f] < neighbour[f], both in [0, n);
 *                       faces need not be sorted
 *   diag                device double[n], every entry > 0
 *   upper, lower        device double[nFaces]
 *   opt                 host, may be NULL
 *   out                 host: receives the handle (NULL on failure)
 * Validates the addressing on the device, repacks A into the handle's
 * sliced-ELL layout (rows in the caller's order, off-diagonals of a row in
 * ascending column order, symmetric diagonal scaling applied) and keeps a
 * copy of owner/neighbour for ldu_face_grad.  Synchronises `stream`.
 * Errors: BAD_ARG, BAD_ADDRESSING, NOT_SPD (diag <= 0 or not finite), OOM,
 * UNSUPPORTED (n or the padded non-zero count above 2^31 - 1), CUDA. */
int ldu_create(int64_t n, int64_t nFaces, const int32_t *owner, const int32_t *neighbour,
               const double *diag, const double *upper, const double *lower,
               const ldu_opts *opt, ldu_stream_t stream, ldu_matrix **out);

/* Replace the values of a handle's matrix, keeping its addressing
 * (device double diag[n], upper[nFaces], lower[nFaces]).  Queued on stream;
 * a non-positive diagonal is reported by the next solve as NOT_SPD. */
int ldu_update_values(ldu_matrix *A, const double *diag, const double *upper,
                      const double *lower, ldu_stream_t stream);

/* Set the matrix of a finite-volume Laplacian from face coefficients:
 * upper = lower = -coef[f], diag[i] = diag_extra[i] + sum of coef over the
 * faces of cell i (the positive assembly of Sec. 2, Eq. 8's operator).
 *   coef        device double[nFaces]
 *   diag_extra  device double[n]: boundary-condition part of the diagonal
 * The row sums are formed in a fixed order, so repeated calls agree bitwise. */
int ldu_set_face_coeffs(ldu_matrix *A, const double *coef, const double *diag_extra,
                        ldu_stream_t stream);

/* y = A x (Sec. 2.1's sparse matrix-vector product; Table 1's first kernel).
 *   precision  LDU_FP64: x, y are device double[n], values in double (two
 *                        passes: D^1/2 x into a work vector of the handle,
 *                        then the product);
 *              LDU_FP32: x, y are device float[n], values and sums in float.
 * x and y may not overlap.  Queued on stream. */
int ldu_spmv(const ldu_matrix *A, int precision, const void *x, void *y, ldu_stream_t stream);

/* Jacobi-preconditioned CG (Sec. 2, Eq. 9; Saad, Iterative Methods, Alg. 9.1
 * with M = diag(A)), FP64, one persistent cooperative launch with three grid
 * barriers per iteration.
 *   b        device double[n]
 *   x        device double[n]: initial guess in, solution out
 *   tol      stop when the recursive ||r||_2/||b||_2 <= tol and the true
 *            residual recomputed at that point confirms it (else the search
 *            restarts from the true residual)
 *   maxit    cap on iterations (>= 0)
 *   iters    host, may be NULL: iterations taken
 *   relres   host, may be NULL: true ||b - A x||_2/||b||_2 at exit
 * b = 0 gives x = 0, relres = 0.  Synchronises stream.
 * Returns OK, NOT_CONVERGED, NOT_SPD (breakdown), BARRIER_TIMEOUT, BAD_ARG, CUDA. */
int pcg_solve(const ldu_matrix *A, const double *b, double *x, double tol, int maxit,
              int *iters, double *relres, ldu_stream_t stream);

/* Pipelined Jacobi-PCG (Sec. 4.1; Ghysels and Vanroose 2014): one grid-level
 * reduction per iteration, overlapped with the matrix-vector product.
 *   precision  LDU_FP64: the recurrences in double, residual replacement when
 *              the recursive residual reaches tol (and every rr_period steps);
 *              LDU_MIXED: the recurrences in float on a float copy of the
 *              matrix; the solution accumulates in double and the residual
 *              is replaced by the double b - A x (its norms, for the
 *              stopping test and relres, summed from its float rounding as
 *              float pairs: relative accuracy about 1e-7) every rr_period steps and
 *              whenever (r, M^-1 r) has dropped by tau^2 (opts; by default
 *              every 16 steps or on a 0.3^2 drop).  Convergence is only
 *              declared on such a double residual.  deflate = 1 adds the
 *              constant-vector deflation for singular-ish pressure systems.
 *   opts       host, may be NULL
 * Other arguments as pcg_solve.  A non-positive pipelined denominator is
 * treated as rounding drift (replace and restart); only a non-positive
 * (A u, u) on a fresh start returns NOT_SPD. */
int pipecg_solve(const ldu_matrix *A, const double *b, double *x, double tol, int maxit,
                 int precision, const pcg_opts *opts, int *iters, double *relres,
                 ldu_stream_t stream);

/* nsteps backward-Euler steps of the heat equation (laplacianFoam's
 * implicit step, Eq. 8): with the handle holding M + A (the diagonal mass
 * term M = rho c V / dt added to the diffusion matrix, for instance through
 * ldu_set_face_coeffs' diag_extra), each step solves
 *     (M + A) T^(n+1) = M T^n
 * starting from T^n, in place.  The handle and its repacked matrix are
 * reused across steps; the right-hand side is formed by a kernel into a
 * buffer of the handle (allocated on the first call).
 *   mass        device double[n]: the diagonal M
 *   T           device double[n]: T^0 in, T^nsteps out
 *   precision   LDU_FP64 (Jacobi-PCG, as pcg_solve) or LDU_MIXED (as
 *               pipecg_solve with LDU_MIXED and opts)
 *   iters_total host, may be NULL: iterations summed over the steps
 *   relres_last host, may be NULL: the last step's true relative residual
 * Stops at the first step that does not return OK and returns its status.
 * Single-system handles only (UNSUPPORTED on a batched handle).
 * Synchronises stream after every step. */
int ldu_heat_steps(ldu_matrix *A, const double *mass, double *T, int nsteps, double tol,
                   int maxit, int precision, const pcg_opts *opts, int *iters_total,
                   double *relres_last, ldu_stream_t stream);

/* Gradient of a loss with respect to the face coefficients of
 * ldu_set_face_coeffs, given the adjoint solution lambda = A^-T dL/dx and
 * the forward solution x:  dcoef[f] = -(lambda[o] - lambda[n]) (x[o] - x[n])
 * with o = owner[f], n = neighbour[f] (device double arrays; dcoef has
 * nFaces entries in the caller's face order).  Queued on stream. */
int ldu_face_grad(const ldu_matrix *A, const double *lambda, const double *x, double *dcoef,
                  ldu_stream_t stream);

/* Gradient of a loss with respect to the boundary part of the diagonal of
 * ldu_set_face_coeffs: ddiag[i] = -lambda[i] x[i] (device double arrays of
 * the caller's cells).  Queued on stream. */
int ldu_diag_grad(const ldu_matrix *A, const double *lambda, const double *x, double *ddiag,
                  ldu_stream_t stream);

/* Gradient of a loss with respect to every stored off-diagonal value taken
 * independently (upper and lower need not stay equal: the derivative of the
 * solution map in non-symmetric directions, exact at the symmetric A that
 * the solvers accept): differentiating A x = b gives dL/dA_ij = -lambda_i x_j
 * with lambda = A^-T dL/dx (= A^-1 dL/dx here), so
 *   dupper[f] = -lambda[owner[f]] x[neighbour[f]]
 *   dlower[f] = -lambda[neighbour[f]] x[owner[f]]
 * (device double[nFaces], the caller's face order); the diagonal's gradient
 * -lambda_i x_i is ldu_diag_grad's.  Queued on stream. */
int ldu_value_grad(const ldu_matrix *A, const double *lambda, const double *x, double *dupper,
                   double *dlower, ldu_stream_t stream);

/* Face coefficients and wall terms of the FVM Laplacian from cell
 * diffusivities (Eq. 8's laplacian operator, discretised as in Sec. 5's
 * lduMatrix): with the harmonic mean k_f = 2 k_o k_n / (k_o + k_n) of the
 * two cells of face f,
 *   coef[f]       = g[f] * k_f           (pass to ldu_set_face_coeffs)
 *   diag_extra[i] = k[i] * bfac[i]       (Dirichlet-wall part of the diagonal)
 *   k           device double[cells], every entry > 0
 *   g           device double[nFaces]: geometric factor |S_f| / |d_on| of each face
 *   bfac        device double[cells]: sum of 2 |S_b| / w_P over the cell's Dirichlet faces
 *   coef, diag_extra   device double[nFaces] / [cells] outputs
 * All arrays in the caller's face and cell order (concatenated for a batched
 * handle).  Queued on stream. */
int ldu_harmonic_coeffs(const ldu_matrix *A, const double *k, const double *g,
                        const double *bfac, double *coef, double *diag_extra,
                        ldu_stream_t stream);

/* Chain rule of ldu_harmonic_coeffs: from dL/dcoef and dL/ddiag_extra (for
 * instance ldu_face_grad's and ldu_diag_grad's outputs),
 *   dk[P] = ddiag_extra[P] * bfac[P]
 *         + sum over the faces f of P of dcoef[f] * g[f] * 2 k_N^2 / (k_P + k_N)^2
 * where N is the other cell of f.  Each cell's sum is formed in a fixed order
 * (no atomics), so repeated calls agree bitwise.  Arguments as
 * ldu_harmonic_coeffs; dk: device double[cells].  Queued on stream. */
int ldu_harmonic_grad(const ldu_matrix *A, const double *k, const double *g, const double *bfac,
                      const double *dcoef, const double *ddiag_extra, double *dk,
                      ldu_stream_t stream);

/* Counters of the last solve (host struct filled from host memory; no sync). */
int ldu_last_stats(const ldu_matrix *A, ldu_solve_stats *stats);

/* Layout facts of a handle. */
int ldu_get_info(const ldu_matrix *A, ldu_info *info);

/* Free a handle and everything it owns (NULL is ignored).  Waits for the
 * device work queued on the handle's kernels to finish. */
void ldu_destroy(ldu_matrix *A);

/* A static string naming a status code. */
const char *ldu_status_string(int status);

/* ---- batches of independent systems -------------------------------------
 * Many systems of uneven size (the laplacianFoam / icoFoam solve repeated
 * over independent meshes) solved by one persistent cooperative launch:
 * each system is solved by a team of blocks sized to its work (one block
 * for small systems), with per-system scalars, stopping tests and status. */

/* Team sizing of a batched launch.  A zeroed struct selects the defaults. */
typedef struct batch_opts {
    int max_team;            /* largest team of blocks on one system (default 32) */
    double team_work_scale;  /* multiplies the work per block that sizes teams;
                                above 1 gives smaller teams (default 1) */
} batch_opts;

/* Create a batched handle.  On a batched handle, ldu_update_values,
 * ldu_set_face_coeffs, ldu_face_grad and ldu_diag_grad take their arrays in
 * the caller's concatenated order; ldu_spmv returns UNSUPPORTED.
 *   nsys            number of systems (> 0)
 *   n, nFaces       host int64[nsys]: cells and internal faces of each system
 *   owner, neighbour, diag, upper, lower
 *                   device arrays of all systems concatenated in order; face
 *                   indices are local to their system (0-based, owner < neighbour)
 * Other arguments and errors as ldu_create; a face outside its own system is
 * BAD_ADDRESSING.  Synchronises stream. */
int ldu_create_batched(int nsys, const int64_t *n, const int64_t *nFaces, const int32_t *owner,
                       const int32_t *neighbour, const double *diag, const double *upper,
                       const double *lower, const ldu_opts *opt, ldu_stream_t stream,
                       ldu_matrix **out);

/* Recompute the team schedule of a batched handle (synchronises stream). */
int ldu_batch_schedule(ldu_matrix *A, const batch_opts *opts, ldu_stream_t stream);

/* Facts about a batched handle (host outputs, each may be NULL). */
int ldu_batch_info(const ldu_matrix *A, int *nsys, int *grid_blocks, int *ntasks, int *max_team);

/* Queue the solve of every system of a batched handle (precision LDU_FP64:
 * Jacobi-PCG; LDU_MIXED: the mixed pipelined method of pipecg_solve), with
 * the caller's concatenated device b and x (x: initial guesses in,
 * solutions out).  Does not synchronise and allocates nothing, so it can be
 * captured in a CUDA graph; ldu_batch_results reads the outcome. */
int pcg_solve_batched_async(const ldu_matrix *A, const double *b, double *x, double tol,
                            int maxit, int precision, const pcg_opts *opts, ldu_stream_t stream);

/* Per-system outcome of the last batched solve (host arrays of nsys entries,
 * each may be NULL): iterations, true relative residual, status.  Returns
 * the worst status.  Synchronises stream. */
int ldu_batch_results(const ldu_matrix *A, int *iters, double *relres, int *status,
                      ldu_stream_t stream);

/* pcg_solve_batched_async followed by ldu_batch_results. */
int pcg_solve_batched(const ldu_matrix *A, const double *b, double *x, double tol, int maxit,
                      int precision, const pcg_opts *opts, int *iters, double *relres,
                      int *status, ldu_stream_t stream);

/* The pressure stage of a PISO step (Sec. 2, icoFoam: the pressure solution
 * and the explicit correction after the momentum predictor), on a handle
 * whose matrix is the pressure matrix of the face coefficients `coef`
 * (upper = lower = -coef, diagonal = the coefficient sums plus the
 * reference-cell pin, e.g. set by ldu_set_face_coeffs):
 *   1. b = -div(phi), div_P = sum of phi_f over the faces P owns minus the
 *      sum over the faces where P is the neighbour (formed per cell in the
 *      order of its neighbours, so repeated calls agree bitwise);
 *   2. A p = b solved from the caller's p (the previous pressure: a warm
 *      start), with pcg_solve (LDU_FP64) or the mixed pipelined method
 *      (LDU_MIXED; opts as pipecg_solve, e.g. deflate for pure-Neumann
 *      pressure systems);
 *   3. phi_f -= coef_f (p[neighbour[f]] - p[owner[f]]), after which
 *      div(phi) equals the solve's residual (zero to its tolerance).
 *   coef   device double[nFaces]
 *   phi    device double[nFaces]: the predicted fluxes in, corrected out
 *   p      device double[n]: initial guess in, pressure out
 *   iters, relres: host, may be NULL (the solve's counts).
 * Single-system handles only (UNSUPPORTED on a batch).  On NOT_CONVERGED
 * the fluxes are corrected with the last iterate; on an error phi is left
 * as it was.  Synchronises stream. */
int ldu_piso_pressure(ldu_matrix *A, const double *coef, double *phi, double *p, double tol,
                      int maxit, int precision, const pcg_opts *opts, int *iters,
                      double *relres, ldu_stream_t stream);

/* ---- aggregation-AMG preconditioned CG (Sec. 5; Table 2's AMG-CG) ----
 *
 * The paper also preconditions CG with a V-cycle of an aggregation-based
 * algebraic multigrid (aggregates grown around a distance-2 maximal
 * independent set, weighted-Jacobi smoothing), taken from CUSP, whose
 * aggregation forms that set in parallel (Bell, Dalton & Olson 2012).  This
 * library reads it as:
 *   graph        the stored off-diagonal entries of A (sparsity patterns are
 *                structural throughout: coarse entries that cancel are kept);
 *   roots        a distance-2 maximal independent set by Luby-style rounds:
 *                row i has priority h_i = mix64((i + 1) * 0x9E3779B97F4A7C15)
 *                (SplitMix64); an undecided row whose (state, h) is the
 *                largest within two steps becomes a root, one that sees a
 *                root within two steps is excluded, until every row is
 *                decided;
 *   aggregates   roots numbered in row order; a row next to a root joins it;
 *                every other row joins its assigned neighbour of largest
 *                |a_ij| (values within 1e-12 of the row's largest |a_ij| are
 *                ties, won by the lower aggregate number);
 *   prolongator  P = (I - w D^-1 A) P_t with P_t the aggregates' indicator
 *                and w = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii;
 *   hierarchy    A_c = P^T A P, repeated until a level has at most
 *                max_coarse rows (or max_levels prolongators exist, or an
 *                aggregation no longer shrinks the level); the coarsest level
 *                is solved with its dense inverse;
 *   cycle        V(1,1) from zero with the same weighted Jacobi;
 *   outer        CG (Saad Alg. 9.1) with M^-1 r = V(r), stopping when the
 *                recursive ||r||_2 <= tol ||b||_2 and the true residual
 *                agrees (otherwise the search restarts from it).
 * The hierarchy is built by device kernels (the host reads only counts
 * between them, and inverts the coarsest level); every sum of the
 * construction is formed in a fixed order, so the same matrix always gives
 * the same hierarchy.  The solve runs entirely in device kernels, its
 * scalars (alpha, beta, the residual norms, the stopping decision) computed
 * and kept on the device. */
typedef struct ldu_amg ldu_amg;   /* opaque AMG hierarchy */

typedef struct amg_opts {
    int max_coarse;     /* coarsest-level rows at most this, 1..4096 (default 500) */
    int max_levels;     /* prolongators at most this, 1..64 (default 12) */
    int lanes_per_row;  /* lanes that share one row of R and of the coarse-level
                           matrices: 1, 2, 4, 8, 16 or 32; 0 = the power of two
                           nearest a quarter of the operator's mean row length
                           (default) */
} amg_opts;

/* Build the hierarchy of an LDU matrix.  n, nFaces, owner, neighbour,
 * diag, upper, lower: as ldu_create (device arrays, validated on the
 * device; the hierarchy uses both triangles, the solvers need a symmetric
 * positive definite A).  aopt: host, may be NULL.  The fine level stores A's
 * off-diagonal part in sliced ELL with 32-row slices (plus 16-bit column
 * offsets from the row when every offset fits), coarse levels in CSR; every
 * level keeps its diagonal and w/diagonal, P and R = P^T in CSR, all values
 * in double and in float.  The construction takes temporary device memory
 * (stream-ordered allocations on `stream`) of the order of the fine matrix
 * times its rows' product lengths, released before returning.  Synchronises
 * stream.  Errors as ldu_create; NOT_SPD if a level's diagonal is not
 * positive or the coarsest matrix is singular; UNSUPPORTED if coarsening
 * stops above 4096 rows or a level's entries exceed int32 indexing. */
int ldu_amg_create(int64_t n, int64_t nFaces, const int32_t *owner, const int32_t *neighbour,
                   const double *diag, const double *upper, const double *lower,
                   const amg_opts *aopt, ldu_stream_t stream, ldu_amg **out);

/* Free a hierarchy (waits for the device first); NULL is a no-op. */
void ldu_amg_destroy(ldu_amg *M);

/* Shape of a hierarchy: *levels = prolongators + 1; rows[l] and nnz[l]
 * (host int64 arrays, each may be NULL) receive each level's rows and stored
 * non-zeros (both triangles and the diagonal), for l < max_levels. */
int ldu_amg_info(const ldu_amg *M, int *levels, int64_t *rows, int64_t *nnz, int max_levels);

/* Aggregate number of every row of level `level` (host int32[rows of that
 * level]); level must have a prolongator.  BAD_ARG otherwise. */
int ldu_amg_aggregates(const ldu_amg *M, int level, int32_t *agg);

/* x = V(b), one V(1,1) cycle from zero.  precision LDU_FP64: b, x are device
 * double[n] and the cycle runs in double; LDU_FP32: device float[n], the
 * cycle runs on the float copies of the level matrices.  b and x must be
 * distinct (BAD_ARG if they are the same pointer).  Queued on stream;
 * allocates nothing. */
int ldu_amg_vcycle(ldu_amg *M, int precision, const void *b, void *x, ldu_stream_t stream);

/* AMG-preconditioned CG.  b: device double[n]; x: device double[n], initial
 * guess in, solution out; iters, relres: host, may be NULL (relres is the
 * true ||b - A x||_2 / ||b||_2 at exit).
 *   precision  LDU_FP64: the cycle in double, Saad Alg. 9.1's beta (the
 *              method as stated); LDU_MIXED: the cycle in float on float
 *              copies of the level matrices, outer CG in double with the
 *              Polak-Ribiere beta (r_new, z_new - z_old) / (r_old, z_old),
 *              which keeps CG convergent under the float cycle's rounding;
 *              the stopping test is on the double residual either way.
 * NOT_SPD on a breakdown (p^T A p <= 0), NOT_CONVERGED when maxit is
 * reached.  Synchronises stream: the host reads the device-resident scalars
 * between batches of iterations sized from the observed convergence rate.
 * One outer iteration (its 16 kernels) is captured as a CUDA graph on the
 * hierarchy's private stream at the first call with a given x and replayed
 * on `stream` for every iteration; a call with another x updates the graph. */
int amg_pcg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int precision,
                  int *iters, double *relres, ldu_stream_t stream);

/* Pipelined AMG-preconditioned CG (Table 2's AMG-PipeCG; Ghysels & Vanroose's
 * pipelined PCG, the method of Sec. 4.1, with M = one FP64 V-cycle): per
 * iteration one cycle m = V(w), one product n = A m, and one pass that
 * updates z, q, s, p, x, r, u, w and forms (r, u), (w, u), (r, r) together.
 * In exact arithmetic its iterates are amg_pcg_solve's.  Stops on the
 * recursive residual and confirms with the true one (a disagreement
 * restarts the recurrences from it); a non-positive step denominator after
 * the first step of a run is rounding drift and takes the same path, only a
 * non-positive (u, A u) on a fresh start returns NOT_SPD.  Arguments, outputs and errors as
 * amg_pcg_solve (FP64 only).  Allocates seven work vectors on a hierarchy's
 * first call; one iteration is captured and replayed as a CUDA graph as in
 * amg_pcg_solve.  Synchronises stream. */
int amg_pipecg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
                     double *relres, ldu_stream_t stream);

/* Jacobi-PCG on a small LDU system without any device allocation.  The paper
 * has no counterpart: this exists for callers that cannot call cudaMalloc
 * (their device memory is owned by another allocator, such as a framework's
 * caching pool or a fixed-budget runtime, or they cannot afford cudaMalloc's
 * implicit device synchronisation) and therefore cannot create a handle.
 * It repacks the caller's arrays and runs the same kernel as pcg_solve with
 * the same layout and launch shape, so the result equals pcg_solve's on a
 * default handle.  All intermediate data live in one fixed-size __device__
 * array (8,130,816 bytes (7.75 MiB)) that every GPU loading the library holds until the
 * process exits.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process, so that first call should come before any stream capture,
 * and the entry point must not be used again after a cudaDeviceReset in the
 * same process.
 *   n <= 32768 cells and nFaces <= 131072: larger inputs return
 *   LDU_ERR_UNSUPPORTED before any GPU work.  At most 262144 stored
 *   off-diagonal slots (8 per row on average, padding included): this limit
 *   is checked on the device after the addressing has been validated (the
 *   stream is synchronised for it), and an input beyond it also returns
 *   LDU_ERR_UNSUPPORTED, before the matrix is repacked.
 *   owner, neighbour, diag, upper, lower, b: device arrays as in ldu_create
 *   and pcg_solve; x: device double[n], initial guess in, solution out;
 *   iters, relres: host, may be NULL.
 * Every call on a device shares the scratch array and clears what it needs
 * zeroed; calls whose work overlaps on the GPU (other streams or threads)
 * race on it.  Synchronises stream.  Errors as ldu_create and pcg_solve. */
int pcg_solve_ldu_noalloc(int64_t n, int64_t nFaces, const int32_t *owner,
                          const int32_t *neighbour, const double *diag, const double *upper,
                          const double *lower, const double *b, double *x, double tol, int maxit,
                          int *iters, double *relres, ldu_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LDUPCG_H */
