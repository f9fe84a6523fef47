/*
 * ldu_oracle.c -- the oracle: a plain, slow, obviously correct FP64 CPU
 * restatement of the Jacobi-preconditioned conjugate-gradient solve of a
 * symmetric finite-volume system stored in OpenFOAM LDU face addressing.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU baseline call it; the CUDA library never does, and the two share no
 * code, header, table or helper.  Loops are in the textbook order, with no
 * blocking, fusion or reordering, so that every routine can be checked
 * against its source by eye:
 *
 *   or_spmv           y = A x over faces                (Sec. 2.1; Sec. 5 lduMatrix)
 *   or_pcg            Jacobi-preconditioned CG          (Sec. 2, Eq. 9; Saad Alg. 9.1)
 *   or_pipecg         pipelined preconditioned CG       (Sec. 4.1; Ghysels & Vanroose
 *                                                        2014, preconditioned variant)
 *   or_mixed_pipecg   FP32 pipelined PCG with FP64 residual replacement and FP64
 *                     solution accumulation (reliable updates or defect correction)
 *   or_face_grad      adjoint face-coefficient gradient -(l_o - l_n)(x_o - x_n)
 *   or_value_grad     adjoint gradient of every stored LDU value: dL/dA_ij = -l_i x_j
 *   or_harmonic_coeffs / or_harmonic_grad
 *                     face coefficients from cell diffusivities through the
 *                     harmonic mean, and the chain rule back to the cells
 *   or_lu_solve       dense LU with partial pivoting (tiny systems)
 *
 * Conventions shared with the library's interface (not its code): upper[f]
 * is A[owner[f], neighbour[f]], lower[f] is A[neighbour[f], owner[f]], the
 * diagonal is diag[]; relres is the true ||b - A x||_2 / ||b||_2 recomputed
 * at exit; iters counts the products A*(search direction) of the loop.
 * Status: 0 converged, 1 not converged within the iteration cap,
 * -1 bad argument, -3 breakdown (the matrix is not SPD), -6 out of memory.
 *
 * Two builds of this one source: the plain single-threaded one (the oracle
 * the tests pin and compare against) and, compiled with -fopenmp, a build
 * whose Jacobi-PCG (or_pcg only) spreads its cell loops over the host cores:
 * the face loop of the product becomes a loop over cells, each row summing
 * the faces that touch it in increasing face order, which is the order in
 * which the face loop adds them, so both builds form bitwise the same A x;
 * only the dot products' summation order differs.  The OpenMP build serves
 * the benchmark's multi-core CPU baseline and its tight reference solutions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_BAD_ARG (-1)
#define OR_NOT_SPD (-3)
#define OR_OOM (-6)

/* ---- FP64 building blocks ------------------------------------------------ */

/* y = A x: the diagonal, then every internal face adds its two off-diagonal
 * products, upper to the owner's row and lower to the neighbour's row. */
void or_spmv(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
             const double *diag, const double *upper, const double *lower,
             const double *x, double *y)
{
    for (int64_t i = 0; i < n; i++)
        y[i] = diag[i] * x[i];
    for (int64_t f = 0; f < nf; f++) {
        y[own[f]] += upper[f] * x[nbr[f]];
        y[nbr[f]] += lower[f] * x[own[f]];
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += a[i] * b[i];
    return s;
}

/* z = M^-1 r with M = diag(A) (Jacobi), or z = r without a preconditioner. */
static void precond(int64_t n, int use_jacobi, const double *diag, const double *r, double *z)
{
    for (int64_t i = 0; i < n; i++)
        z[i] = use_jacobi ? r[i] / diag[i] : r[i];
}

/* r = b - A x */
static void residual(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                     const double *diag, const double *upper, const double *lower,
                     const double *b, const double *x, double *r)
{
    or_spmv(n, nf, own, nbr, diag, upper, lower, x, r);
    for (int64_t i = 0; i < n; i++)
        r[i] = b[i] - r[i];
}

double or_true_relres(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                      const double *diag, const double *upper, const double *lower,
                      const double *b, const double *x)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r)
        return NAN;
    residual(n, nf, own, nbr, diag, upper, lower, b, x, r);
    double bn = sqrt(dot(n, b, b));
    double rn = sqrt(dot(n, r, r));
    free(r);
    return bn > 0.0 ? rn / bn : rn;
}

/* ---- the operator of one Jacobi-PCG solve ----------------------------------
 * Plain build: A x is or_spmv's face loop, dots and updates are plain loops.
 * OpenMP build: rows are formed independently from the list of faces that
 * touch each cell (built once per solve, faces in increasing order, so each
 * row adds its face terms in the face loop's order) and every cell loop is
 * shared among the threads; dot products are OpenMP sum reductions. */
typedef struct {
    int64_t n, nf;
    const int32_t *own, *nbr;
    const double *diag, *upper, *lower;
#ifdef _OPENMP
    int64_t *rstart;   /* [n + 1]: faces of cell i are rface[rstart[i] .. rstart[i+1]) */
    int64_t *rface;    /* [2 nf]: 2 f + 1 where the cell is the face's neighbour (lower) */
#endif
} pcg_op;

static int op_init(pcg_op *A, int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                   const double *diag, const double *upper, const double *lower)
{
    A->n = n; A->nf = nf; A->own = own; A->nbr = nbr;
    A->diag = diag; A->upper = upper; A->lower = lower;
#ifdef _OPENMP
    A->rstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    A->rface = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * nf > 0 ? 2 * nf : 1));
    if (!A->rstart || !A->rface) {
        free(A->rstart); free(A->rface);
        return OR_OOM;
    }
    for (int64_t f = 0; f < nf; f++) {
        A->rstart[own[f] + 1]++;
        A->rstart[nbr[f] + 1]++;
    }
    for (int64_t i = 0; i < n; i++)
        A->rstart[i + 1] += A->rstart[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) {
        free(A->rstart); free(A->rface);
        return OR_OOM;
    }
    for (int64_t i = 0; i < n; i++)
        fill[i] = A->rstart[i];
    for (int64_t f = 0; f < nf; f++) {
        A->rface[fill[own[f]]++] = 2 * f;
        A->rface[fill[nbr[f]]++] = 2 * f + 1;
    }
    free(fill);
#endif
    return OR_OK;
}

static void op_free(pcg_op *A)
{
#ifdef _OPENMP
    free(A->rstart);
    free(A->rface);
#else
    (void)A;
#endif
}

static void op_spmv(const pcg_op *A, const double *x, double *y)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; i++) {
        double s = A->diag[i] * x[i];
        for (int64_t e = A->rstart[i]; e < A->rstart[i + 1]; e++) {
            int64_t f = A->rface[e] >> 1;
            if (A->rface[e] & 1)
                s += A->lower[f] * x[A->own[f]];
            else
                s += A->upper[f] * x[A->nbr[f]];
        }
        y[i] = s;
    }
#else
    or_spmv(A->n, A->nf, A->own, A->nbr, A->diag, A->upper, A->lower, x, y);
#endif
}

static double op_dot(const pcg_op *A, const double *a, const double *b)
{
    double s = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : s)
#endif
    for (int64_t i = 0; i < A->n; i++)
        s += a[i] * b[i];
    return s;
}

/* r = b - A x */
static void op_residual(const pcg_op *A, const double *b, const double *x, double *r)
{
    op_spmv(A, x, r);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < A->n; i++)
        r[i] = b[i] - r[i];
}

/* z = M^-1 r with M = diag(A) (Jacobi), or z = r without a preconditioner;
 * then p = z when p is given */
static void op_precond(const pcg_op *A, int use_jacobi, const double *r, double *z, double *p)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < A->n; i++) {
        z[i] = use_jacobi ? r[i] / A->diag[i] : r[i];
        if (p)
            p[i] = z[i];
    }
}

/* Set the number of threads of this build's solves (ignored by the plain build). */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of threads the solves of this build use (1 for the plain build). */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Jacobi-preconditioned CG (Saad, Iterative Methods, Alg. 9.1) ---------
 * Stops when the recursively updated ||r||/||b|| reaches tol; the residual
 * is then recomputed as b - A x, and if that true residual is still above
 * tol it replaces r and the search restarts from p = M^-1 r.
 * hist (optional, maxit+1 entries) receives the recursive relres per step.
 * ab (optional, 2 maxit entries) receives alpha_k and beta_k of every step k
 * (beta_k = 0 where the search restarted): the coefficients of the Lanczos
 * tridiagonal matrix of M^-1 A that CG builds implicitly (Saad, Sec. 6.7.3). */
int or_pcg(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
           const double *diag, const double *upper, const double *lower,
           const double *b, double *x, double tol, int maxit, int use_jacobi,
           int *iters, double *relres, double *hist, double *ab)
{
    if (n < 0 || nf < 0 || maxit < 0 || !(tol >= 0.0))
        return OR_BAD_ARG;
    *iters = 0;
    pcg_op A;
    if (op_init(&A, n, nf, own, nbr, diag, upper, lower) != OR_OK)
        return OR_OOM;
    double bnorm = sqrt(op_dot(&A, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; i++)
            x[i] = 0.0;
        *relres = 0.0;
        op_free(&A);
        return OR_OK;
    }
    size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(bytes), *z = (double *)malloc(bytes);
    double *p = (double *)malloc(bytes), *q = (double *)malloc(bytes);
    if (!r || !z || !p || !q) {
        free(r); free(z); free(p); free(q);
        op_free(&A);
        return OR_OOM;
    }
    int status = OR_NOT_CONVERGED, it = 0;
    op_residual(&A, b, x, r);
    double rnorm = sqrt(op_dot(&A, r, r));
    if (hist)
        hist[0] = rnorm / bnorm;
    if (rnorm / bnorm <= tol) {
        status = OR_OK;
        goto done;
    }
    op_precond(&A, use_jacobi, r, z, p);
    double rz = op_dot(&A, r, z);
    for (;;) {
        if (it >= maxit) {
            status = OR_NOT_CONVERGED;
            break;
        }
        op_spmv(&A, p, q);
        double pq = op_dot(&A, p, q);
        if (!(pq > 0.0)) {
            status = OR_NOT_SPD;
            break;
        }
        double alpha = rz / pq;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        if (ab) {
            ab[2 * it] = alpha;
            ab[2 * it + 1] = 0.0;
        }
        it++;
        rnorm = sqrt(op_dot(&A, r, r));
        if (hist)
            hist[it] = rnorm / bnorm;
        if (rnorm / bnorm <= tol) {
            op_residual(&A, b, x, r);
            rnorm = sqrt(op_dot(&A, r, r));
            if (rnorm / bnorm <= tol) {
                status = OR_OK;
                break;
            }
            op_precond(&A, use_jacobi, r, z, p);
            rz = op_dot(&A, r, z);
            continue;
        }
        op_precond(&A, use_jacobi, r, z, NULL);
        double rz_new = op_dot(&A, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        if (ab)
            ab[2 * it - 1] = beta;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < n; i++)
            p[i] = z[i] + beta * p[i];
    }
done:
    *iters = it;
    *relres = or_true_relres(n, nf, own, nbr, diag, upper, lower, b, x);
    free(r); free(z); free(p); free(q);
    op_free(&A);
    return status;
}

/* ---- pipelined preconditioned CG (Ghysels & Vanroose, Parallel Computing
 * 40 (2014), preconditioned pipelined CG) -------------------------------------
 * One reduction per iteration gives gamma = (r,u), delta = (w,u) and ||r||^2;
 * the products m = M^-1 w and n = A m do not depend on them.
 *   beta  = gamma / gamma_old,  alpha = gamma / (delta - beta*gamma/alpha_old)
 *   (first iteration: beta = 0, alpha = gamma / delta)
 *   z = n + beta z,  q = m + beta q,  s = w + beta s,  p = u + beta p
 *   x += alpha p,  r -= alpha s,  u -= alpha q,  w -= alpha z
 * Residual replacement: whenever the recursive ||r||/||b|| reaches tol (and,
 * if rr_period > 0, every rr_period iterations) the recurrences are reset
 * from the true residual: r = b - A x, u = M^-1 r, w = A u, s = A p,
 * q = M^-1 s, z = A q.  The solve ends only on a replaced (true) residual.
 * Rounding can drive the denominator delta - beta*gamma/alpha_old (which is
 * (p, A p) in exact arithmetic) to zero or below once the recurrences have
 * drifted; that is treated as a loss of accuracy, not indefiniteness: the
 * vectors are replaced from the true residual and the method restarts with
 * beta = 0.  Only a non-positive delta = (A u, u) on a fresh start means
 * the matrix is not SPD. */
static void pipe_replace(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                         const double *diag, const double *upper, const double *lower,
                         const double *b, const double *x, const double *p,
                         double *r, double *u, double *w, double *s, double *q, double *z)
{
    residual(n, nf, own, nbr, diag, upper, lower, b, x, r);
    precond(n, 1, diag, r, u);
    or_spmv(n, nf, own, nbr, diag, upper, lower, u, w);
    or_spmv(n, nf, own, nbr, diag, upper, lower, p, s);
    precond(n, 1, diag, s, q);
    or_spmv(n, nf, own, nbr, diag, upper, lower, q, z);
}

int or_pipecg(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
              const double *diag, const double *upper, const double *lower,
              const double *b, double *x, double tol, int maxit, int rr_period,
              int *iters, double *relres, double *hist)
{
    if (n < 0 || nf < 0 || maxit < 0 || !(tol >= 0.0))
        return OR_BAD_ARG;
    *iters = 0;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; i++)
            x[i] = 0.0;
        *relres = 0.0;
        return OR_OK;
    }
    size_t bytes = sizeof(double) * (size_t)n;
    double *v[9];
    for (int k = 0; k < 9; k++) {
        v[k] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!v[k]) {
            for (int j = 0; j < k; j++)
                free(v[j]);
            return OR_OOM;
        }
    }
    (void)bytes;
    double *r = v[0], *u = v[1], *w = v[2], *m = v[3], *nv = v[4];
    double *z = v[5], *q = v[6], *s = v[7], *p = v[8];

    residual(n, nf, own, nbr, diag, upper, lower, b, x, r);
    precond(n, 1, diag, r, u);
    or_spmv(n, nf, own, nbr, diag, upper, lower, u, w);

    int status = OR_NOT_CONVERGED, it = 0, since = 0, fresh = 1;
    double gamma_old = 0.0, alpha_old = 0.0;
    for (;;) {
        double gamma = dot(n, r, u);
        double delta = dot(n, w, u);
        double rr = dot(n, r, r);
        if (hist)
            hist[it] = sqrt(rr) / bnorm;
        int replace = sqrt(rr) / bnorm <= tol || (rr_period > 0 && since >= rr_period);
        if (replace) {
            pipe_replace(n, nf, own, nbr, diag, upper, lower, b, x, p, r, u, w, s, q, z);
            since = 0;
            gamma = dot(n, r, u);
            delta = dot(n, w, u);
            rr = dot(n, r, r);
            if (sqrt(rr) / bnorm <= tol) {
                status = OR_OK;
                break;
            }
        }
        if (it >= maxit) {
            status = OR_NOT_CONVERGED;
            break;
        }
        precond(n, 1, diag, w, m);
        or_spmv(n, nf, own, nbr, diag, upper, lower, m, nv);
        double beta, alpha, denom;
        if (fresh) {
            beta = 0.0;
            denom = delta;
        } else {
            beta = gamma / gamma_old;
            denom = delta - beta * gamma / alpha_old;
        }
        if (!(denom > 0.0) || !(gamma > 0.0)) {
            if (fresh) {
                status = OR_NOT_SPD;
                break;
            }
            pipe_replace(n, nf, own, nbr, diag, upper, lower, b, x, p, r, u, w, s, q, z);
            since = 0;
            fresh = 1;
            continue;
        }
        fresh = 0;
        alpha = gamma / denom;
        for (int64_t i = 0; i < n; i++) {
            z[i] = nv[i] + beta * z[i];
            q[i] = m[i] + beta * q[i];
            s[i] = w[i] + beta * s[i];
            p[i] = u[i] + beta * p[i];
            x[i] += alpha * p[i];
            r[i] -= alpha * s[i];
            u[i] -= alpha * q[i];
            w[i] -= alpha * z[i];
        }
        gamma_old = gamma;
        alpha_old = alpha;
        it++;
        since++;
    }
    *iters = it;
    *relres = or_true_relres(n, nf, own, nbr, diag, upper, lower, b, x);
    for (int k = 0; k < 9; k++)
        free(v[k]);
    return status;
}

/* ---- FP32 building blocks for the mixed-precision solve ----------------- */

static void spmv32(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                   const float *diag, const float *upper, const float *lower,
                   const float *x, float *y)
{
    for (int64_t i = 0; i < n; i++)
        y[i] = diag[i] * x[i];
    for (int64_t f = 0; f < nf; f++) {
        y[own[f]] += upper[f] * x[nbr[f]];
        y[nbr[f]] += lower[f] * x[own[f]];
    }
}

/* FP32 products summed in double */
static double dot32(int64_t n, const float *a, const float *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += (double)(a[i] * b[i]);
    return s;
}

/* ---- mixed precision: FP32 pipelined PCG with FP64 residual replacement ----
 * The pipelined Jacobi-PCG recurrences above run in float (matrix rounded
 * to float; vector updates in float; dot products summed in double; alpha
 * and beta in double, rounded to float where they scale a vector).  FP64 is
 * used only for the solution accumulation and the true residual: at a
 * replacement the float correction xc is folded into the FP64 solution,
 * x += sigma*xc, the residual r64 = b - A x is formed in FP64 and tested
 * against tol, and the float recurrences are re-seeded from it,
 *   r = r64/sigma, u = M^-1 r, w = A u, s = A p, q = M^-1 s, z = A q,
 * where sigma is the power of two nearest sqrt(r64, M^-1 r64) (so rescaling
 * is exact) and p, gamma_old are rescaled by the change of sigma.
 * A replacement happens
 *   - every `period` float iterations (period > 0),
 *   - when gamma = (r,u) has dropped below tau^2 times its value at the last
 *     replacement (tau > 0),
 *   - when the predicted ||r||_2/||b||, sqrt(ratio*gamma)*sigma/||b|| with
 *     ratio = ||r64||^2/(r64, M^-1 r64) from the last replacement, reaches tol,
 *   - after a numerical breakdown (non-positive denominator; the method then
 *     restarts with beta = 0), and at the iteration cap.
 * With restart = 1 every replacement also restarts the search (p = 0,
 * beta = 0): that is classic defect correction, an FP32 inner solve of
 * A d = r to relative tolerance tau followed by x += d in FP64.  With
 * restart = 0 the search directions survive the replacement (a reliable
 * update), which keeps the Krylov convergence of the FP64 method.
 * iters counts float products A*m; replacements counts FP64 residuals,
 * including the initial one.  A non-positive delta on a fresh start
 * means the matrix is not SPD.
 *
 * deflate = 1 adds deflation of the constant vector W = 1 (deflated CG,
 * Saad, Yeung, Erhel and Guyomarc'h, SIAM J. Sci. Comput. 21 (2000), with
 * the Jacobi preconditioner, in pipelined form): with a1 = A W (FP64) and
 * c = (W, a1), every replacement first applies the coarse correction
 * x += (W, r64)/c W, r64 -= (W, r64)/c a1, and every step removes the
 * A-component of W from the new direction, mu = (a1, u)/c:
 *   p = u + beta p - mu W,  s = w + beta s - mu a1,
 *   q = m + beta q - mu M^-1 a1,  z = n + beta z - mu A M^-1 a1,
 * with denominator delta - beta*gamma/alpha_old - (a1, u)^2/c.  This takes
 * the near-null constant mode of pure-Neumann (pressure) systems out of the
 * float iteration, where the rounding of the float operator cannot resolve
 * it.  W, a1, M^-1 a1 and A M^-1 a1 are formed in FP64 and rounded to
 * float for the recurrences. */
/* Trace of or_mixed_pipecg_ex (for the tests that pin its control logic):
 * one record of OR_TRACE_LEN doubles per event,
 *   [0] iteration count at the event, [1] event: 0 step, 1 replacement,
 *   step:        [2] (a1, p)/(|a1| |p|) after the update (deflation; else 0),
 *                [3] gamma / gamma_ref of the fresh dot products,
 *                [4] the denominator alpha was formed with, divided by
 *                    (p, A p) of the new direction (FP64 matrix; equal in
 *                    exact arithmetic),
 *   replacement: [2] the predicted relres sqrt(ratio gamma) sigma/||b|| that
 *                    the trigger saw, [3] the true relres after the fold (and
 *                    coarse correction), [4] (W, r64)/(|W| |r64|) after the
 *                    coarse correction (deflation; else 0),
 *                [5] trigger bits: 1 forced (start or breakdown), 2 period,
 *                    4 tau drop, 8 predicted convergence, 16 iteration cap.
 * flags: OR_MIXED_SIGMA1 keeps the float unit sigma at 1 instead of the power
 * of two nearest sqrt(r64, M^-1 r64). */
#define OR_TRACE_LEN 6
#define OR_MIXED_SIGMA1 1

int or_mixed_pipecg_ex(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                       const double *diag, const double *upper, const double *lower,
                       const double *b, double *x, double tol, int period, double tau,
                       int restart, int deflate, int maxit, int *iters, int *replacements,
                       double *relres, int flags, double *trace, int trace_cap, int *trace_len)
{
    int ntr = 0;
    if (trace_len)
        *trace_len = 0;
    if (n < 0 || nf < 0 || maxit < 0 || period < 0 || !(tol >= 0.0) || !(tau >= 0.0))
        return OR_BAD_ARG;
    *iters = 0;
    *replacements = 0;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; i++)
            x[i] = 0.0;
        *relres = 0.0;
        return OR_OK;
    }
    size_t nn = (size_t)(n > 0 ? n : 1), ff = (size_t)(nf > 0 ? nf : 1);
    double *r64 = (double *)malloc(sizeof(double) * nn);
    double *a1 = (double *)malloc(sizeof(double) * nn);
    double *t64 = (double *)malloc(sizeof(double) * nn);
    float *d32 = (float *)malloc(sizeof(float) * nn);
    float *u32 = (float *)malloc(sizeof(float) * ff);
    float *l32 = (float *)malloc(sizeof(float) * ff);
    float *v[14] = {0};
    int ok = r64 && a1 && t64 && d32 && u32 && l32;
    for (int k = 0; k < 14 && ok; k++) {
        v[k] = (float *)calloc(nn, sizeof(float));
        ok = v[k] != NULL;
    }
    int status = OR_NOT_CONVERGED;
    if (!ok) {
        status = OR_OOM;
        goto out;
    }
    float *r = v[0], *u = v[1], *w = v[2], *m = v[3], *nv = v[4];
    float *z = v[5], *q = v[6], *s = v[7], *p = v[8], *xc = v[9];
    float *W32 = v[10], *a132 = v[11], *ma132 = v[12], *ama132 = v[13];
    for (int64_t i = 0; i < n; i++)
        d32[i] = (float)diag[i];
    for (int64_t f = 0; f < nf; f++) {
        u32[f] = (float)upper[f];
        l32[f] = (float)lower[f];
    }
    double cW = 1.0;
    if (deflate) {
        for (int64_t i = 0; i < n; i++)
            r64[i] = 1.0;                                   /* W = 1 */
        or_spmv(n, nf, own, nbr, diag, upper, lower, r64, a1);   /* a1 = A W */
        cW = 0.0;
        for (int64_t i = 0; i < n; i++)
            cW += a1[i];                                    /* (W, A W) */
        if (!(cW > 0.0)) {
            status = OR_NOT_SPD;
            goto out;
        }
        for (int64_t i = 0; i < n; i++)
            r64[i] = a1[i] / diag[i];                       /* M^-1 a1 */
        or_spmv(n, nf, own, nbr, diag, upper, lower, r64, t64);  /* A M^-1 a1 */
        for (int64_t i = 0; i < n; i++) {
            W32[i] = 1.0f;
            a132[i] = (float)a1[i];
            ma132[i] = (float)r64[i];
            ama132[i] = (float)t64[i];
        }
    }
    double sigma = 1.0, ratio = 1.0, gamma_old = 0.0, alpha_old = 0.0, gamma_ref = 0.0;
    int it = 0, since = 0, fresh = 1, force = 1, nrep = 0;
    for (;;) {
        double gamma = dot32(n, r, u);
        double delta = dot32(n, w, u);
        double eps = deflate ? dot32(n, a132, u) : 0.0;
        double predicted = sqrt(ratio * gamma) * sigma / bnorm;
        int trigger = (force ? 1 : 0) | ((period > 0 && since >= period) ? 2 : 0)
                      | ((tau > 0.0 && gamma <= tau * tau * gamma_ref) ? 4 : 0)
                      | (predicted <= tol ? 8 : 0) | (it >= maxit ? 16 : 0);
        if (trigger) {
            for (int64_t i = 0; i < n; i++) {
                x[i] += sigma * (double)xc[i];
                xc[i] = 0.0f;
            }
            residual(n, nf, own, nbr, diag, upper, lower, b, x, r64);
            if (deflate) {
                double a0 = 0.0;
                for (int64_t i = 0; i < n; i++)
                    a0 += r64[i];                           /* (W, r64) */
                a0 /= cW;
                for (int64_t i = 0; i < n; i++) {
                    x[i] += a0;
                    r64[i] -= a0 * a1[i];
                }
            }
            nrep++;
            double rn2 = dot(n, r64, r64);
            *relres = sqrt(rn2) / bnorm;
            if (trace && ntr < trace_cap) {
                double *t = trace + (size_t)OR_TRACE_LEN * ntr++;
                double wr = 0.0;
                if (deflate) {
                    for (int64_t i = 0; i < n; i++)
                        wr += r64[i];                       /* (W, r64), W = 1 */
                    wr /= sqrt((double)n) * sqrt(rn2) + 1e-300;
                }
                t[0] = it; t[1] = 1; t[2] = predicted; t[3] = *relres; t[4] = wr;
                t[5] = trigger;
            }
            if (*relres <= tol) {
                status = OR_OK;
                break;
            }
            if (it >= maxit) {
                status = OR_NOT_CONVERGED;
                break;
            }
            double g64 = 0.0;
            for (int64_t i = 0; i < n; i++)
                g64 += r64[i] * r64[i] / diag[i];
            if (!(g64 > 0.0)) {
                status = OR_NOT_SPD;
                break;
            }
            ratio = rn2 / g64;
            double sigma_new = (flags & OR_MIXED_SIGMA1) ? 1.0 : exp2(round(log2(sqrt(g64))));
            if (restart) {
                for (int64_t i = 0; i < n; i++)
                    p[i] = 0.0f;
                fresh = 1;
            } else {
                float f = (float)(sigma / sigma_new);
                for (int64_t i = 0; i < n; i++)
                    p[i] *= f;
                gamma_old *= (double)f * (double)f;
            }
            sigma = sigma_new;
            for (int64_t i = 0; i < n; i++) {
                r[i] = (float)(r64[i] / sigma);
                u[i] = r[i] / d32[i];
            }
            spmv32(n, nf, own, nbr, d32, u32, l32, u, w);
            spmv32(n, nf, own, nbr, d32, u32, l32, p, s);
            for (int64_t i = 0; i < n; i++)
                q[i] = s[i] / d32[i];
            spmv32(n, nf, own, nbr, d32, u32, l32, q, z);
            gamma = dot32(n, r, u);
            delta = dot32(n, w, u);
            eps = deflate ? dot32(n, a132, u) : 0.0;
            gamma_ref = gamma;
            since = 0;
            force = 0;
        }
        for (int64_t i = 0; i < n; i++)
            m[i] = w[i] / d32[i];
        spmv32(n, nf, own, nbr, d32, u32, l32, m, nv);
        double beta, denom;
        if (fresh) {
            beta = 0.0;
            denom = delta;
        } else {
            beta = gamma / gamma_old;
            denom = delta - beta * gamma / alpha_old;
        }
        if (deflate)
            denom -= eps * eps / cW;
        if (!(denom > 0.0) || !(gamma > 0.0)) {
            if (fresh) {
                status = OR_NOT_SPD;
                break;
            }
            fresh = 1;
            force = 1;
            continue;
        }
        fresh = 0;
        double alpha = gamma / denom;
        float a = (float)alpha, bt = (float)beta, mu = (float)(eps / cW);
        for (int64_t i = 0; i < n; i++) {
            z[i] = nv[i] + bt * z[i];
            q[i] = m[i] + bt * q[i];
            s[i] = w[i] + bt * s[i];
            p[i] = u[i] + bt * p[i];
            if (deflate) {
                z[i] -= mu * ama132[i];
                q[i] -= mu * ma132[i];
                s[i] -= mu * a132[i];
                p[i] -= mu * W32[i];
            }
            xc[i] += a * p[i];
            r[i] -= a * s[i];
            u[i] -= a * q[i];
            w[i] -= a * z[i];
        }
        if (trace && ntr < trace_cap) {
            double *t = trace + (size_t)OR_TRACE_LEN * ntr++;
            double ap = 0.0, aa = 0.0, pp = 0.0, pap = 0.0;
            if (deflate) {
                for (int64_t i = 0; i < n; i++) {
                    ap += a1[i] * (double)p[i];
                    aa += a1[i] * a1[i];
                    pp += (double)p[i] * (double)p[i];
                }
                ap /= sqrt(aa) * sqrt(pp) + 1e-300;
            }
            for (int64_t i = 0; i < n; i++)
                t64[i] = (double)p[i];
            or_spmv(n, nf, own, nbr, diag, upper, lower, t64, r64);
            for (int64_t i = 0; i < n; i++)
                pap += t64[i] * r64[i];
            t[0] = it + 1; t[1] = 0; t[2] = ap; t[3] = gamma_ref > 0.0 ? gamma / gamma_ref : 0.0;
            t[4] = denom / pap; t[5] = 0.0;
        }
        gamma_old = gamma;
        alpha_old = alpha;
        it++;
        since++;
    }
    *iters = it;
    *replacements = nrep;
    if (trace_len)
        *trace_len = ntr;
out:
    free(r64); free(a1); free(t64); free(d32); free(u32); free(l32);
    for (int k = 0; k < 14; k++)
        free(v[k]);
    return status;
}

int or_mixed_pipecg(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                    const double *diag, const double *upper, const double *lower,
                    const double *b, double *x, double tol, int period, double tau,
                    int restart, int deflate, int maxit, int *iters, int *replacements,
                    double *relres)
{
    return or_mixed_pipecg_ex(n, nf, own, nbr, diag, upper, lower, b, x, tol, period, tau,
                              restart, deflate, maxit, iters, replacements, relres, 0, NULL, 0,
                              NULL);
}

/* ---- adjoint face gradient ------------------------------------------------
 * With A symmetric and c_f the coefficient of internal face f (upper = lower
 * = -c_f, +c_f on both diagonals), L(x(c)) and lambda = A^-T dL/dx give
 * dL/dc_f = -(lambda_o - lambda_n)(x_o - x_n). */
void or_face_grad(int64_t nf, const int32_t *own, const int32_t *nbr,
                  const double *lambda, const double *x, double *grad)
{
    for (int64_t f = 0; f < nf; f++)
        grad[f] = -(lambda[own[f]] - lambda[nbr[f]]) * (x[own[f]] - x[nbr[f]]);
}

/* Gradient of L(x(A)) with respect to each stored entry of an LDU matrix
 * taken as independent (upper and lower need not stay equal): differentiating
 * A x = b gives dx = -A^-1 dA x, so dL/dA_ij = -lambda_i x_j with
 * lambda = A^-T dL/dx.  upper[f] = A[o, n], lower[f] = A[n, o], diag = A[i, i]. */
void or_value_grad(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                   const double *lambda, const double *x, double *ddiag, double *dup,
                   double *dlo)
{
    for (int64_t i = 0; i < n; i++)
        ddiag[i] = -lambda[i] * x[i];
    for (int64_t f = 0; f < nf; f++) {
        dup[f] = -lambda[own[f]] * x[nbr[f]];
        dlo[f] = -lambda[nbr[f]] * x[own[f]];
    }
}

/* ---- cell diffusivity -> face coefficients (harmonic mean) -----------------
 * The FVM Laplacian's face coefficient is c_f = g_f k_f with the harmonic
 * mean k_f = 2 k_o k_n / (k_o + k_n) of the two cells' diffusivities and a
 * geometric factor g_f = |S_f| / |d_on|; a Dirichlet wall adds k_P bfac_P to
 * the diagonal of its cell (bfac_P = 2 |S_b| / w_P summed over the cell's
 * Dirichlet faces). */
void or_harmonic_coeffs(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                        const double *k, const double *g, const double *bfac,
                        double *coef, double *extra)
{
    for (int64_t f = 0; f < nf; f++) {
        double ko = k[own[f]], kn = k[nbr[f]];
        coef[f] = g[f] * (2.0 * ko * kn / (ko + kn));
    }
    for (int64_t i = 0; i < n; i++)
        extra[i] = k[i] * bfac[i];
}

/* Chain rule of the map above: given dL/dc_f and dL/dextra_P,
 *   dL/dk_P = sum over the faces f of P of dL/dc_f g_f dk_f/dk_P
 *             + dL/dextra_P bfac_P,
 * with dk_f/dk_o = 2 k_n^2 / (k_o + k_n)^2 (and symmetrically for n).
 * Face loop, each face adding to both of its cells. */
void or_harmonic_grad(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                      const double *k, const double *g, const double *bfac,
                      const double *dcoef, const double *dextra, double *dk)
{
    for (int64_t i = 0; i < n; i++)
        dk[i] = dextra[i] * bfac[i];
    for (int64_t f = 0; f < nf; f++) {
        double ko = k[own[f]], kn = k[nbr[f]], s = ko + kn;
        double w = dcoef[f] * g[f] * 2.0 / (s * s);
        dk[own[f]] += w * kn * kn;
        dk[nbr[f]] += w * ko * ko;
    }
}

/* ---- dense LU with partial pivoting (row-major, n x n, A and b overwritten;
 * the solution is returned in b).  For tiny systems only. */
int or_lu_solve(int64_t n, double *A, double *b)
{
    for (int64_t k = 0; k < n; k++) {
        int64_t piv = k;
        double best = fabs(A[k * n + k]);
        for (int64_t i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > best) {
                best = fabs(A[i * n + k]);
                piv = i;
            }
        if (best == 0.0)
            return OR_NOT_SPD;
        if (piv != k) {
            for (int64_t j = 0; j < n; j++) {
                double t = A[k * n + j];
                A[k * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int64_t i = k + 1; i < n; i++) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int64_t j = k + 1; j < n; j++)
                A[i * n + j] -= l * A[k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int64_t j = i + 1; j < n; j++)
            s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    return OR_OK;
}
