/* A plain C caller of libldupcg (no Python, no torch): assembles the 7-point
 * finite-volume Laplacian of an 8 x 8 x 8 box in LDU form on the host
 * (Dirichlet walls at x = 0 and x = 1), copies it to the GPU with the CUDA
 * runtime, and solves A x = b with FP64 Jacobi-PCG, the mixed pipelined
 * method and AMG-preconditioned CG, checking each true relative residual on
 * the host.  Exit status 0 when every solve meets the tolerance. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "ldupcg.h"

#define N1 8
#define NC (N1 * N1 * N1)

static int check(int st, const char *what) {
    if (st != LDU_OK) {
        fprintf(stderr, "%s: %s (%d)\n", what, ldu_status_string(st), st);
        return 1;
    }
    return 0;
}

int main(void) {
    static int32_t own[3 * NC], nbr[3 * NC];
    static double diag[NC], up[3 * NC], lo[3 * NC], b[NC], x[NC];
    int64_t nf = 0;
    for (int k = 0; k < N1; ++k)
        for (int j = 0; j < N1; ++j)
            for (int i = 0; i < N1; ++i) {
                const int c = i + N1 * (j + N1 * k);
                diag[c] = (i == 0 || i == N1 - 1) ? 2.0 : 0.0;   /* Dirichlet half-cell terms */
                b[c] = sin(0.37 * c) + 0.5;
            }
    for (int c = 0; c < NC; ++c) {
        const int i = c % N1, j = (c / N1) % N1, k = c / (N1 * N1);
        const int nb[3] = {i + 1 < N1 ? c + 1 : -1, j + 1 < N1 ? c + N1 : -1,
                           k + 1 < N1 ? c + N1 * N1 : -1};
        for (int a = 0; a < 3; ++a)
            if (nb[a] >= 0) {
                own[nf] = c;
                nbr[nf] = nb[a];
                up[nf] = lo[nf] = -1.0;
                diag[c] += 1.0;
                diag[nb[a]] += 1.0;
                ++nf;
            }
    }
    int32_t *d_own, *d_nbr;
    double *d_diag, *d_up, *d_lo, *d_b, *d_x;
    cudaMalloc((void **)&d_own, sizeof(int32_t) * nf);
    cudaMalloc((void **)&d_nbr, sizeof(int32_t) * nf);
    cudaMalloc((void **)&d_diag, sizeof(double) * NC);
    cudaMalloc((void **)&d_up, sizeof(double) * nf);
    cudaMalloc((void **)&d_lo, sizeof(double) * nf);
    cudaMalloc((void **)&d_b, sizeof(double) * NC);
    cudaMalloc((void **)&d_x, sizeof(double) * NC);
    cudaMemcpy(d_own, own, sizeof(int32_t) * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(d_nbr, nbr, sizeof(int32_t) * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(d_diag, diag, sizeof(double) * NC, cudaMemcpyHostToDevice);
    cudaMemcpy(d_up, up, sizeof(double) * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(d_lo, lo, sizeof(double) * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(d_b, b, sizeof(double) * NC, cudaMemcpyHostToDevice);

    int fails = 0;
    ldu_matrix *A = NULL;
    fails += check(ldu_create(NC, nf, d_own, d_nbr, d_diag, d_up, d_lo, NULL, NULL, &A),
                   "ldu_create");
    ldu_amg *M = NULL;
    fails += check(ldu_amg_create(NC, nf, d_own, d_nbr, d_diag, d_up, d_lo, NULL, NULL, &M),
                   "ldu_amg_create");
    if (fails)
        return 1;
    const double tol = 1e-10;
    for (int solver = 0; solver < 3; ++solver) {
        int iters = 0;
        double relres = 0.0;
        cudaMemset(d_x, 0, sizeof(double) * NC);
        int st;
        const char *name;
        if (solver == 0) {
            name = "pcg_solve";
            st = pcg_solve(A, d_b, d_x, tol, 1000, &iters, &relres, NULL);
        } else if (solver == 1) {
            name = "pipecg_solve(mixed)";
            st = pipecg_solve(A, d_b, d_x, tol, 1000, LDU_MIXED, NULL, &iters, &relres, NULL);
        } else {
            name = "amg_pcg_solve";
            st = amg_pcg_solve(M, d_b, d_x, tol, 100, LDU_FP64, &iters, &relres, NULL);
        }
        fails += check(st, name);
        cudaMemcpy(x, d_x, sizeof(double) * NC, cudaMemcpyDeviceToHost);
        /* the true residual ||b - A x|| / ||b||, from the host arrays */
        double rn = 0.0, bn = 0.0;
        static double r[NC];
        for (int c = 0; c < NC; ++c)
            r[c] = b[c] - diag[c] * x[c];
        for (int64_t f = 0; f < nf; ++f) {
            r[own[f]] -= up[f] * x[nbr[f]];
            r[nbr[f]] -= lo[f] * x[own[f]];
        }
        for (int c = 0; c < NC; ++c) {
            rn += r[c] * r[c];
            bn += b[c] * b[c];
        }
        const double true_rel = sqrt(rn / bn);
        printf("%-22s iterations %4d  relres %.3e  host-checked %.3e\n", name, iters, relres,
               true_rel);
        if (!(true_rel <= tol * 1.01))
            ++fails;
    }
    ldu_amg_destroy(M);
    ldu_destroy(A);
    cudaFree(d_own);
    cudaFree(d_nbr);
    cudaFree(d_diag);
    cudaFree(d_up);
    cudaFree(d_lo);
    cudaFree(d_b);
    cudaFree(d_x);
    if (fails == 0)
        printf("c abi ok\n");
    return fails ? 1 : 0;
}
