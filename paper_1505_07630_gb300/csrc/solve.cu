// solve.cu -- persistent cooperative kernels of the three solvers.
//
// Every solver works on the symmetrically scaled system
//     Ahat xhat = bhat,   Ahat = D^-1/2 A D^-1/2,  xhat = D^1/2 x,  bhat = D^-1/2 b,
// on which plain CG produces the iterates of Jacobi-preconditioned CG on A
// (M = D) in exact arithmetic: rhat = D^-1/2 r, phat = D^1/2 p, and
// (rhat, rhat) = (r, M^-1 r).  The stopping test uses the true-space norm
// ||r||_2^2 = sum_i d_i rhat_i^2.
//
// One block owns a contiguous range of slices; a "pass" is one sweep of every
// block over its range, ended by a grid barrier.  Dot products are summed per
// block in a fixed order into a slot, and after the barrier every block sums
// all slots in the same order, so every block takes the same decisions and
// results do not vary from run to run.
//
//   pcg64   Jacobi-PCG (Eq. 9; Saad Alg. 9.1), FP64, 3 passes / iteration:
//           q = Ahat p | x += a p, r -= a q | p = r + b p
//   pipe64  pipelined PCG (Sec. 4.1; Ghysels & Vanroose), FP64, 1 pass /
//           iteration: the product n = Ahat w uses only w, which is complete
//           at the barrier that also completes the reduction, so product,
//           all eight recurrences and the next dot products share one sweep;
//           w is double-buffered because neighbours gather it while it is
//           rewritten.  Residual replacement: 3 passes.
//   mixed   the same pipelined sweep in float; FP64 holds the solution and
//           the periodic true residual (4 passes per replacement).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ldupcg_impl.cuh"

using namespace ldu;

#include "solve_kernels.cuh"

namespace {

// ---------------------------------------------------------------------------
// host side

enum Kind { kPcg = 0, kPipe = 1, kMixed = 2, kMixedDeflated = 3 };

template <int R>
const void *kernel_ptr(Kind k) {
    switch (k) {
    case kPcg: return (const void *)k_pcg64<R, Batch<R>::pcg>;
    case kPipe: return (const void *)k_pipe64<R, Batch<R>::pipe>;
    case kMixed: return (const void *)k_mixed<R, Batch<R>::mixed, false>;
    default: return (const void *)k_mixed<R, Batch<R>::mixed, true>;
    }
}

const void *pick_kernel(const ldu_matrix *A, Kind k) {
    switch (A->C) {
    case 32: return kernel_ptr<1>(k);
    case 64: return kernel_ptr<2>(k);
    default: return kernel_ptr<4>(k);
    }
}

int map_status(int dev) {
    switch (dev) {
    case kDevOk: return LDU_OK;
    case kDevNotConverged: return LDU_NOT_CONVERGED;
    case kDevNotSpd: return LDU_ERR_NOT_SPD;
    case kDevTimeout: return LDU_ERR_BARRIER_TIMEOUT;
    default: return LDU_ERR_CUDA;
    }
}

int run_solver(const ldu_matrix *Ac, Kind kind, const double *b, double *x, double tol, int maxit,
               const pcg_opts *o, int *iters, double *relres, cudaStream_t st) {
    ldu_matrix *A = const_cast<ldu_matrix *>(Ac);
    if (!A || maxit < 0 || !(tol >= 0.0) || (A->n > 0 && (!b || !x)))
        return LDU_ERR_BAD_ARG;
    pcg_opts opt{};
    if (o)
        opt = *o;
    if (opt.rr_period < 0 || opt.tau < 0.0 || opt.barrier_timeout_s < 0.0 ||
        (opt.deflate != 0 && opt.deflate != 1))
        return LDU_ERR_BAD_ARG;
    if (kind == kMixed && opt.rr_period == 0 && !o)
        opt.rr_period = 16;
    if (kind == kMixed && o && o->rr_period == 0 && o->tau == 0.0)
        opt.rr_period = 16;
    A->last = ldu_solve_stats{};
    if (A->n == 0) {
        if (iters)
            *iters = 0;
        if (relres)
            *relres = 0.0;
        A->last.status = LDU_OK;
        return LDU_OK;
    }
    const void *kern = pick_kernel(A, (kind == kMixed && opt.deflate) ? kMixedDeflated : kind);
    int grid = 0;
    size_t smem = 0;
    int rc = grid_for(A, kern, A->block_threads, &grid, &smem);
    if (rc != LDU_OK)
        return rc;
    SolveParams P;
    P.A = view_of(A);
    P.A.meta_smem = smem > 0;
    P.sync.count = A->bar_count;
    P.sync.err = A->bar_err;
    const double tmo = opt.barrier_timeout_s > 0.0 ? opt.barrier_timeout_s : 10.0;
    P.sync.timeout_ns = (unsigned long long)(tmo * 1e9);
    P.slots = A->slots;
    P.tasks = nullptr;
    P.out = A->out_dev;
    P.b = b;
    P.x = x;
    for (int k = 0; k < 10; ++k)
        P.v64[k] = A->v64[k];
    for (int k = 0; k < 10; ++k)
        P.v32[k] = A->v32[k];
    P.tol = tol;
    P.maxit = maxit;
    P.rr_period = opt.rr_period;
    P.tau = opt.tau;
    P.restart = opt.restart;
    P.deflate = kind == kMixed ? opt.deflate : 0;
    P.fault_inject = opt.fault_inject;
    cudaError_t e;
    if ((e = cudaMemsetAsync(A->bar_count, 0, sizeof(unsigned) * 64, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemsetAsync(A->bar_err, 0, sizeof(int) * 64, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemsetAsync(A->out_dev, 0xff, sizeof(SolveOut), st)) != cudaSuccess)
        return cuda_status(e);
    void *args[] = {&P};
    rc = launch_persistent(kern, grid, A->block_threads, args, smem, st);
    if (rc != LDU_OK)
        return rc;
    int flags_err[2] = {0, 0};
    if ((e = cudaMemcpyAsync(A->out_host, A->out_dev, sizeof(SolveOut), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(&flags_err[0], A->bar_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(&flags_err[1], A->flags_dev, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_status(e);
    const SolveOut &out = *A->out_host;
    int status;
    if (flags_err[0] == kDevTimeout)
        status = LDU_ERR_BARRIER_TIMEOUT;
    else if (flags_err[1] & (kFlagBadDiag | kFlagNonFinite))
        status = LDU_ERR_NOT_SPD;
    else
        status = map_status(out.status);
    A->last.status = status;
    A->last.iters = out.iters;
    A->last.replacements = out.replacements;
    A->last.relres = out.relres;
    A->last.bnorm = out.bnorm;
    A->last.grid_blocks = grid;
    A->last.block_threads = A->block_threads;
    if (status == LDU_OK || status == LDU_NOT_CONVERGED || status == LDU_ERR_NOT_SPD) {
        if (iters)
            *iters = out.iters;
        if (relres)
            *relres = out.relres;
    }
    return status;
}

}  // namespace

extern "C" {

int pcg_solve(const ldu_matrix *A, const double *b, double *x, double tol, int maxit, int *iters,
              double *relres, ldu_stream_t stream) {
    return run_solver(A, kPcg, b, x, tol, maxit, nullptr, iters, relres, (cudaStream_t)stream);
}

int pipecg_solve(const ldu_matrix *A, const double *b, double *x, double tol, int maxit,
                 int precision, const pcg_opts *opts, int *iters, double *relres,
                 ldu_stream_t stream) {
    if (precision == LDU_FP64)
        return run_solver(A, kPipe, b, x, tol, maxit, opts, iters, relres, (cudaStream_t)stream);
    if (precision == LDU_MIXED)
        return run_solver(A, kMixed, b, x, tol, maxit, opts, iters, relres, (cudaStream_t)stream);
    return LDU_ERR_BAD_ARG;
}

}  // extern "C"
