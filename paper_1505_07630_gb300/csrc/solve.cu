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
//           the periodic true residual (3 passes per replacement: fold the
//           float correction into x; true residual together with s = Ahat p;
//           w = Ahat r and z = Ahat s).  The float sweeps stage their matrix
//           slices in shared memory with bulk copies when it fits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ldupcg_impl.cuh"

using namespace ldu;

#include "solve_kernels.cuh"

namespace {

// b = mass * T, the right-hand side of a backward-Euler step
__global__ void k_mass_rhs(int64_t n, const double *__restrict__ mass,
                           const double *__restrict__ T, double *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = mass[i] * T[i];
}

// b = -div(phi) for the pressure stage of a PISO step: row r (a cell) adds
// +phi_f over the faces where it is the neighbour (the slot holds the lower
// coefficient) and -phi_f over the faces it owns, in its slot order (the
// order of its neighbours), so that repeated calls agree bitwise
__global__ void k_neg_div(int n, int C, const int *__restrict__ slice_ptr,
                          const int *__restrict__ slice_w, const uint32_t *__restrict__ fid,
                          const double *__restrict__ phi, double *__restrict__ b) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int s = r / C, i = r - s * C;
        const int base = slice_ptr[s] + i, w = slice_w[s];
        double acc = 0.0;
        for (int q = 0; q < w; ++q) {
            const uint32_t f = fid[base + q * C];
            if (f == kPadFid)
                continue;
            const double v = phi[f & ~kLowerBit];
            acc += (f & kLowerBit) ? v : -v;
        }
        b[r] = acc;
    }
}

// phi_f -= c_f (p_N - p_P), P the owner and N the neighbour of face f
__global__ void k_flux_correct(int64_t nf, const int32_t *__restrict__ own,
                               const int32_t *__restrict__ nbr, const double *__restrict__ coef,
                               const double *__restrict__ p, double *__restrict__ phi) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x)
        phi[f] = fma(-coef[f], p[nbr[f]] - p[own[f]], phi[f]);
}

// ---------------------------------------------------------------------------
// host side

enum Kind { kPcg = 0, kPipe = 1, kMixed = 2, kMixedDeflated = 3 };

// Resident blocks per SM the mixed kernel is compiled for: 2 by default;
// 3 or 4 (fewer registers, more warps) where that compiles without spills.
int mixed_minb(int R, int blocks_per_sm) {
    if (blocks_per_sm >= 4 && R == 1)
        return 4;
    if (blocks_per_sm >= 3 && R <= 2)
        return 3;
    return 2;
}

template <int R>
const void *kernel_ptr(Kind k, int minb, bool stg) {
    switch (k) {
    case kPcg: return (const void *)k_pcg64<R, Batch<R>::pcg>;
    case kPipe: return (const void *)k_pipe64<R, Batch<R>::pipe>;
    case kMixedDeflated:
        if (stg)
            return (const void *)k_mixed<R, Batch<R>::mixed, true, 2, true>;
        return (const void *)k_mixed<R, Batch<R>::mixed, true, 2, false>;
    default:
        if (stg) {
            if constexpr (R <= 2) {
                if (minb == 3)
                    return (const void *)k_mixed<R, MixedBatch<R, 3>::kb, false, 3, true>;
            }
            if constexpr (R == 1) {
                if (minb == 4)
                    return (const void *)k_mixed<R, MixedBatch<R, 4>::kb, false, 4, true>;
            }
            return (const void *)k_mixed<R, Batch<R>::mixed, false, 2, true>;
        }
        if constexpr (R <= 2) {
            if (minb == 3)
                return (const void *)k_mixed<R, MixedBatch<R, 3>::kb, false, 3, false>;
        }
        if constexpr (R == 1) {
            if (minb == 4)
                return (const void *)k_mixed<R, MixedBatch<R, 4>::kb, false, 4, false>;
        }
        return (const void *)k_mixed<R, Batch<R>::mixed, false, 2, false>;
    }
}

const void *pick_kernel(const ldu_matrix *A, Kind k, bool stg) {
    const int R = A->C / 32;
    const int minb = mixed_minb(R, A->blocks_per_sm);
    switch (A->C) {
    case 32: return kernel_ptr<1>(k, minb, stg);
    case 64: return kernel_ptr<2>(k, minb, stg);
    default: return kernel_ptr<4>(k, minb, stg);
    }
}

// Default replacement rule of the mixed solve: every 16 float iterations,
// and sooner once (r, r) has dropped by 0.3^2.  Measured on the 64^3, 96^3
// and 128^3 lognormal cases it keeps the FP64 method's iteration counts
// (417, 616, 752) with 29, 41 and 50 replacements; every 12 needs 36, 53
// and 64, and every 16 without the drop test loses 12 % of the iterations
// at 128^3 to a plateau near convergence.
constexpr int kMixedPeriod = 16;
constexpr double kMixedTau = 0.3;

// Largest dynamic shared memory a block of the staged mixed kernel may take
// and still leave room for minb resident blocks per SM (228 KB per SM, less
// 1 KB reserved and the kernel's static shared memory per block).
size_t staged_smem_max(int minb) {
    return (size_t)228 * 1024 / (size_t)minb - 5 * 1024;
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
    if (kind == kMixed && opt.rr_period == 0 && opt.tau == 0.0) {
        opt.rr_period = kMixedPeriod;
        opt.tau = kMixedTau;
    }
    A->last = ldu_solve_stats{};
    if (A->n == 0) {
        if (iters)
            *iters = 0;
        if (relres)
            *relres = 0.0;
        A->last.status = LDU_OK;
        return LDU_OK;
    }
    const Kind kk = (kind == kMixed && opt.deflate) ? kMixedDeflated : kind;
    size_t meta = 0;
    // the grid has at least min(SMs, cap) blocks: size the metadata for that
    meta_smem_bytes(A->n_slices, std::min(A->num_sms, grid_cap(A)), &meta);
    const int meta_cap = (int)(meta / sizeof(int2));
    size_t smem = meta;
    const int minb = mixed_minb(A->C / 32, A->blocks_per_sm);
    bool stg = (kk == kMixed || (kk == kMixedDeflated && minb == 2)) && A->staging == 0 &&
               A->max_w > 0;
    int nst = 0;
    if (stg) {
        // deepest pipeline that leaves room for minb blocks per SM
        const int cb = A->col16 ? 2 : 4;
        for (int d = kMaxStages; d >= 2 && nst == 0; --d) {
            const size_t b = staged_smem_bytes(meta_cap, A->block_threads / 32, A->max_w, A->C, cb, d);
            if (b <= staged_smem_max(minb)) {
                smem = b;
                nst = d;
            }
        }
        stg = nst > 0;
    }
    const void *kern = pick_kernel(A, kk, stg);
    int grid = 0;
    int rc = grid_for_smem(A, kern, A->block_threads, smem, &grid);
    if (rc != LDU_OK)
        return rc;
    SolveParams P;
    P.A = view_of(A);
    P.A.meta_smem = meta > 0;
    P.A.meta_cap = meta_cap;
    P.A.stage_w = stg ? A->max_w : 0;
    P.A.stages = nst;
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
    else if (flags_err[0] != 0)
        status = LDU_ERR_CUDA;
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
    A->last.staged = stg ? 1 : 0;
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

int ldu_heat_steps(ldu_matrix *A, const double *mass, double *T, int nsteps, double tol,
                   int maxit, int precision, const pcg_opts *opts, int *iters_total,
                   double *relres_last, ldu_stream_t stream) {
    if (!A || nsteps < 0 || (A->n > 0 && (!mass || !T)) ||
        (precision != LDU_FP64 && precision != LDU_MIXED))
        return LDU_ERR_BAD_ARG;
    if (A->row_cell)
        return LDU_ERR_UNSUPPORTED;   // single-system handles only
    cudaStream_t st = (cudaStream_t)stream;
    if (iters_total)
        *iters_total = 0;
    if (relres_last)
        *relres_last = 0.0;
    if (A->n == 0 || nsteps == 0)
        return LDU_OK;
    if (!A->rhs) {
        cudaError_t e = cudaMalloc((void **)&A->rhs, sizeof(double) * (size_t)A->n);
        if (e != cudaSuccess)
            return cuda_status(e);
        A->device_bytes += (int64_t)sizeof(double) * A->n;
    }
    int total = 0, rc = LDU_OK;
    double rr = 0.0;
    for (int step = 0; step < nsteps; ++step) {
        // b = mass T^n; T^n is also the initial guess of T^(n+1)
        k_mass_rhs<<<(int)std::min<int64_t>((A->n + 255) / 256, 1 << 20), 256, 0, st>>>(
            A->n, mass, T, A->rhs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_status(e);
        int it = 0;
        rc = precision == LDU_FP64
                 ? run_solver(A, kPcg, A->rhs, T, tol, maxit, opts, &it, &rr, st)
                 : run_solver(A, kMixed, A->rhs, T, tol, maxit, opts, &it, &rr, st);
        total += it;
        if (rc != LDU_OK)
            break;
    }
    if (iters_total)
        *iters_total = total;
    if (relres_last)
        *relres_last = rr;
    return rc;
}

int ldu_piso_pressure(ldu_matrix *A, const double *coef, double *phi, double *p, double tol,
                      int maxit, int precision, const pcg_opts *opts, int *iters,
                      double *relres, ldu_stream_t stream) {
    if (!A || (A->n > 0 && !p) || (A->nf > 0 && (!coef || !phi)) ||
        (precision != LDU_FP64 && precision != LDU_MIXED))
        return LDU_ERR_BAD_ARG;
    if (A->row_cell)
        return LDU_ERR_UNSUPPORTED;   // single-system handles only
    cudaStream_t st = (cudaStream_t)stream;
    if (iters)
        *iters = 0;
    if (relres)
        *relres = 0.0;
    if (A->n == 0)
        return LDU_OK;
    if (!A->rhs) {
        cudaError_t e = cudaMalloc((void **)&A->rhs, sizeof(double) * (size_t)A->n);
        if (e != cudaSuccess)
            return cuda_status(e);
        A->device_bytes += (int64_t)sizeof(double) * A->n;
    }
    const int grid_n = (int)std::min<int64_t>((A->n + 255) / 256, 1 << 20);
    k_neg_div<<<grid_n, 256, 0, st>>>((int)A->n, A->C, A->slice_ptr, A->slice_w, A->fid, phi,
                                      A->rhs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_status(e);
    const int rc = run_solver(A, precision == LDU_FP64 ? kPcg : kMixed, A->rhs, p, tol, maxit,
                              opts, iters, relres, st);
    if (rc != LDU_OK && rc != LDU_NOT_CONVERGED)
        return rc;
    if (A->nf > 0) {
        k_flux_correct<<<(int)std::min<int64_t>((A->nf + 255) / 256, 1 << 20), 256, 0, st>>>(
            A->nf, A->owner, A->neighbour, coef, p, phi);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    return rc;
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
