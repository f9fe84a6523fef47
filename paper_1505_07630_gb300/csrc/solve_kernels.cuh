// solve_kernels.cuh -- the persistent cooperative solver kernels (see
// solve.cu for the algorithms) and their parameter block.  Included by the
// .cu files that launch them; each gets its own copy (anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "ldupcg_impl.cuh"

namespace {

using namespace ldu;

struct SolveParams {
    SellView A;
    GridSync sync;
    double *slots;       // [2][gridDim.x][kNumDots]
    SolveOut *out;
    const double *b;     // caller, n entries
    double *x;           // caller, n entries: x0 in, solution out
    double *v64[10];
    float *v32[8];
    double tol;
    int maxit;
    int rr_period;
    double tau;
    int restart;
    int fault_inject;
};

__device__ __forceinline__ double *slot_of(const SolveParams &P, int parity) {
    return P.slots + ((size_t)parity * gridDim.x + blockIdx.x) * kNumDots;
}
__device__ __forceinline__ const double *slots_all(const SolveParams &P, int parity) {
    return P.slots + (size_t)parity * gridDim.x * kNumDots;
}

// Reduce K partials over the grid: block sums -> slot -> barrier -> totals.
// Returns false when the barrier failed (the kernel must return).
template <int K>
__device__ __forceinline__ bool reduce_grid(const SolveParams &P, double (&part)[K], double (&tot)[K],
                                            unsigned &epoch, int &parity) {
    block_sum_to_slot<K>(part, slot_of(P, parity));
    if (!grid_sync(P.sync, epoch))
        return false;
    grid_total<K>(slots_all(P, parity), tot);
    parity ^= 1;
    return true;
}

#define LANE_ROWS                                             \
    const int lane = threadIdx.x & 31;                        \
    const int warp = threadIdx.x >> 5;                        \
    const int nwarps = blockDim.x >> 5;                       \
    const SliceRange range = block_slices(P.A.n_slices);      \
    (void)range

#define FOR_MY_SLICES(s) for (int s = range.begin + warp; s < range.end; s += nwarps)

// pass 0 of every solver: bhat = b / sd, xhat = x0 * sd (rows < n), zero the
// listed vectors; partial ||b||^2 in part[0]
template <int R>
__device__ __forceinline__ void prep_pass(const SolveParams &P, double *bh, double *xh, double (&part)[1]) {
    LANE_ROWS;
    const SellView &A = P.A;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = row0 + j;
            const double bi = r < A.n ? P.b[r] : 0.0;
            const double xi = r < A.n ? P.x[r] : 0.0;
            bh[r] = bi * A.isd[r];
            xh[r] = xi * A.sd[r];
            part[0] = fma(bi, bi, part[0]);
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void zero_rows(const SolveParams &P, T *v) {
    LANE_ROWS;
    FOR_MY_SLICES(s) {
        T z[R];
#pragma unroll
        for (int j = 0; j < R; ++j)
            z[j] = T(0);
        st_rows<R>(v + s * P.A.C + R * lane, z);
    }
}

// x = xhat / sd for rows < n
template <int R>
__device__ __forceinline__ void unscale_pass(const SolveParams &P, const double *xh) {
    LANE_ROWS;
    const SellView &A = P.A;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = row0 + j;
            if (r < A.n)
                P.x[r] = xh[r] * A.isd[r];
        }
    }
}

__device__ __forceinline__ void zero_solution(const SolveParams &P) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.A.n; r += gridDim.x * blockDim.x)
        P.x[r] = 0.0;
}

__device__ __forceinline__ void write_out(const SolveParams &P, int status, int iters, int reps, double relres,
                          double bnorm) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.out->status = status;
        P.out->iters = iters;
        P.out->replacements = reps;
        P.out->relres = relres;
        P.out->bnorm = bnorm;
    }
}

// r = bhat - (I + Ahat_off) xhat (FP64); partials (r,r) and sum d r^2
template <int R, int KB>
__device__ __forceinline__ void residual64_pass(const SolveParams &P, const double *bh, const double *xh, double *r,
                                double (&part)[2]) {
    LANE_ROWS;
    const SellView &A = P.A;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double acc[R], bb[R], dd[R];
        ld_rows<R>(xh + row0, acc);
        sell_accum<double, R, KB>(A, s, lane, xh, acc);
        ld_rows<R>(bh + row0, bb);
        ld_rows<R>(A.dg + row0, dd);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            acc[j] = bb[j] - acc[j];
            part[0] = fma(acc[j], acc[j], part[0]);
            part[1] = fma(dd[j] * acc[j], acc[j], part[1]);
        }
        st_rows<R>(r + row0, acc);
    }
}

// ============================================================================
// Jacobi-PCG, FP64
// v64: 0 xhat, 1 bhat, 2 r, 3 p, 4 q
template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_pcg64(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;   // test hook: this block never arrives at a barrier
    LANE_ROWS;
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2], *p = P.v64[3], *q = P.v64[4];
    unsigned epoch = 0;
    int parity = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, bh, xh, b2);
    zero_rows<double, R>(P, p);   // the first p = r + 0 * p must not see stale values
    if (!reduce_grid<1>(P, b2, t1, epoch, parity))
        return;
    const double bnorm = sqrt(t1[0]);
    if (bnorm == 0.0) {
        zero_solution(P);
        write_out(P, kDevOk, 0, 0, 0.0, 0.0);
        return;
    }
    double part[2] = {0.0, 0.0}, tot[2];
    residual64_pass<R, KB>(P, bh, xh, r, part);
    if (!reduce_grid<2>(P, part, tot, epoch, parity))
        return;
    double gamma = tot[0];
    double relres = sqrt(tot[1]) / bnorm;
    int status = kDevNotConverged, it = 0, reps = 1;
    bool truth = true;   // relres is of a freshly computed true residual
    double beta = 0.0;
    if (relres <= P.tol) {
        status = kDevOk;
    } else {
        for (;;) {
            // p = r + beta p
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double rr[R], pp[R];
                ld_rows<R>(r + row0, rr);
                ld_rows<R>(p + row0, pp);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    pp[j] = fma(beta, pp[j], rr[j]);
                st_rows<R>(p + row0, pp);
            }
            if (!grid_sync(P.sync, epoch))
                return;
            if (it >= P.maxit) {
                status = kDevNotConverged;
                break;
            }
            // q = Ahat p ; (p, q)
            double pq[1] = {0.0}, tpq[1];
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double acc[R];
                ld_rows<R>(p + row0, acc);
                double pp[R];
#pragma unroll
                for (int j = 0; j < R; ++j)
                    pp[j] = acc[j];
                sell_accum<double, R, KB>(A, s, lane, p, acc);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    pq[0] = fma(pp[j], acc[j], pq[0]);
                st_rows<R>(q + row0, acc);
            }
            if (!reduce_grid<1>(P, pq, tpq, epoch, parity))
                return;
            if (!(tpq[0] > 0.0)) {
                status = kDevNotSpd;
                break;
            }
            const double alpha = gamma / tpq[0];
            // x += alpha p ; r -= alpha q ; (r, r), sum d r^2
            double pr[2] = {0.0, 0.0}, tr[2];
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double xx[R], pp[R], rr[R], qq[R], dd[R];
                ld_rows<R>(xh + row0, xx);
                ld_rows<R>(p + row0, pp);
                ld_rows<R>(r + row0, rr);
                ld_rows<R>(q + row0, qq);
                ld_rows<R>(A.dg + row0, dd);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    xx[j] = fma(alpha, pp[j], xx[j]);
                    rr[j] = fma(-alpha, qq[j], rr[j]);
                    pr[0] = fma(rr[j], rr[j], pr[0]);
                    pr[1] = fma(dd[j] * rr[j], rr[j], pr[1]);
                }
                st_rows<R>(xh + row0, xx);
                st_rows<R>(r + row0, rr);
            }
            if (!reduce_grid<2>(P, pr, tr, epoch, parity))
                return;
            ++it;
            relres = sqrt(tr[1]) / bnorm;
            truth = false;
            double gamma_new = tr[0];
            if (relres <= P.tol) {
                // confirm with the true residual; restart the search if it disagrees
                double pt[2] = {0.0, 0.0}, tt[2];
                residual64_pass<R, KB>(P, bh, xh, r, pt);
                if (!reduce_grid<2>(P, pt, tt, epoch, parity))
                    return;
                ++reps;
                relres = sqrt(tt[1]) / bnorm;
                truth = true;
                if (relres <= P.tol) {
                    status = kDevOk;
                    break;
                }
                gamma = tt[0];
                beta = 0.0;
                continue;
            }
            beta = gamma_new / gamma;
            gamma = gamma_new;
        }
    }
    if (!truth) {
        double pt[2] = {0.0, 0.0}, tt[2];
        residual64_pass<R, KB>(P, bh, xh, r, pt);
        if (!reduce_grid<2>(P, pt, tt, epoch, parity))
            return;
        ++reps;
        relres = sqrt(tt[1]) / bnorm;
    }
    unscale_pass<R>(P, xh);
    write_out(P, status, it, reps, relres, bnorm);
}

// ============================================================================
// pipelined PCG, FP64
// v64: 0 xhat, 1 bhat, 2 r, 3 w(a), 4 w(b), 5 z, 6 s, 7 p
template <int R, int KB>
__device__ __forceinline__ bool pipe64_replace(const SolveParams &P, const double *w_cur_c, double (&tot)[3],
                               unsigned &epoch, int &parity) {
    LANE_ROWS;
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2];
    double *w = const_cast<double *>(w_cur_c);
    double *z = P.v64[5], *sv = P.v64[6], *p = P.v64[7];
    // r = bhat - Ahat xhat
    double d2[2] = {0.0, 0.0}, t2[2];
    residual64_pass<R, KB>(P, bh, xh, r, d2);
    if (!grid_sync(P.sync, epoch))
        return false;
    // w = Ahat r ; s = Ahat p
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double aw[R], as[R];
        ld_rows<R>(r + row0, aw);
        ld_rows<R>(p + row0, as);
        sell_accum2<double, R, KB>(A, s, lane, r, p, aw, as);
        st_rows<R>(w + row0, aw);
        st_rows<R>(sv + row0, as);
    }
    if (!grid_sync(P.sync, epoch))
        return false;
    // z = Ahat s ; gamma = (r,r), delta = (w,r), rho = sum d r^2
    double part[3] = {0.0, 0.0, 0.0};
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double az[R], rr[R], ww[R], dd[R];
        ld_rows<R>(sv + row0, az);
        sell_accum<double, R, KB>(A, s, lane, sv, az);
        st_rows<R>(z + row0, az);
        ld_rows<R>(r + row0, rr);
        ld_rows<R>(w + row0, ww);
        ld_rows<R>(A.dg + row0, dd);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            part[0] = fma(rr[j], rr[j], part[0]);
            part[1] = fma(ww[j], rr[j], part[1]);
            part[2] = fma(dd[j] * rr[j], rr[j], part[2]);
        }
    }
    (void)d2;
    (void)t2;
    return reduce_grid<3>(P, part, tot, epoch, parity);
}

template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_pipe64(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;
    LANE_ROWS;
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2];
    double *wbuf[2] = {P.v64[3], P.v64[4]};
    double *z = P.v64[5], *sv = P.v64[6], *p = P.v64[7];
    unsigned epoch = 0;
    int parity = 0, wc = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, bh, xh, b2);
    zero_rows<double, R>(P, p);
    zero_rows<double, R>(P, z);
    zero_rows<double, R>(P, sv);
    if (!reduce_grid<1>(P, b2, t1, epoch, parity))
        return;
    const double bnorm = sqrt(t1[0]);
    if (bnorm == 0.0) {
        zero_solution(P);
        write_out(P, kDevOk, 0, 0, 0.0, 0.0);
        return;
    }
    double tot[3];
    if (!pipe64_replace<R, KB>(P, wbuf[wc], tot, epoch, parity))
        return;
    int reps = 1, it = 0, since = 0, status = kDevNotConverged;
    bool truth = true, fresh = true;
    double gamma = tot[0], delta = tot[1], relres = sqrt(tot[2]) / bnorm;
    double gamma_old = 0.0, alpha_old = 0.0;
    for (;;) {
        const bool want = relres <= P.tol || (P.rr_period > 0 && since >= P.rr_period);
        if (want && !truth) {
            if (!pipe64_replace<R, KB>(P, wbuf[wc], tot, epoch, parity))
                return;
            ++reps;
            since = 0;
            truth = true;
            gamma = tot[0];
            delta = tot[1];
            relres = sqrt(tot[2]) / bnorm;
        }
        if (truth && relres <= P.tol) {
            status = kDevOk;
            break;
        }
        if (it >= P.maxit) {
            status = kDevNotConverged;
            break;
        }
        double beta, denom;
        if (fresh) {
            beta = 0.0;
            denom = delta;
        } else {
            beta = gamma / gamma_old;
            denom = delta - beta * gamma / alpha_old;
        }
        if (!(denom > 0.0) || !(gamma > 0.0)) {
            if (fresh) {
                status = kDevNotSpd;
                break;
            }
            // rounding drift: replace from the true residual and restart
            if (!pipe64_replace<R, KB>(P, wbuf[wc], tot, epoch, parity))
                return;
            ++reps;
            since = 0;
            truth = true;
            fresh = true;
            gamma = tot[0];
            delta = tot[1];
            relres = sqrt(tot[2]) / bnorm;
            continue;
        }
        fresh = false;
        const double alpha = gamma / denom;
        const double *w = wbuf[wc];
        double *wn = wbuf[wc ^ 1];
        double part[3] = {0.0, 0.0, 0.0};
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double nn[R], ww[R];
            ld_rows<R>(w + row0, ww);
#pragma unroll
            for (int j = 0; j < R; ++j)
                nn[j] = ww[j];
            sell_accum<double, R, KB>(A, s, lane, w, nn);
            double zz[R], ss[R], pp[R], xx[R], rr[R], dd[R];
            ld_rows<R>(z + row0, zz);
            ld_rows<R>(sv + row0, ss);
            ld_rows<R>(p + row0, pp);
            ld_rows<R>(xh + row0, xx);
            ld_rows<R>(r + row0, rr);
            ld_rows<R>(A.dg + row0, dd);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                zz[j] = fma(beta, zz[j], nn[j]);
                ss[j] = fma(beta, ss[j], ww[j]);
                pp[j] = fma(beta, pp[j], rr[j]);
                xx[j] = fma(alpha, pp[j], xx[j]);
                rr[j] = fma(-alpha, ss[j], rr[j]);
                ww[j] = fma(-alpha, zz[j], ww[j]);
                part[0] = fma(rr[j], rr[j], part[0]);
                part[1] = fma(ww[j], rr[j], part[1]);
                part[2] = fma(dd[j] * rr[j], rr[j], part[2]);
            }
            st_rows<R>(z + row0, zz);
            st_rows<R>(sv + row0, ss);
            st_rows<R>(p + row0, pp);
            st_rows<R>(xh + row0, xx);
            st_rows<R>(r + row0, rr);
            st_rows<R>(wn + row0, ww);
        }
        if (!reduce_grid<3>(P, part, tot, epoch, parity))
            return;
        wc ^= 1;
        gamma_old = gamma;
        alpha_old = alpha;
        gamma = tot[0];
        delta = tot[1];
        relres = sqrt(tot[2]) / bnorm;
        truth = false;
        ++it;
        ++since;
    }
    if (!truth) {
        double pt[2] = {0.0, 0.0}, tt[2];
        residual64_pass<R, KB>(P, bh, xh, r, pt);
        if (!reduce_grid<2>(P, pt, tt, epoch, parity))
            return;
        ++reps;
        relres = sqrt(tt[1]) / bnorm;
    }
    unscale_pass<R>(P, xh);
    write_out(P, status, it, reps, relres, bnorm);
}

// ============================================================================
// mixed precision: float pipelined recurrences, FP64 solution and residual
// v64: 0 xhat, 1 bhat
// v32: 0 xc, 1 r, 2 w(a), 3 w(b), 4 z, 5 s, 6 p
template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_mixed(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;
    LANE_ROWS;
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1];
    float *xc = P.v32[0], *r = P.v32[1];
    float *wbuf[2] = {P.v32[2], P.v32[3]};
    float *z = P.v32[4], *sv = P.v32[5], *p = P.v32[6];
    unsigned epoch = 0;
    int parity = 0, wc = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, bh, xh, b2);
    zero_rows<float, R>(P, xc);
    zero_rows<float, R>(P, p);
    zero_rows<float, R>(P, z);
    zero_rows<float, R>(P, sv);
    if (!reduce_grid<1>(P, b2, t1, epoch, parity))
        return;
    const double bnorm = sqrt(t1[0]);
    if (bnorm == 0.0) {
        zero_solution(P);
        write_out(P, kDevOk, 0, 0, 0.0, 0.0);
        return;
    }
    double sigma = 1.0, ratio = 1.0, gamma = 0.0, delta = 0.0, gamma_old = 0.0, alpha_old = 0.0;
    double gamma_ref = 0.0, relres = 1.0;
    int it = 0, since = 0, reps = 0, status = kDevNotConverged;
    bool fresh = true, force = true;
    for (;;) {
        const double predicted = sqrt(ratio * gamma) * sigma / bnorm;
        const bool trigger = force || (P.rr_period > 0 && since >= P.rr_period) ||
                             (P.tau > 0.0 && gamma <= P.tau * P.tau * gamma_ref) ||
                             predicted <= P.tol || it >= P.maxit;
        if (trigger) {
            // U1: fold the float correction into the FP64 solution
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double xx[R];
                float cc[R], zr[R];
                ld_rows<R>(xh + row0, xx);
                ld_rows<R>(xc + row0, cc);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    xx[j] = fma(sigma, (double)cc[j], xx[j]);
                    zr[j] = 0.0f;
                }
                st_rows<R>(xh + row0, xx);
                st_rows<R>(xc + row0, zr);
            }
            if (!grid_sync(P.sync, epoch))
                return;
            // U2: FP64 true residual, stored in float in units of the old sigma
            const double inv_sigma = 1.0 / sigma;   // power of two: exact
            double part[2] = {0.0, 0.0}, tot[2];
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double acc[R], bb[R], dd[R];
                ld_rows<R>(xh + row0, acc);
                sell_accum<double, R, KB>(A, s, lane, xh, acc);
                ld_rows<R>(bh + row0, bb);
                ld_rows<R>(A.dg + row0, dd);
                float rf[R];
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const double rj = bb[j] - acc[j];
                    part[0] = fma(rj, rj, part[0]);
                    part[1] = fma(dd[j] * rj, rj, part[1]);
                    rf[j] = (float)(rj * inv_sigma);
                }
                st_rows<R>(r + row0, rf);
            }
            if (!reduce_grid<2>(P, part, tot, epoch, parity))
                return;
            ++reps;
            relres = sqrt(tot[1]) / bnorm;
            if (relres <= P.tol) {
                status = kDevOk;
                break;
            }
            if (it >= P.maxit) {
                status = kDevNotConverged;
                break;
            }
            if (!(tot[0] > 0.0)) {
                status = kDevNotSpd;
                break;
            }
            ratio = tot[1] / tot[0];
            const double sigma_new = exp2(rint(log2(sqrt(tot[0]))));
            const float f = (float)(sigma / sigma_new);
            const float pf = P.restart ? 0.0f : f;
            if (P.restart)
                fresh = true;
            else
                gamma_old *= (double)f * (double)f;
            sigma = sigma_new;
            // U3: w = f (Ahat r) ; s = pf (Ahat p)
            float *w = wbuf[wc];
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                float aw[R], as[R];
                ld_rows<R>(r + row0, aw);
                ld_rows<R>(p + row0, as);
                sell_accum2<float, R, KB>(A, s, lane, r, p, aw, as);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    aw[j] *= f;
                    as[j] *= pf;
                }
                st_rows<R>(w + row0, aw);
                st_rows<R>(sv + row0, as);
            }
            if (!grid_sync(P.sync, epoch))
                return;
            // U4: z = Ahat s ; r *= f ; p *= pf ; gamma = (r,r), delta = (w,r)
            double pd[2] = {0.0, 0.0}, td[2];
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                float az[R], rr[R], pp[R], ww[R];
                ld_rows<R>(sv + row0, az);
                sell_accum<float, R, KB>(A, s, lane, sv, az);
                st_rows<R>(z + row0, az);
                ld_rows<R>(r + row0, rr);
                ld_rows<R>(p + row0, pp);
                ld_rows<R>(w + row0, ww);
                float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    rr[j] *= f;
                    pp[j] *= pf;
                    g0 = fmaf(rr[j], rr[j], g0);
                    g1 = fmaf(ww[j], rr[j], g1);
                }
                pd[0] += (double)g0;
                pd[1] += (double)g1;
                st_rows<R>(r + row0, rr);
                st_rows<R>(p + row0, pp);
            }
            if (!reduce_grid<2>(P, pd, td, epoch, parity))
                return;
            gamma = td[0];
            delta = td[1];
            gamma_ref = gamma;
            since = 0;
            force = false;
        }
        double beta, denom;
        if (fresh) {
            beta = 0.0;
            denom = delta;
        } else {
            beta = gamma / gamma_old;
            denom = delta - beta * gamma / alpha_old;
        }
        if (!(denom > 0.0) || !(gamma > 0.0)) {
            if (fresh) {
                status = kDevNotSpd;
                break;
            }
            fresh = true;
            force = true;
            continue;
        }
        fresh = false;
        const double alpha = gamma / denom;
        const float a = (float)alpha, bt = (float)beta;
        const float *w = wbuf[wc];
        float *wn = wbuf[wc ^ 1];
        double part[2] = {0.0, 0.0}, tot[2];
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            float nn[R], ww[R];
            ld_rows<R>(w + row0, ww);
#pragma unroll
            for (int j = 0; j < R; ++j)
                nn[j] = ww[j];
            sell_accum<float, R, KB>(A, s, lane, w, nn);
            float zz[R], ss[R], pp[R], xx[R], rr[R];
            ld_rows<R>(z + row0, zz);
            ld_rows<R>(sv + row0, ss);
            ld_rows<R>(p + row0, pp);
            ld_rows<R>(xc + row0, xx);
            ld_rows<R>(r + row0, rr);
            float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                zz[j] = fmaf(bt, zz[j], nn[j]);
                ss[j] = fmaf(bt, ss[j], ww[j]);
                pp[j] = fmaf(bt, pp[j], rr[j]);
                xx[j] = fmaf(a, pp[j], xx[j]);
                rr[j] = fmaf(-a, ss[j], rr[j]);
                ww[j] = fmaf(-a, zz[j], ww[j]);
                g0 = fmaf(rr[j], rr[j], g0);
                g1 = fmaf(ww[j], rr[j], g1);
            }
            part[0] += (double)g0;
            part[1] += (double)g1;
            st_rows<R>(z + row0, zz);
            st_rows<R>(sv + row0, ss);
            st_rows<R>(p + row0, pp);
            st_rows<R>(xc + row0, xx);
            st_rows<R>(r + row0, rr);
            st_rows<R>(wn + row0, ww);
        }
        if (!reduce_grid<2>(P, part, tot, epoch, parity))
            return;
        wc ^= 1;
        gamma_old = gamma;
        alpha_old = alpha;
        gamma = tot[0];
        delta = tot[1];
        ++it;
        ++since;
    }
    unscale_pass<R>(P, xh);
    write_out(P, status, it, reps, relres, bnorm);
}

}  // namespace
