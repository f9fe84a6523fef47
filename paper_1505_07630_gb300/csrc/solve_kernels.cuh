// solve_kernels.cuh -- the persistent cooperative solver kernels (see
// solve.cu for the algorithms) and their parameter block.  Included by the
// .cu files that launch them; each gets its own copy (anonymous namespace).
//
// Control: the scalar recurrences (alpha, beta, stopping tests, replacement
// triggers) run in thread 0 of every block, in FP64, on totals that are
// bitwise identical in every block; thread 0 publishes its decisions in a
// shared-memory block and the other threads read them after __syncthreads.
// Per-iteration dot products are reduced as float pairs (FF); the rare
// FP64 reductions (start-up, residual replacement) stay in double.  Tests
// compare squared norms with precomputed squared thresholds, so an
// iteration needs no square root.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "ldupcg_impl.cuh"

namespace {

using namespace ldu;

struct SolveParams {
    SellView A;
    GridSync sync;
    double *slots;       // reduction slots of the scopes; FF sums use the cells as float2
    const int *tasks;    // batched launches: per-block task lists (see solve_batched.cu)
    SolveOut *out;
    const double *b;     // caller, n entries
    double *x;           // caller, n entries: x0 in, solution out
    double *v64[10];
    float *v32[10];
    double tol;
    int maxit;
    int rr_period;
    double tau;
    int restart;
    int deflate;
    int fault_inject;
};

// The blocks that solve one system together and what they share: the whole
// grid for a single solve, a team of blocks (or one block) for one system of
// a batch.  Barriers and reductions are scoped to these members.
struct Scope {
    int members;          // blocks in the scope
    int rank;             // this block's rank in it
    unsigned *count;      // barrier counter of the scope (unused when members == 1)
    double *slots;        // [2][members][kNumDots] reduction slots
    SliceRange range;     // slices this block sweeps
    int row0;             // first row of the system in the padded layout
    int n;                // real rows of the system
    long long b_off;      // offset of the system in the caller's b and x
    int id;               // index of the system's SolveOut
};

__device__ __forceinline__ double *slot_of(const Scope &sc, int parity) {
    return sc.slots + ((size_t)parity * sc.members + sc.rank) * kNumDots;
}
__device__ __forceinline__ const double *slots_all(const Scope &sc, int parity) {
    return sc.slots + (size_t)parity * sc.members * kNumDots;
}

// Barrier over the scope's blocks; a one-block scope needs only __syncthreads.
__device__ __forceinline__ bool scope_sync(const Scope &sc, const GridSync &g, unsigned &epoch,
                                           bool lead = true) {
    if (sc.members == 1) {
        __syncthreads();
        return true;
    }
    GridSync t = g;
    t.count = sc.count;
    return team_sync(t, epoch, (unsigned)sc.members, lead);
}

// The whole grid as one scope (single-system launch).
__device__ __forceinline__ Scope grid_scope(const SolveParams &P) {
    Scope sc;
    sc.members = gridDim.x;
    sc.rank = blockIdx.x;
    sc.count = P.sync.count;
    sc.slots = P.slots;
    sc.range = block_slices(P.A.n_slices);
    sc.row0 = 0;
    sc.n = P.A.n;
    sc.b_off = 0;
    sc.id = 0;
    return sc;
}

// Slots taken per batch by sell_accum for each solver and rows per lane R:
// the largest batch that compiles without register spills at 128
// registers per thread (two 256-thread blocks per SM).
template <int R>
struct Batch {
    static constexpr int pcg = R == 4 ? 2 : 3;
    static constexpr int pipe = R == 1 ? 3 : 1;
    static constexpr int mixed = R == 4 ? 2 : (R == 2 ? 3 : 6);
};

// The mixed sweep is bound by chains of dependent loads, so more resident
// warps help; these (rows per lane, blocks per SM) pairs compile without
// spills at the register share that occupancy leaves (80 registers at 3
// blocks, 64 at 4), with the batch given here.
template <int R, int MINB>
struct MixedBatch {
    static constexpr int kb = MINB == 2 ? Batch<R>::mixed : (R == 1 && MINB == 3 ? 3 : 2);
};

// FP64 reduction of K partials: block sums -> slot -> barrier -> totals.
// Returns false when the barrier failed (the kernel must return).
// tail(totals) runs in thread 0 before the totals reach the block (see
// grid_total).  The block sum ends with a __syncthreads after every thread's
// writes, so the barrier needs no leading one.
template <int K, typename Tail = NoTail>
__device__ __forceinline__ bool reduce_d(const SolveParams &P, const Scope &sc, double (&part)[K],
                                         double (&tot)[K], unsigned &epoch, int &parity,
                                         Tail tail = Tail()) {
    block_sum_to_slot<K>(part, slot_of(sc, parity));
    if (!scope_sync(sc, P.sync, epoch, false))
        return false;
    grid_total<K>(slots_all(sc, parity), tot, sc.members, tail);
    parity ^= 1;
    return true;
}

// The same with float-pair arithmetic (per-iteration dot products).
template <int K, typename Tail = NoTail>
__device__ __forceinline__ bool reduce_f(const SolveParams &P, const Scope &sc, FF (&part)[K],
                                         double (&tot)[K], unsigned &epoch, int &parity,
                                         Tail tail = Tail()) {
    block_sum_ff<K>(part, reinterpret_cast<float2 *>(slot_of(sc, parity)));
    if (!scope_sync(sc, P.sync, epoch, false))
        return false;
    grid_total_ff<K>(reinterpret_cast<const float2 *>(slots_all(sc, parity)), tot, sc.members,
                     tail);
    parity ^= 1;
    return true;
}

// A power of two close to 1/x (1 for x == 0): scales FP64 partials into the
// float range before a float-pair reduction, exactly.
__device__ __forceinline__ double inv_pow2(double x) {
    if (!(x > 0.0) || !isfinite(x))
        return 1.0;
    return ldexp(1.0, -ilogb(x));
}

#define LANE_ROWS                                             \
    const int lane = threadIdx.x & 31;                        \
    const int warp = threadIdx.x >> 5;                        \
    const int nwarps = blockDim.x >> 5;                       \
    const SliceRange range = sc.range;                        \
    (void)range

#define FOR_MY_SLICES(s) for (int s = range.begin + warp; s < range.end; s += nwarps)

// pass 0 of every solver: bhat = b / sd, xhat = x0 * sd (rows < n); partial
// ||b||^2 in part[0]
template <int R>
__device__ __forceinline__ void prep_pass(const SolveParams &P, const Scope &sc, double *bh,
                                          double *xh, double (&part)[1]) {
    LANE_ROWS;
    const SellView &A = P.A;
    const double *b = P.b + sc.b_off;
    const double *x = P.x + sc.b_off;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = row0 + j;
            const int i = r - sc.row0;
            const double bi = i < sc.n ? b[i] : 0.0;
            const double xi = i < sc.n ? x[i] : 0.0;
            bh[r] = bi * A.isd[r];
            xh[r] = xi * A.sd[r];
            part[0] = fma(bi, bi, part[0]);
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void zero_rows(const SolveParams &P, const Scope &sc, T *v) {
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
__device__ __forceinline__ void unscale_pass(const SolveParams &P, const Scope &sc,
                                             const double *xh) {
    LANE_ROWS;
    const SellView &A = P.A;
    double *x = P.x + sc.b_off;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = row0 + j;
            const int i = r - sc.row0;
            if (i < sc.n)
                x[i] = xh[r] * A.isd[r];
        }
    }
}

__device__ __forceinline__ void zero_solution(const SolveParams &P, const Scope &sc) {
    double *x = P.x + sc.b_off;
    for (int i = sc.rank * blockDim.x + threadIdx.x; i < sc.n; i += sc.members * blockDim.x)
        x[i] = 0.0;
}

__device__ __forceinline__ void write_out(const SolveParams &P, const Scope &sc, int status,
                                          int iters, int reps, double relres, double bnorm) {
    if (sc.rank == 0 && threadIdx.x == 0) {
        SolveOut *o = P.out + sc.id;
        o->status = status;
        o->iters = iters;
        o->replacements = reps;
        o->relres = relres;
        o->bnorm = bnorm;
    }
}

// r = bhat - (I + Ahat_off) xhat (FP64); partials (r,r) and sum d r^2
template <int R, int KB>
__device__ __forceinline__ void residual64_pass(const SolveParams &P, const Scope &sc,
                                                const double *bh, const double *xh, double *r,
                                                double (&part)[2]) {
    LANE_ROWS;
    const SellView &A = P.A;
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double acc[R], bb[R], dd[R];
        ld_rows<R>(xh + row0, acc);
        sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, xh, acc);
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
struct PcgCtl {
    double alpha, beta;
    int exit, check, truth;
};

template <int R, int KB>
__device__ __forceinline__ bool pcg64_body(const SolveParams &P, const Scope &sc) {
    __syncthreads();   // the previous body of this block is done with shared state
    LANE_ROWS;
    load_slice_meta(P.A, sc.range);
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2], *p = P.v64[3], *q = P.v64[4];
    __shared__ PcgCtl ctl;
    const bool t0 = threadIdx.x == 0;
    unsigned epoch = 0;
    int parity = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, sc, bh, xh, b2);
    zero_rows<double, R>(P, sc, p);   // the first p = r + 0 * p must not see stale values
    if (!reduce_d<1>(P, sc, b2, t1, epoch, parity))
        return false;
    const double bn2 = t1[0];
    if (bn2 == 0.0) {
        zero_solution(P, sc);
        write_out(P, sc, kDevOk, 0, 0, 0.0, 0.0);
        return true;
    }
    const double thr2 = P.tol * P.tol * bn2;   // stop when sum d r^2 <= tol^2 ||b||^2
    double part[2] = {0.0, 0.0}, tot[2];
    residual64_pass<R, KB>(P, sc, bh, xh, r, part);
    if (!reduce_d<2>(P, sc, part, tot, epoch, parity))
        return false;
    // thread-0 state
    double gamma = tot[0], rho = tot[1];
    int status = kDevNotConverged, it = 0, reps = 1;
    // float-pair sums carry (r,r)-sized values scaled by sg, d-weighted ones by sr
    const double sg = inv_pow2(gamma), sr = inv_pow2(rho);
    if (t0) {
        ctl.exit = rho <= thr2;
        ctl.beta = 0.0;
        ctl.truth = 1;
        if (ctl.exit)
            status = kDevOk;
    }
    __syncthreads();
    while (!ctl.exit) {
        // p = r + beta p
        const double beta = ctl.beta;
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
        if (!scope_sync(sc, P.sync, epoch))
            return false;
        if (t0 && it >= P.maxit) {
            ctl.exit = 1;
            status = kDevNotConverged;
        }
        __syncthreads();
        if (ctl.exit)
            break;
        // q = Ahat p ; (p, q)
        double pq = 0.0;
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double acc[R], pp[R];
            ld_rows<R>(p + row0, acc);
#pragma unroll
            for (int j = 0; j < R; ++j)
                pp[j] = acc[j];
            sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, p, acc);
#pragma unroll
            for (int j = 0; j < R; ++j)
                pq = fma(pp[j], acc[j], pq);
            st_rows<R>(q + row0, acc);
        }
        FF fpq[1] = {ff_from_double(pq * sg)};
        double tpq[1];
        if (!reduce_f<1>(P, sc, fpq, tpq, epoch, parity))
            return false;
        if (t0) {
            const double pqv = tpq[0] / sg;
            if (!(pqv > 0.0)) {
                status = kDevNotSpd;
                ctl.exit = 1;
            } else {
                ctl.alpha = gamma / pqv;
            }
        }
        __syncthreads();
        if (ctl.exit)
            break;
        const double alpha = ctl.alpha;
        // x += alpha p ; r -= alpha q ; (r, r), sum d r^2
        double g0 = 0.0, g1 = 0.0;
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
                g0 = fma(rr[j], rr[j], g0);
                g1 = fma(dd[j] * rr[j], rr[j], g1);
            }
            st_rows<R>(xh + row0, xx);
            st_rows<R>(r + row0, rr);
        }
        FF fr[2] = {ff_from_double(g0 * sg), ff_from_double(g1 * sr)};
        double tr[2];
        if (!reduce_f<2>(P, sc, fr, tr, epoch, parity))
            return false;
        if (t0) {
            ++it;
            ctl.truth = 0;
            const double gamma_new = tr[0] / sg;
            rho = tr[1] / sr;
            if (rho <= thr2) {
                ctl.check = 1;
            } else {
                ctl.check = 0;
                ctl.beta = gamma_new / gamma;
                gamma = gamma_new;
            }
        }
        __syncthreads();
        if (ctl.check) {
            // confirm with the true residual; restart the search if it disagrees
            double pt[2] = {0.0, 0.0}, tt[2];
            residual64_pass<R, KB>(P, sc, bh, xh, r, pt);
            if (!reduce_d<2>(P, sc, pt, tt, epoch, parity))
                return false;
            if (t0) {
                ++reps;
                ctl.truth = 1;
                rho = tt[1];
                if (rho <= thr2) {
                    status = kDevOk;
                    ctl.exit = 1;
                } else {
                    gamma = tt[0];
                    ctl.beta = 0.0;
                }
            }
            __syncthreads();
        }
    }
    if (!ctl.truth) {
        double pt[2] = {0.0, 0.0}, tt[2];
        residual64_pass<R, KB>(P, sc, bh, xh, r, pt);
        if (!reduce_d<2>(P, sc, pt, tt, epoch, parity))
            return false;
        if (t0) {
            ++reps;
            rho = tt[1];
        }
    }
    unscale_pass<R>(P, sc, xh);
    if (t0)
        write_out(P, sc, status, it, reps, sqrt(rho / bn2), sqrt(bn2));
    return true;
}

template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_pcg64(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;   // test hook: this block never arrives at a barrier
    const Scope sc = grid_scope(P);
    pcg64_body<R, KB>(P, sc);
}

// ============================================================================
// pipelined PCG, FP64
// v64: 0 xhat, 1 bhat, 2 r, 3 w(a), 4 w(b), 5 z, 6 s, 7 p
template <int R, int KB>
__device__ __forceinline__ bool pipe64_replace(const SolveParams &P, const Scope &sc, double *w,
                                               double (&tot)[3], unsigned &epoch, int &parity) {
    LANE_ROWS;
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2];
    double *z = P.v64[5], *sv = P.v64[6], *p = P.v64[7];
    // r = bhat - Ahat xhat
    double d2[2] = {0.0, 0.0};
    residual64_pass<R, KB>(P, sc, bh, xh, r, d2);
    if (!scope_sync(sc, P.sync, epoch))
        return false;
    // w = Ahat r ; s = Ahat p
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double aw[R], as[R];
        ld_rows<R>(r + row0, aw);
        ld_rows<R>(p + row0, as);
        sell_accum2<double, R, KB>(A, slice_meta(A, s, range), lane, r, p, aw, as);
        st_rows<R>(w + row0, aw);
        st_rows<R>(sv + row0, as);
    }
    if (!scope_sync(sc, P.sync, epoch))
        return false;
    // z = Ahat s ; gamma = (r,r), delta = (w,r), rho = sum d r^2
    double part[3] = {0.0, 0.0, 0.0};
    FOR_MY_SLICES(s) {
        const int row0 = s * A.C + R * lane;
        double az[R], rr[R], ww[R], dd[R];
        ld_rows<R>(sv + row0, az);
        sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, sv, az);
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
    return reduce_d<3>(P, sc, part, tot, epoch, parity);
}

struct PipeCtl {
    double alpha, beta;
    int action;   // 0 step, 1 replace, 2 exit
};

template <int R, int KB>
__device__ __forceinline__ bool pipe64_body(const SolveParams &P, const Scope &sc) {
    __syncthreads();   // the previous body of this block is done with shared state
    LANE_ROWS;
    load_slice_meta(P.A, sc.range);
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *r = P.v64[2];
    double *wa = P.v64[3], *wb = P.v64[4];
    double *z = P.v64[5], *sv = P.v64[6], *p = P.v64[7];
    __shared__ PipeCtl ctl;
    const bool t0 = threadIdx.x == 0;
    unsigned epoch = 0;
    int parity = 0, wc = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, sc, bh, xh, b2);
    zero_rows<double, R>(P, sc, p);
    zero_rows<double, R>(P, sc, z);
    zero_rows<double, R>(P, sc, sv);
    if (!reduce_d<1>(P, sc, b2, t1, epoch, parity))
        return false;
    const double bn2 = t1[0];
    if (bn2 == 0.0) {
        zero_solution(P, sc);
        write_out(P, sc, kDevOk, 0, 0, 0.0, 0.0);
        return true;
    }
    const double thr2 = P.tol * P.tol * bn2;
    double tot[3];
    if (!pipe64_replace<R, KB>(P, sc, wa, tot, epoch, parity))
        return false;
    // thread-0 state
    int reps = 1, it = 0, since = 0, status = kDevNotConverged;
    bool truth = true, fresh = true;
    double gamma = tot[0], delta = tot[1], rho = tot[2];
    double gamma_old = 0.0, alpha_old = 0.0;
    const double sg = inv_pow2(gamma), sr = inv_pow2(rho);
    for (;;) {
        if (t0) {
            const bool want = rho <= thr2 || (P.rr_period > 0 && since >= P.rr_period);
            if (want && !truth) {
                ctl.action = 1;
            } else if (truth && rho <= thr2) {
                status = kDevOk;
                ctl.action = 2;
            } else if (it >= P.maxit) {
                status = kDevNotConverged;
                ctl.action = 2;
            } else {
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
                        ctl.action = 2;
                    } else {
                        // rounding drift: replace from the true residual and restart
                        fresh = true;
                        ctl.action = 1;
                    }
                } else {
                    fresh = false;
                    ctl.action = 0;
                    ctl.beta = beta;
                    ctl.alpha = gamma / denom;
                }
            }
        }
        __syncthreads();
        const int action = ctl.action;
        if (action == 2)
            break;
        double *w = wc ? wb : wa;
        if (action == 1) {
            if (!pipe64_replace<R, KB>(P, sc, w, tot, epoch, parity))
                return false;
            if (t0) {
                ++reps;
                since = 0;
                truth = true;
                gamma = tot[0];
                delta = tot[1];
                rho = tot[2];
            }
            continue;
        }
        const double alpha = ctl.alpha, beta = ctl.beta;
        double *wn = wc ? wa : wb;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double nn[R], ww[R];
            ld_rows<R>(w + row0, ww);
#pragma unroll
            for (int j = 0; j < R; ++j)
                nn[j] = ww[j];
            sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, w, nn);
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
                g0 = fma(rr[j], rr[j], g0);
                g1 = fma(ww[j], rr[j], g1);
                g2 = fma(dd[j] * rr[j], rr[j], g2);
            }
            st_rows<R>(z + row0, zz);
            st_rows<R>(sv + row0, ss);
            st_rows<R>(p + row0, pp);
            st_rows<R>(xh + row0, xx);
            st_rows<R>(r + row0, rr);
            st_rows<R>(wn + row0, ww);
        }
        FF fp[3] = {ff_from_double(g0 * sg), ff_from_double(g1 * sg), ff_from_double(g2 * sr)};
        double tp[3];
        if (!reduce_f<3>(P, sc, fp, tp, epoch, parity))
            return false;
        wc ^= 1;
        if (t0) {
            gamma_old = gamma;
            alpha_old = alpha;
            gamma = tp[0] / sg;
            delta = tp[1] / sg;
            rho = tp[2] / sr;
            truth = false;
            ++it;
            ++since;
        }
    }
    __shared__ int s_need;   // truth is thread-0 state: broadcast the decision
    if (t0)
        s_need = !truth;
    __syncthreads();
    if (s_need) {
        double pt[2] = {0.0, 0.0}, tt[2];
        residual64_pass<R, KB>(P, sc, bh, xh, r, pt);
        if (!reduce_d<2>(P, sc, pt, tt, epoch, parity))
            return false;
        if (t0) {
            ++reps;
            rho = tt[1];
        }
    }
    unscale_pass<R>(P, sc, xh);
    if (t0)
        write_out(P, sc, status, it, reps, sqrt(rho / bn2), sqrt(bn2));
    return true;
}

template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_pipe64(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;   // test hook: this block never arrives at a barrier
    const Scope sc = grid_scope(P);
    pipe64_body<R, KB>(P, sc);
}

// ============================================================================
// mixed precision: float pipelined recurrences, FP64 solution and residual
// v64: 0 xhat, 1 bhat, 2 rt (FP64 residual, deflation only), 3 w0, 4 q0
// v32: 0 xc, 1 r, 2 w(a), 3 w(b), 4 z, 5 s, 6 p, 7 w0f, 8 q0f, 9 t0f
//
// Deflation (optional) of the constant vector: in the scaled space it is
// w0 = D^1/2 1 / ||D^1/2 1||, with q0 = Ahat w0, t0 = Ahat q0 and
// c = (w0, q0), all formed in FP64 at the start of the solve.
struct MixedCtl {
    double sigma, sigma_new;
    float a, bt, mu, f, pf;
    int action;   // 0 step, 1 replace, 2 exit
};

// The scalar state of the recurrences, kept by thread 0 in shared memory so
// that it occupies no registers in the other threads.
struct MixedState {
    double sigma, ratio, gamma, delta, eps, gamma_old, alpha_old, gamma_ref, rho;
    int it, since, reps, status, fresh, force;
};

// Gathers in flight per batch in the staged sweep, spill-free at the
// register budget of MINB resident blocks of 256 threads.
template <int R, int MINB>
struct StagedBatch {
    static constexpr int ks = MINB == 2 ? (R == 1 ? 6 : 1) : (R == 1 ? (MINB == 4 ? 3 : 6) : 2);
};

// pipe_in: the block's slice pipeline (STG), opened once per launch by the
// kernel, so that a block solving several systems in turn never
// re-initialises a live mbarrier
template <int R, int KB, bool DEFL, bool STG = false, int SKS = 6>
__device__ __forceinline__ bool mixed_body(const SolveParams &P, const Scope &sc,
                                           SlicePipe *pipe_in = nullptr) {
    __syncthreads();   // the previous body of this block is done with shared state
    LANE_ROWS;
    load_slice_meta(P.A, sc.range);
    const SellView &A = P.A;
    double *xh = P.v64[0], *bh = P.v64[1], *rt = P.v64[2], *w0 = P.v64[3], *q0 = P.v64[4];
    float *xc = P.v32[0], *r = P.v32[1], *wa = P.v32[2], *wb = P.v32[3];
    float *z = P.v32[4], *sv = P.v32[5], *p = P.v32[6];
    float *w0f = P.v32[7], *q0f = P.v32[8], *t0f = P.v32[9];
    constexpr bool defl = DEFL;   // a separate instantiation keeps the plain loop lean
    // per-warp slice pipeline: its mbarriers are set up once per solve
    SlicePipe unused;
    SlicePipe &pipe = STG ? *pipe_in : unused;
    // drains this body's copies on every exit path
    PipeGuard guard{STG ? pipe_in : nullptr, P.sync.timeout_ns};
    __shared__ MixedCtl ctl;
    const bool t0 = threadIdx.x == 0;
    unsigned epoch = 0;
    int parity = 0, wc = 0;

    double b2[1] = {0.0}, t1[1];
    prep_pass<R>(P, sc, bh, xh, b2);
    zero_rows<float, R>(P, sc, xc);
    zero_rows<float, R>(P, sc, p);
    zero_rows<float, R>(P, sc, z);
    zero_rows<float, R>(P, sc, sv);
    if (!reduce_d<1>(P, sc, b2, t1, epoch, parity))
        return false;
    const double bn2 = t1[0];
    if (bn2 == 0.0) {
        zero_solution(P, sc);
        write_out(P, sc, kDevOk, 0, 0, 0.0, 0.0);
        return true;
    }
    const double thr2 = P.tol * P.tol * bn2;
    double cW = 1.0;   // (w0, q0)
    if (defl) {
        // ||D^1/2 1||^2 = sum d
        double pd[1] = {0.0}, td[1];
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double dd[R];
            ld_rows<R>(A.dg + row0, dd);
#pragma unroll
            for (int j = 0; j < R; ++j)
                pd[0] += dd[j];
        }
        if (!reduce_d<1>(P, sc, pd, td, epoch, parity))
            return false;
        const double inv_norm = 1.0 / sqrt(td[0]);
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double ss[R];
            float sf[R];
            ld_rows<R>(A.sd + row0, ss);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                ss[j] = (row0 + j < A.n) ? ss[j] * inv_norm : 0.0;
                sf[j] = (float)ss[j];
            }
            st_rows<R>(w0 + row0, ss);
            st_rows<R>(w0f + row0, sf);
        }
        if (!scope_sync(sc, P.sync, epoch))
            return false;
        double pc[1] = {0.0}, tc[1];
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double acc[R], ww[R];
            float qf[R];
            ld_rows<R>(w0 + row0, acc);
#pragma unroll
            for (int j = 0; j < R; ++j)
                ww[j] = acc[j];
            sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, w0, acc);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                pc[0] = fma(ww[j], acc[j], pc[0]);
                qf[j] = (float)acc[j];
            }
            st_rows<R>(q0 + row0, acc);
            st_rows<R>(q0f + row0, qf);
        }
        if (!reduce_d<1>(P, sc, pc, tc, epoch, parity))
            return false;
        cW = tc[0];
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            double acc[R];
            float tf[R];
            ld_rows<R>(q0 + row0, acc);
            sell_accum<double, R, KB>(A, slice_meta(A, s, range), lane, q0, acc);
#pragma unroll
            for (int j = 0; j < R; ++j)
                tf[j] = (float)acc[j];
            st_rows<R>(t0f + row0, tf);
        }
        if (!scope_sync(sc, P.sync, epoch))
            return false;
    }
    __shared__ MixedState S;   // thread 0 only
    // Thread 0's decisions.  They run in the tail of a reduction (see
    // reduce_f), so the barrier that publishes the totals also publishes
    // ctl: replace (1) with the next float unit, step (0) with a, bt, mu,
    // or exit (2).
    auto plan_replace = [&]() {
        // The float unit sigma of the next period, a power of two near the
        // residual's norm, chosen before the true residual is formed (from
        // the recursive residual, or ||b|| at the start) so that one pass can
        // store r and s in the new unit.  Powers of two scale float
        // arithmetic exactly, so the choice only keeps the float values in
        // range.
        const double est = S.gamma > 0.0 && S.gamma < 1e300 ? S.sigma * sqrt(S.gamma) : sqrt(bn2);
        const double sigma_new = exp2(rint(log2(est)));
        const float f = (float)(S.sigma / sigma_new);
        ctl.sigma_new = sigma_new;
        ctl.f = f;
        ctl.pf = P.restart ? 0.0f : f;
        ctl.action = 1;
    };
    auto plan_step = [&]() {   // alpha, beta from fresh dot products
        const double gamma = S.gamma;
        double beta, denom;
        if (S.fresh) {
            beta = 0.0;
            denom = S.delta;
        } else {
            beta = gamma / S.gamma_old;
            denom = S.delta - beta * gamma / S.alpha_old;
        }
        if (defl)
            denom -= S.eps * S.eps / cW;
        if (!(denom > 0.0) || !(gamma > 0.0)) {
            if (S.fresh) {
                S.status = kDevNotSpd;
                ctl.action = 2;
            } else {
                S.fresh = 1;   // replace, then restart
                S.force = 1;
                plan_replace();
            }
        } else {
            S.fresh = 0;
            const double alpha = gamma / denom;
            ctl.action = 0;
            ctl.a = (float)alpha;
            ctl.bt = (float)beta;
            ctl.mu = defl ? (float)(S.eps / cW) : 0.0f;
            S.gamma_old = gamma;
            S.alpha_old = alpha;
        }
    };
    auto after_sweep = [&](const double (&t)[3]) {
        S.gamma = t[0];
        S.delta = t[1];
        S.eps = t[2];
        ++S.it;
        ++S.since;
        const bool trigger = S.force || (P.rr_period > 0 && S.since >= P.rr_period) ||
                             (P.tau > 0.0 && S.gamma <= P.tau * P.tau * S.gamma_ref) ||
                             S.ratio * S.gamma * S.sigma * S.sigma <= thr2 || S.it >= P.maxit;
        if (trigger)
            plan_replace();
        else
            plan_step();
    };
    if (t0) {
        S.sigma = 1.0;
        S.ratio = 1.0;
        S.gamma = S.delta = S.eps = 0.0;
        S.gamma_old = S.alpha_old = S.gamma_ref = 0.0;
        S.rho = bn2;
        S.it = S.since = S.reps = 0;
        S.status = kDevNotConverged;
        S.fresh = 1;
        S.force = 1;
        ctl.sigma = 1.0;
        plan_replace();
    }
    __syncthreads();
    for (;;) {
        if (ctl.action == 1) {
            const double sig = ctl.sigma;
            // U1: fold the float correction into the FP64 solution
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                double xx[R];
                float cc[R], zr[R];
                ld_rows<R>(xh + row0, xx);
                ld_rows<R>(xc + row0, cc);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    xx[j] = fma(sig, (double)cc[j], xx[j]);
                    zr[j] = 0.0f;
                }
                st_rows<R>(xh + row0, xx);
                st_rows<R>(xc + row0, zr);
            }
            if (!scope_sync(sc, P.sync, epoch))
                return false;
            // U2: FP64 true residual (deflated by the coarse correction),
            // stored in float in the new unit; in the same pass
            // s = pf (Ahat p), which needs no scalar from this replacement
            const double inv_sigma = 1.0 / ctl.sigma_new;   // power of two: exact
            const float pf = ctl.pf;
            double part[2] = {0.0, 0.0}, tot[2];
            // the residual is formed in FP64; its two norms, which steer only
            // the replacement rule and the stopping test, are summed from its
            // float rounding as float pairs (relative accuracy about 1e-7),
            // which keeps three FP64 operations a row off the FP64 pipe
            // (measured 1.8 % of the 128^3 solve)
            FF nf[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            const float inv_sigma_f = (float)inv_sigma;
            if (!defl) {
                FOR_MY_SLICES(s) {
                    const int row0 = s * A.C + R * lane;
                    double acc[R], bb[R], dd[R];
                    float as[R];
                    ld_rows<R>(xh + row0, acc);
                    ld_rows<R>(p + row0, as);
                    sell_accum_df<R, KB>(A, slice_meta(A, s, range), lane, xh, p, acc, as);
                    ld_rows<R>(bh + row0, bb);
                    ld_rows<R>(A.dg + row0, dd);
                    float rf[R], e0 = 0.0f, e1 = 0.0f;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        rf[j] = (float)(bb[j] - acc[j]) * inv_sigma_f;   // power of two: exact
                        e0 = fmaf(rf[j], rf[j], e0);
                        e1 = fmaf((float)dd[j] * rf[j], rf[j], e1);
                        as[j] *= pf;
                    }
                    nf[0] = ff_add(nf[0], FF{e0, 0.0f});
                    nf[1] = ff_add(nf[1], FF{e1, 0.0f});
                    st_rows<R>(r + row0, rf);
                    st_rows<R>(sv + row0, as);
                }
            } else {
                double pw[1] = {0.0}, tw[1];
                FOR_MY_SLICES(s) {
                    const int row0 = s * A.C + R * lane;
                    double acc[R], bb[R], ww[R];
                    float as[R];
                    ld_rows<R>(xh + row0, acc);
                    ld_rows<R>(p + row0, as);
                    sell_accum_df<R, KB>(A, slice_meta(A, s, range), lane, xh, p, acc, as);
                    ld_rows<R>(bh + row0, bb);
                    ld_rows<R>(w0 + row0, ww);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        acc[j] = bb[j] - acc[j];
                        pw[0] = fma(ww[j], acc[j], pw[0]);
                        as[j] *= pf;
                    }
                    st_rows<R>(rt + row0, acc);
                    st_rows<R>(sv + row0, as);
                }
                if (!reduce_d<1>(P, sc, pw, tw, epoch, parity))
                    return false;
                const double a0 = tw[0] / cW;   // every thread: same value, a few FP64 ops once
                // U2b: x += a0 w0 ; r -= a0 q0 (own rows only)
                FOR_MY_SLICES(s) {
                    const int row0 = s * A.C + R * lane;
                    double xx[R], rr[R], ww[R], qq[R], dd[R];
                    float rf[R];
                    ld_rows<R>(xh + row0, xx);
                    ld_rows<R>(rt + row0, rr);
                    ld_rows<R>(w0 + row0, ww);
                    ld_rows<R>(q0 + row0, qq);
                    ld_rows<R>(A.dg + row0, dd);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        xx[j] = fma(a0, ww[j], xx[j]);
                        const double rj = fma(-a0, qq[j], rr[j]);
                        part[0] = fma(rj, rj, part[0]);
                        part[1] = fma(dd[j] * rj, rj, part[1]);
                        rf[j] = (float)(rj * inv_sigma);
                    }
                    st_rows<R>(xh + row0, xx);
                    st_rows<R>(r + row0, rf);
                }
            }
            auto after_residual = [&](const double (&t)[2]) {
                ++S.reps;
                S.rho = t[1];
                if (S.rho <= thr2) {
                    S.status = kDevOk;
                    ctl.action = 2;
                } else if (S.it >= P.maxit) {
                    S.status = kDevNotConverged;
                    ctl.action = 2;
                } else if (!(t[0] > 0.0)) {
                    S.status = kDevNotSpd;
                    ctl.action = 2;
                } else {
                    S.ratio = t[1] / t[0];
                    if (P.restart)
                        S.fresh = 1;
                    else
                        S.gamma_old *= (double)ctl.f * (double)ctl.f;
                    S.sigma = ctl.sigma_new;
                    ctl.sigma = ctl.sigma_new;
                }
            };
            if (!defl) {
                // the float-pair sums are in units of sigma_new^2
                const double s2 = ctl.sigma_new * ctl.sigma_new;
                auto after_residual_f = [&](const double (&t)[2]) {
                    const double ts[2] = {t[0] * s2, t[1] * s2};
                    after_residual(ts);
                };
                if (!reduce_f<2>(P, sc, nf, tot, epoch, parity, after_residual_f))
                    return false;
            } else if (!reduce_d<2>(P, sc, part, tot, epoch, parity, after_residual)) {
                return false;
            }
            if (ctl.action == 2)
                break;
            // U3: w = Ahat r ; z = Ahat s ; p *= pf ; gamma, delta (, eps).
            // r and s are complete after the reduction's barrier and are only
            // read here.
            float *w = wc ? wb : wa;
            KahanF g0, g1, g2;
            if constexpr (STG)
                pipe_begin(A, pipe, range, warp, nwarps, lane);
            bool staged_ok = true;
            FOR_MY_SLICES(s) {
                const int row0 = s * A.C + R * lane;
                float aw[R], az[R], pp[R], qq[R];
                ld_rows<R>(r + row0, aw);
                ld_rows<R>(sv + row0, az);
                float rr[R];
#pragma unroll
                for (int j = 0; j < R; ++j)
                    rr[j] = aw[j];
                if constexpr (STG) {
                    const char *stage = pipe_front(pipe, P.sync.timeout_ns);
                    if (!stage) {
                        staged_ok = false;
                        break;
                    }
                    const int ws = slice_meta(A, s, range).y;
                    if (A.col16)
                        sell_accum2_staged<R, (SKS + 1) / 2, short>(
                            stage, pipe.val_off, ws, A.C, lane, row0, A.n_pad, r, sv,
                            aw, az);
                    else
                        sell_accum2_staged<R, (SKS + 1) / 2, int>(
                            stage, pipe.val_off, ws, A.C, lane, row0, A.n_pad, r, sv,
                            aw, az);
                    pipe_pop(A, pipe, range, nwarps, lane);
                } else {
                    sell_accum2<float, R, KB>(A, slice_meta(A, s, range), lane, r, sv, aw, az);
                }
                st_rows<R>(w + row0, aw);
                st_rows<R>(z + row0, az);
                ld_rows<R>(p + row0, pp);
                if (defl)
                    ld_rows<R>(q0f + row0, qq);
                float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    pp[j] *= pf;
                    e0 = fmaf(rr[j], rr[j], e0);
                    e1 = fmaf(aw[j], rr[j], e1);
                    if (defl)
                        e2 = fmaf(qq[j], rr[j], e2);
                }
                g0.add(e0);
                g1.add(e1);
                g2.add(e2);
                st_rows<R>(p + row0, pp);
            }
            if constexpr (STG) {
                if (!staged_ok) {
                    if (lane == 0)
                        atomicCAS(P.sync.err, 0, kDevTimeout);
                    pipe_drain(pipe, P.sync.timeout_ns);
                } else {
                    pipe_prime(A, pipe, range, warp, nwarps, lane);
                }
            }
            FF fd[3] = {g0.ff(), g1.ff(), g2.ff()};
            double td[3];
            auto after_replace = [&](const double (&t)[3]) {
                S.gamma = t[0];
                S.delta = t[1];
                S.eps = t[2];
                S.gamma_ref = t[0];
                S.since = 0;
                S.force = 0;
                plan_step();
            };
            if (!reduce_f<3>(P, sc, fd, td, epoch, parity, after_replace))
                return false;
        }
        if (ctl.action == 2)
            break;
        if (ctl.action == 1)
            continue;
        const float a = ctl.a, bt = ctl.bt, mu = ctl.mu;
        const float *w = wc ? wb : wa;
        float *wn = wc ? wa : wb;
        KahanF g0, g1, g2;   // per-thread partial dots, compensated
        // staged sweep: this warp's slices s_k = first + k * nwarps, the
        // matrix of slices k + 1 .. k + nst - 1 in flight while slice k is
        // computed
        bool staged_ok = true;
        if constexpr (STG)
            pipe_begin(A, pipe, range, warp, nwarps, lane);
        // the vectors' own rows are read and written with an evict-last L2
        // policy (measured 3 % faster at 128^3 than default caching)
        const uint64_t vpol = l2_evict_last_policy();
        FOR_MY_SLICES(s) {
            const int row0 = s * A.C + R * lane;
            float nn[R], ww[R];
            ld_rows_pol<R>(w + row0, ww, vpol);
#pragma unroll
            for (int j = 0; j < R; ++j)
                nn[j] = ww[j];
            // the row vectors do not depend on the matrix: in the staged
            // sweep their loads can go before the (memory-clobbering) wait
            // so that their latency overlaps the gathers instead of
            // following them; the plain sweep leaves the order to the
            // compiler
            float zz[R], ss[R], pp[R], xx[R], rr[R];
            float dw[R], dq[R], dt[R];
            auto load_rows = [&]() {
                ld_rows_pol<R>(z + row0, zz, vpol);
                ld_rows_pol<R>(sv + row0, ss, vpol);
                ld_rows_pol<R>(p + row0, pp, vpol);
                ld_rows_pol<R>(xc + row0, xx, vpol);
                ld_rows_pol<R>(r + row0, rr, vpol);
                if (defl) {
                    ld_rows<R>(w0f + row0, dw);
                    ld_rows<R>(q0f + row0, dq);
                    ld_rows<R>(t0f + row0, dt);
                }
            };
            constexpr bool early = STG && R <= 2;   // 4 rows a lane: registers run short
            if constexpr (early)
                load_rows();
            if constexpr (STG) {
                const char *stage = pipe_front(pipe, P.sync.timeout_ns);
                if (!stage) {
                    staged_ok = false;
                    break;
                }
                const int ws = slice_meta(A, s, range).y;
                if (A.col16)
                    sell_accum_staged<R, SKS, short>(stage, pipe.val_off, ws, A.C, lane, row0,
                                                     A.n_pad, w, nn);
                else
                    sell_accum_staged<R, SKS, int>(stage, pipe.val_off, ws, A.C, lane, row0,
                                                   A.n_pad, w, nn);
                pipe_pop(A, pipe, range, nwarps, lane);
            } else {
                sell_accum<float, R, KB>(A, slice_meta(A, s, range), lane, w, nn);
            }
            if constexpr (!early)
                load_rows();
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
            if (defl) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    zz[j] = fmaf(-mu, dt[j], fmaf(bt, zz[j], nn[j]));
                    ss[j] = fmaf(-mu, dq[j], fmaf(bt, ss[j], ww[j]));
                    pp[j] = fmaf(-mu, dw[j], fmaf(bt, pp[j], rr[j]));
                    xx[j] = fmaf(a, pp[j], xx[j]);
                    rr[j] = fmaf(-a, ss[j], rr[j]);
                    ww[j] = fmaf(-a, zz[j], ww[j]);
                    e0 = fmaf(rr[j], rr[j], e0);
                    e1 = fmaf(ww[j], rr[j], e1);
                    e2 = fmaf(dq[j], rr[j], e2);
                }
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    zz[j] = fmaf(bt, zz[j], nn[j]);
                    ss[j] = fmaf(bt, ss[j], ww[j]);
                    pp[j] = fmaf(bt, pp[j], rr[j]);
                    xx[j] = fmaf(a, pp[j], xx[j]);
                    rr[j] = fmaf(-a, ss[j], rr[j]);
                    ww[j] = fmaf(-a, zz[j], ww[j]);
                    e0 = fmaf(rr[j], rr[j], e0);
                    e1 = fmaf(ww[j], rr[j], e1);
                }
            }
            g0.add(e0);
            g1.add(e1);
            g2.add(e2);
            st_rows_pol<R>(z + row0, zz, vpol);
            st_rows_pol<R>(sv + row0, ss, vpol);
            st_rows_pol<R>(p + row0, pp, vpol);
            st_rows_pol<R>(xc + row0, xx, vpol);
            st_rows_pol<R>(r + row0, rr, vpol);
            st_rows_pol<R>(wn + row0, ww, vpol);
        }
        if constexpr (STG) {
            if (!staged_ok) {
                // a copy never completed: record it, let copies still in
                // flight land (bounded), and stop at the next barrier
                if (lane == 0)
                    atomicCAS(P.sync.err, 0, kDevTimeout);
                pipe_drain(pipe, P.sync.timeout_ns);
            } else {
                pipe_prime(A, pipe, range, warp, nwarps, lane);
            }
        }
        FF fp[3] = {g0.ff(), g1.ff(), g2.ff()};
        double tp[3];
        if (!reduce_f<3>(P, sc, fp, tp, epoch, parity, after_sweep))
            return false;
        wc ^= 1;
    }
    unscale_pass<R>(P, sc, xh);
    if (t0)
        write_out(P, sc, S.status, S.it, S.reps, sqrt(S.rho / bn2), sqrt(bn2));
    return true;
}

template <int R, int KB, bool DEFL, int MINB, bool STG>
__global__ void __launch_bounds__(256, MINB) k_mixed(SolveParams P) {
    if (P.fault_inject && blockIdx.x == 0)
        return;   // test hook: this block never arrives at a barrier
    const Scope sc = grid_scope(P);
    // the deflated loop carries three more vectors: fewer gathers in flight
    constexpr int ks = DEFL ? (StagedBatch<R, MINB>::ks + 1) / 2 : StagedBatch<R, MINB>::ks;
    SlicePipe pipe;
    if constexpr (STG)
        pipe = pipe_open(P.A, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x & 31);
    mixed_body<R, KB, DEFL, STG, ks>(P, sc, &pipe);
}

}  // namespace
