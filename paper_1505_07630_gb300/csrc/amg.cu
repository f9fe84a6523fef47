// amg.cu -- aggregation-AMG preconditioned CG (Sec. 5; Table 2's AMG-CG).
//
// The paper preconditions its CG with a V-cycle of an aggregation-based AMG
// (aggregates around a distance-2 maximal independent set, weighted-Jacobi
// smoother with omega = 4/3).  The reading implemented here:
//   aggregation   roots: a distance-2 maximal independent set formed by
//                 Luby-style rounds on SplitMix64 priorities (Bell, Dalton &
//                 Olson 2012, the parallel aggregation of CUSP); rows next to
//                 a root join it, the rest join their strongest assigned
//                 neighbour (largest |a_ij|; ties within 1e-12 of the row's
//                 largest |a_ij| go to the lower aggregate);
//   prolongator   P = (I - w D^-1 A) P_t, w = 4 / (3 rho), rho the Gershgorin
//                 bound of D^-1 A (max_i sum_j |a_ij| / a_ii);
//   coarse        A_c = P^T A P until a level has at most max_coarse rows,
//                 whose dense inverse is applied;
//   cycle         V(1,1) with the same weighted Jacobi, from zero;
//   outer         PCG (Saad Alg. 9.1) with z = V(r), stopping on the
//                 recursive ||r|| and confirming with the true residual.
// The hierarchy is built on the device (amg_setup.cuh): aggregation from a
// distance-2 maximal independent set formed in parallel, smoothed
// prolongator, transpose and Galerkin product, with the host only reading
// counts between kernels; every step of a solve runs in the kernels below,
// the scalars of the outer PCG staying on the device, so that the host only
// reads them between batches of iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ldupcg_impl.cuh"
#include "amg_setup.cuh"
#include "setup_kernels.cuh"

using namespace ldu;

namespace {

constexpr double kTie = 1e-12;
constexpr int kMaxCoarse = 4096;   // largest coarsest level (dense inverse: 128 MiB)
// a coarse level's A goes to sliced ELL when its padded slots are at most
// this multiple of its off-diagonal entries, else to CSR.  Measured on the
// 128^3 hierarchy in float: the 263k-row level (30 entries a row, 29 %
// padding) in sliced ELL made the cycle 12 % slower than CSR with 8 lanes a
// row, so only an unpadded coarse level would take it.
constexpr double kSellPad = 1.0;

// ---- host sparse matrices ----------------------------------------------------

struct HCsr {
    int64_t n = 0, m = 0;           // rows, columns
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;       // sorted within each row
    std::vector<double> val;
};

// Gauss-Jordan inverse with partial pivoting (row-major, n x n); false if singular
bool dense_inverse(const HCsr &A, std::vector<double> &inv) {
    const int64_t n = A.n;
    std::vector<double> M((size_t)(n * n), 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k)
            M[(size_t)(i * n + A.col[(size_t)k])] = A.val[(size_t)k];
    inv.assign((size_t)(n * n), 0.0);
    for (int64_t i = 0; i < n; ++i)
        inv[(size_t)(i * n + i)] = 1.0;
    for (int64_t c = 0; c < n; ++c) {
        int64_t piv = c;
        for (int64_t r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)(r * n + c)]) > std::fabs(M[(size_t)(piv * n + c)]))
                piv = r;
        if (M[(size_t)(piv * n + c)] == 0.0)
            return false;
        if (piv != c)
            for (int64_t k = 0; k < n; ++k) {
                std::swap(M[(size_t)(c * n + k)], M[(size_t)(piv * n + k)]);
                std::swap(inv[(size_t)(c * n + k)], inv[(size_t)(piv * n + k)]);
            }
        const double p = 1.0 / M[(size_t)(c * n + c)];
        for (int64_t k = 0; k < n; ++k) {
            M[(size_t)(c * n + k)] *= p;
            inv[(size_t)(c * n + k)] *= p;
        }
        for (int64_t r = 0; r < n; ++r) {
            if (r == c)
                continue;
            const double f = M[(size_t)(r * n + c)];
            if (f == 0.0)
                continue;
            for (int64_t k = 0; k < n; ++k) {
                M[(size_t)(r * n + k)] -= f * M[(size_t)(c * n + k)];
                inv[(size_t)(r * n + k)] -= f * inv[(size_t)(c * n + k)];
            }
        }
    }
    return true;
}

// ---- device layouts ----------------------------------------------------------
//
// The fine level keeps A's off-diagonal part in sliced ELL with 32-row
// slices (one warp per slice, one thread per row, slot k of row s*32+i at
// sp[s] + 32k + i; padding slots hold column 0 and value 0): a mesh's rows
// are short and even, so padding is near zero and every load coalesces.
// Coarse levels (tens of entries a row, uneven), P and R = P^T are CSR read
// by groups of LPR lanes per row, LPR a power of two sized from the mean row
// length.  Every level also keeps its diagonal d and w/d.  Values exist in
// double and in float over one shared index structure: the FP64 cycle
// follows the method in double; the mixed solve applies the cycle in float
// (this GPU's FP64 pipe, about 2 FMAs per SM and clock, would otherwise bound
// the sparse products) inside the FP64 outer CG.

template <typename T>
struct DSell {
    int n;
    const int *sp, *sw, *col;
    const T *val;
    const short *c16 = nullptr;   // column - row per slot when every offset fits (else null)
};

template <typename T>
struct DCsr {
    int n;
    const int *ptr, *col;
    const T *val;
};

// scalars of the outer PCG, resident on the device between kernels
struct AmgScalars {
    double tol2, bn2, thr2, rr, rz, pq, alpha, beta;
    double gamma, delta, gamma_old, alpha_old;   // pipelined CG
    int it, maxit;
    int done;      // 1: the remaining kernels of the iteration return at once
    int conv;      // 1: the recursive residual met the tolerance
    int status;    // LDU_OK, LDU_NOT_CONVERGED or LDU_ERR_NOT_SPD
    int restart;   // 1: the next search direction is z itself
};

constexpr int kWarps = 8;                 // warps (slices) per block
constexpr int kThreads = kWarps * 32;
constexpr int kBlocksPerSm = 8;           // every kernel is built to keep 8 blocks resident (32 registers)
constexpr int kMaxBlocks = 152 * kBlocksPerSm;   // grid cap: one wave of 8 blocks on each of 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(kFullMask, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(kFullMask, v, o);
    return v;
}

// Deterministic grid sum of NV values: every block stores its partial in
// part[NV * block]; the last block to finish adds the partials in a fixed
// order (strided over its threads, then a fixed tree) into tot (thread 0)
// and re-arms the counter.  Returns true in every thread of the last block.
template <int NV>
__device__ bool grid_sum_last(const double (&v)[NV], double *part, unsigned *count,
                              double (&tot)[NV]) {
    __shared__ double sm[NV][kWarps];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0)
            sm[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w)
                s += sm[k][w];
            part[NV * blockIdx.x + k] = s;
        }
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last)
        return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads)
            s[k] += __ldcg(part + NV * b + k);
        s[k] = warp_sum(s[k]);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k)
            sm[k][warp] = s[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w)
                t += sm[k][w];
            tot[k] = t;
        }
        *count = 0u;
    }
    return true;
}

// (r, z) of a new preconditioned residual: beta of the next direction, or
// only (r, z) when the search restarts.  rzo = (r_new, z_old) gives the
// Polak-Ribiere beta of flexible CG (the float cycle), 0 the Fletcher-Reeves
// beta of Saad Alg. 9.1 (the FP64 cycle).
__device__ __forceinline__ void set_rz(AmgScalars *S, double rz, double rzo) {
    if (S->restart) {
        S->rz = rz;
    } else {
        S->beta = (rz - rzo) / S->rz;
        S->rz = rz;
    }
}

// sum over the off-diagonal slots of row s*32+i of a_ij f(j), in slot order
template <typename T, typename F>
__device__ __forceinline__ T sell_row(const DSell<T> &A, int s, int i, F f) {
    const int w = A.sw[s];
    const int base = A.sp[s] + i;
    T acc = T(0);
    int k = 0;
    if (A.c16) {   // 16-bit offsets: 2 instead of 4 bytes per slot (padding slots point at the row)
        // rows past n in the last slice hold only padding: they gather at row n - 1 (value 0)
        const int row = min(s * 32 + i, A.n - 1);
        for (; k + 2 <= w; k += 2) {
            const int c0 = row + __ldcs(A.c16 + base + k * 32);
            const int c1 = row + __ldcs(A.c16 + base + (k + 1) * 32);
            const T v0 = __ldcs(A.val + base + k * 32), v1 = __ldcs(A.val + base + (k + 1) * 32);
            const T f0 = f(c0), f1 = f(c1);
            acc = fma(v0, f0, acc);
            acc = fma(v1, f1, acc);
        }
        if (k < w)
            acc = fma(__ldcs(A.val + base + k * 32), f(row + __ldcs(A.c16 + base + k * 32)), acc);
        return acc;
    }
    for (; k + 2 <= w; k += 2) {
        const int c0 = __ldg(A.col + base + k * 32), c1 = __ldg(A.col + base + (k + 1) * 32);
        const T v0 = __ldcs(A.val + base + k * 32), v1 = __ldcs(A.val + base + (k + 1) * 32);
        const T f0 = f(c0), f1 = f(c1);
        acc = fma(v0, f0, acc);
        acc = fma(v1, f1, acc);
    }
    if (k < w)
        acc = fma(__ldcs(A.val + base + k * 32), f(__ldg(A.col + base + k * 32)), acc);
    return acc;
}

#define FOR_SLICES(A)                                                                         \
    for (int s = blockIdx.x * kWarps + (threadIdx.x >> 5), nsl = ((A).n + 31) >> 5; s < nsl; \
         s += gridDim.x * kWarps)

// rows of a CSR matrix by groups of LPR lanes: epi(row, sum_k val_k g(col_k),
// pre(row)) in the group's first lane, pre(row) being loaded before the sum.
// Rows are taken 32/LPR at a time per warp, so every lane of a warp reaches
// each shuffle; each lane adds its entries (every LPR-th) in order.
template <int LPR, typename T, typename Pre, typename G, typename E>
__device__ __forceinline__ void csr_rows(const DCsr<T> &M, Pre pre, G g, E epi) {
    constexpr int GPW = 32 / LPR;
    const int lane = threadIdx.x & 31, grp = lane / LPR, gl = lane % LPR;
    const int warp = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kThreads) >> 5);
    for (int base = warp * GPW; base < M.n; base += nwarps * GPW) {
        const int row = base + grp;
        const bool lead = gl == 0 && row < M.n;
        decltype(pre(0)) pv{};
        if (lead)
            pv = pre(row);
        T acc = T(0);
        if (row < M.n) {
            const int e = M.ptr[row + 1];
            for (int k = M.ptr[row] + gl; k < e; k += LPR)
                acc = fma(__ldcs(M.val + k), g(__ldcs(M.col + k)), acc);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1)
            acc += __shfl_down_sync(kFullMask, acc, o, LPR);
        if (lead)
            epi(row, acc, pv);
    }
}

template <typename T>
struct Row3 {
    T a, b, c;
};

// the residual after pre-smoothing from zero, t = (w/d) b having been
// written by the producer of b:  r = b - A t
template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_pre(DSell<T> A, const T *__restrict__ d,
                                                      const T *__restrict__ b,
                                                      const T *__restrict__ t,
                                                      T *__restrict__ r, const int *skip) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const T off = sell_row(A, s, lane, [&](int c) { return t[c]; });
        if (row < A.n)
            r[row] = b[row] - fma(d[row], t[row], off);
    }
}

template <int LPR, typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_pre_csr(DCsr<T> A, const T *__restrict__ d,
                                                          const T *__restrict__ b,
                                                          const T *__restrict__ t,
                                                          T *__restrict__ r, const int *skip) {
    if (skip && *skip)
        return;
    csr_rows<LPR>(
        A, [&](int row) { return Row3<T>{b[row], d[row], t[row]}; }, [&](int c) { return t[c]; },
        [&](int row, T off, Row3<T> v) { r[row] = v.a - fma(v.b, v.c, off); });
}

// post-smoothing: x = t + (w/d) (b - A t).  With DOT (level 0 inside the
// outer PCG: b is the outer residual in the cycle's precision, x its
// preconditioned z) also (r, z_new) and, with PR, (r, z_old) into the outer
// scalars: each thread sums its few rows in T, the grid in double (a float
// cycle's dot products need no more: the float z carries 1e-7 already)
template <typename T, bool DOT, bool PR>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_post(DSell<T> A, const T *__restrict__ d,
                                                       const T *__restrict__ wd,
                                                       const T *__restrict__ b,
                                                       const T *__restrict__ t,
                                                       T *__restrict__ x, const int *skip,
                                                       AmgScalars *S, double *part,
                                                       unsigned *count) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    T dot = T(0), doto = T(0);   // this thread's rows (a handful), then FP64 across threads
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const T off = sell_row(A, s, lane, [&](int c) { return t[c]; });
        if (row < A.n) {
            const T bi = b[row], ti = t[row];
            const T xi = fma(wd[row], bi - fma(d[row], ti, off), ti);
            if (DOT) {
                if (PR)
                    doto = fma(bi, x[row], doto);
                dot = fma(bi, xi, dot);
            }
            x[row] = xi;
        }
    }
    if (DOT) {
        double v[2] = {(double)dot, (double)doto}, tot[2];
        if (grid_sum_last<2>(v, part, count, tot) && threadIdx.x == 0)
            set_rz(S, tot[0], tot[1]);
    }
}

template <int LPR, typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_post_csr(DCsr<T> A, const T *__restrict__ d,
                                                           const T *__restrict__ wd,
                                                           const T *__restrict__ b,
                                                           const T *__restrict__ t,
                                                           T *__restrict__ x, const int *skip) {
    if (skip && *skip)
        return;
    csr_rows<LPR>(
        A, [&](int row) { return Row3<T>{b[row], d[row], t[row]}; }, [&](int c) { return t[c]; },
        [&](int row, T off, Row3<T> v) { x[row] = fma(wd[row], v.a - fma(v.b, v.c, off), v.c); });
}

// b_c = R r, and t_c = (w/d)_c b_c for the coarse level's pre-smoothing
// (wdc null when the coarse level is the coarsest)
template <int LPR, typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_restrict(DCsr<T> R, const T *__restrict__ r,
                                                           const T *__restrict__ wdc,
                                                           T *__restrict__ bc, T *__restrict__ tc,
                                                           const int *skip) {
    if (skip && *skip)
        return;
    csr_rows<LPR>(
        R, [&](int row) { return wdc ? wdc[row] : T(0); }, [&](int c) { return r[c]; },
        [&](int row, T v, T w) {
            bc[row] = v;
            if (wdc)
                tc[row] = w * v;
        });
}

// t += P x_c
template <int LPR, typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_prolong(DCsr<T> P, const T *__restrict__ xc,
                                                          T *__restrict__ t, const int *skip) {
    if (skip && *skip)
        return;
    csr_rows<LPR>(
        P, [&](int row) { return t[row]; }, [&](int c) { return xc[c]; },
        [&](int row, T v, T t0) { t[row] = t0 + v; });
}

// x = Minv b on the coarsest level, one warp per row; with DOT (a system
// that is its own coarsest level) also the outer PCG's dot products
template <typename T, bool DOT, bool PR>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_dense(int n, const T *__restrict__ Minv,
                                                        const T *__restrict__ b,
                                                        T *__restrict__ x, const int *skip,
                                                        AmgScalars *S, double *part,
                                                        unsigned *count) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    T dot = T(0), doto = T(0);
    for (int row = blockIdx.x * kWarps + (threadIdx.x >> 5); row < n; row += gridDim.x * kWarps) {
        T s = T(0);
        for (int k = lane; k < n; k += 32)
            s = fma(Minv[(size_t)row * n + k], b[k], s);
        s = warp_sum(s);
        if (lane == 0) {
            if (DOT) {
                if (PR)
                    doto = fma(b[row], x[row], doto);
                dot = fma(b[row], s, dot);
            }
            x[row] = s;
        }
    }
    if (DOT) {
        double v[2] = {(double)dot, (double)doto}, tot[2];
        if (grid_sum_last<2>(v, part, count, tot) && threadIdx.x == 0)
            set_rz(S, tot[0], tot[1]);
    }
}

// the cycle's input from a double vector: t = (w/d) b (wd null: none) and,
// for a float cycle, bv = b rounded (bv null: the cycle reads b itself)
template <typename T>
__device__ __forceinline__ void cycle_input(int i, double bi, const T *wd, T *t, T *bv) {
    if (bv)
        bv[i] = (T)bi;
    if (wd)
        t[i] = wd[i] * (T)bi;
}

// stand-alone cycle input
template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_scale(int n, const T *__restrict__ wd,
                                                        const T *__restrict__ b,
                                                        T *__restrict__ t) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
        t[i] = wd[i] * b[i];
}

// r = b - A x (FP64) with (r, r) and (b, b) reduced, and the cycle's input
// from r; mode 0 starts a solve (bn2, thr2, rr), mode 1 measures the true
// residual (rr only); both make the next direction restart
template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_residual(DSell<double> A,
                                                           const double *__restrict__ d,
                                                           const double *__restrict__ b,
                                                           const double *__restrict__ x,
                                                           double *__restrict__ r,
                                                           const T *__restrict__ wd,
                                                           T *__restrict__ t, T *__restrict__ bv,
                                                           int mode, AmgScalars *S, double *part,
                                                           unsigned *count) {
    const int lane = threadIdx.x & 31;
    double rr = 0.0, bb = 0.0;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off = sell_row(A, s, lane, [&](int c) { return x[c]; });
        if (row < A.n) {
            const double bi = b[row];
            const double ri = bi - fma(d[row], x[row], off);
            r[row] = ri;
            cycle_input(row, ri, wd, t, bv);
            rr = fma(ri, ri, rr);
            bb = fma(bi, bi, bb);
        }
    }
    double v[2] = {rr, bb}, tot[2];
    if (grid_sum_last<2>(v, part, count, tot) && threadIdx.x == 0) {
        S->rr = tot[0];
        if (mode == 0) {
            S->bn2 = tot[1];
            S->thr2 = S->tol2 * tot[1];
        }
        S->done = 0;
        S->conv = 0;
        S->restart = 1;
    }
}

// p = z + beta p, or p = z after a restart
template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_p(int n, const T *__restrict__ z,
                                                    double *__restrict__ p,
                                                    const AmgScalars *S) {
    if (S->done)
        return;
    const int restart = S->restart;
    const double beta = S->beta;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
        p[i] = restart ? (double)z[i] : fma(beta, p[i], (double)z[i]);
}

// q = A p with (p, q) reduced into alpha
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_q(DSell<double> A, const double *__restrict__ d,
                                                    const double *__restrict__ p,
                                                    double *__restrict__ q, AmgScalars *S,
                                                    double *part, unsigned *count) {
    if (S->done)
        return;
    const int lane = threadIdx.x & 31;
    double pq = 0.0;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off = sell_row(A, s, lane, [&](int c) { return p[c]; });
        if (row < A.n) {
            const double pi = p[row];
            const double qi = fma(d[row], pi, off);
            q[row] = qi;
            pq = fma(pi, qi, pq);
        }
    }
    double v[1] = {pq}, tot[1];
    if (grid_sum_last<1>(v, part, count, tot) && threadIdx.x == 0) {
        S->pq = tot[0];
        S->restart = 0;
        if (!(tot[0] > 0.0) || !(S->rz > 0.0)) {
            S->status = LDU_ERR_NOT_SPD;
            S->done = 1;
        } else {
            S->alpha = S->rz / tot[0];
        }
    }
}

// x += alpha p; r -= alpha q and the cycle's input from r; (r, r) reduced;
// the iteration is counted and the loop stops when the recursive residual
// meets the tolerance or maxit iterations have run
template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_amg_xr(int n, const double *__restrict__ p,
                                                     const double *__restrict__ q,
                                                     double *__restrict__ x,
                                                     double *__restrict__ r,
                                                     const T *__restrict__ wd, T *__restrict__ t,
                                                     T *__restrict__ bv, AmgScalars *S,
                                                     double *part, unsigned *count) {
    if (S->done)
        return;
    const double alpha = S->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        cycle_input(i, ri, wd, t, bv);
        rr = fma(ri, ri, rr);
    }
    double v[1] = {rr}, tot[1];
    if (grid_sum_last<1>(v, part, count, tot) && threadIdx.x == 0) {
        S->rr = tot[0];
        S->it += 1;
        if (tot[0] <= S->thr2) {
            S->conv = 1;
            S->done = 1;
        } else if (S->it >= S->maxit) {
            S->status = LDU_NOT_CONVERGED;
            S->done = 1;
        }
    }
}

// ---- pipelined PCG (Ghysels & Vanroose) with the FP64 cycle ------------------

// w = A u with gamma = (r, u) and delta = (w, u); the cycle's next input
// t0 = (w/d) w; the recurrences restart (beta = 0) at the next update
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_pp_init(DSell<double> A, const double *__restrict__ d,
                                                      const double *__restrict__ u,
                                                      const double *__restrict__ r,
                                                      double *__restrict__ w,
                                                      const double *__restrict__ wd,
                                                      double *__restrict__ t, AmgScalars *S,
                                                      double *part, unsigned *count) {
    const int lane = threadIdx.x & 31;
    double g = 0.0, dl = 0.0;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off = sell_row(A, s, lane, [&](int c) { return u[c]; });
        if (row < A.n) {
            const double ui = u[row];
            const double wi = fma(d[row], ui, off);
            w[row] = wi;
            if (wd)
                t[row] = wd[row] * wi;
            g = fma(r[row], ui, g);
            dl = fma(wi, ui, dl);
        }
    }
    double v[2] = {g, dl}, tot[2];
    if (grid_sum_last<2>(v, part, count, tot) && threadIdx.x == 0) {
        S->gamma = tot[0];
        S->delta = tot[1];
        S->restart = 1;
        S->done = 0;
        S->conv = 0;
    }
}

// y = A x on the fine level (FP64)
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) k_pp_spmv(DSell<double> A, const double *__restrict__ d,
                                                      const double *__restrict__ x,
                                                      double *__restrict__ y,
                                                      const AmgScalars *S) {
    if (S->done)
        return;
    const int lane = threadIdx.x & 31;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off = sell_row(A, s, lane, [&](int c) { return x[c]; });
        if (row < A.n)
            y[row] = fma(d[row], x[row], off);
    }
}

struct PipeVecs {
    const double *m, *nv;
    double *z, *q, *s, *p, *x, *r, *u, *w;
};

// one pipelined step: beta and alpha from the last step's scalars (every
// thread forms the same values), the eight recurrences, the cycle's next
// input t0 = (w/d) w, and (r, u), (w, u), (r, r) for the next step; the
// last block counts the step and tests convergence
constexpr int kUpdateBlocksPerSm = 6;   // the eight-vector update needs more than 32 registers
__global__ void __launch_bounds__(kThreads, kUpdateBlocksPerSm) k_pp_update(int n, PipeVecs V,
                                                        const double *__restrict__ wd,
                                                        double *__restrict__ t, AmgScalars *S,
                                                        double *part, unsigned *count) {
    if (S->done)
        return;
    const int restart = S->restart;
    const double gamma = S->gamma, delta = S->delta;
    double beta = 0.0, den = delta;
    if (!restart) {
        beta = gamma / S->gamma_old;
        den = delta - beta * gamma / S->alpha_old;
    }
    const bool ok = den > 0.0 && gamma > 0.0;
    const double alpha = ok ? gamma / den : 0.0;
    double g = 0.0, dl = 0.0, rr = 0.0;
    if (ok) {
        for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
            double zi, qi, si, pi;
            if (restart) {
                zi = V.nv[i];
                qi = V.m[i];
                si = V.w[i];
                pi = V.u[i];
            } else {
                zi = fma(beta, V.z[i], V.nv[i]);
                qi = fma(beta, V.q[i], V.m[i]);
                si = fma(beta, V.s[i], V.w[i]);
                pi = fma(beta, V.p[i], V.u[i]);
            }
            V.z[i] = zi;
            V.q[i] = qi;
            V.s[i] = si;
            V.p[i] = pi;
            V.x[i] = fma(alpha, pi, V.x[i]);
            const double ri = fma(-alpha, si, V.r[i]);
            const double ui = fma(-alpha, qi, V.u[i]);
            const double wi = fma(-alpha, zi, V.w[i]);
            V.r[i] = ri;
            V.u[i] = ui;
            V.w[i] = wi;
            if (wd)
                t[i] = wd[i] * wi;
            g = fma(ri, ui, g);
            dl = fma(wi, ui, dl);
            rr = fma(ri, ri, rr);
        }
    }
    double v[3] = {g, dl, rr}, tot[3];
    if (grid_sum_last<3>(v, part, count, tot) && threadIdx.x == 0) {
        if (!ok) {
            if (restart) {   // (u, A u) <= 0 on a fresh start: A is not SPD
                S->status = LDU_ERR_NOT_SPD;
                S->done = 1;
                return;
            }
            // the denominator is (p, A p) > 0 in exact arithmetic: a
            // non-positive one is drift of the recurrences (near the limit
            // of FP64), so this run ends as a converged one would and the
            // host confirms it with the true residual, restarting from it
            S->conv = 1;
            S->done = 1;
            return;
        }
        S->gamma_old = gamma;
        S->alpha_old = alpha;
        S->gamma = tot[0];
        S->delta = tot[1];
        S->rr = tot[2];
        S->restart = 0;
        S->it += 1;
        if (tot[2] <= S->thr2) {
            S->conv = 1;
            S->done = 1;
        } else if (S->it >= S->maxit) {
            S->status = LDU_NOT_CONVERGED;
            S->done = 1;
        }
    }
}

int grid_rows(int64_t n) {   // blocks for one thread per row (one warp per 32-row slice)
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, kMaxBlocks));
}

int grid_warps(int64_t n) {  // blocks for one warp per row
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kWarps - 1) / kWarps, kMaxBlocks));
}

int grid_lpr(int64_t n, int lpr) {   // blocks for lpr lanes per row
    return (int)std::max<int64_t>(
        1, std::min<int64_t>((n * lpr + kThreads - 1) / kThreads, kMaxBlocks));
}

// lanes per row: the power of two nearest a quarter of the mean row length, 1..32
int lpr_for(int64_t rows, int64_t nnz) {
    const double q = rows > 0 ? 0.25 * (double)nnz / (double)rows : 0.0;
    int l = 1;
    while (l < 32 && q >= l * 1.4142135623730951)
        l *= 2;
    return l;
}

// launchers of the CSR kernels at their lanes-per-row instance
#define AMG_LPR_LAUNCHER(NAME, KERNEL)                                                    \
    template <typename T, typename... Args>                                               \
    void NAME(int lpr, int grid, cudaStream_t st, Args... args) {                         \
        switch (lpr) {                                                                    \
        case 1: KERNEL<1, T><<<grid, kThreads, 0, st>>>(args...); break;                  \
        case 2: KERNEL<2, T><<<grid, kThreads, 0, st>>>(args...); break;                  \
        case 4: KERNEL<4, T><<<grid, kThreads, 0, st>>>(args...); break;                  \
        case 8: KERNEL<8, T><<<grid, kThreads, 0, st>>>(args...); break;                  \
        case 16: KERNEL<16, T><<<grid, kThreads, 0, st>>>(args...); break;                \
        default: KERNEL<32, T><<<grid, kThreads, 0, st>>>(args...); break;                \
        }                                                                                 \
    }
AMG_LPR_LAUNCHER(launch_pre_csr, k_amg_pre_csr)
AMG_LPR_LAUNCHER(launch_post_csr, k_amg_post_csr)
AMG_LPR_LAUNCHER(launch_restrict, k_amg_restrict)
AMG_LPR_LAUNCHER(launch_prolong, k_amg_prolong)
#undef AMG_LPR_LAUNCHER

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src, int64_t *bytes) {
    *dst = nullptr;
    const size_t sz = sizeof(T) * std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc((void **)dst, sz);
    if (e != cudaSuccess)
        return e;
    *bytes += (int64_t)sz;
    if (!src.empty())
        e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

// a double array and its float rounding
cudaError_t upload2(double **d64, float **d32, const std::vector<double> &src, int64_t *bytes) {
    cudaError_t e = upload(d64, src, bytes);
    if (e != cudaSuccess)
        return e;
    const std::vector<float> f(src.begin(), src.end());
    return upload(d32, f, bytes);
}

template <typename T>
cudaError_t alloc(T **dst, int64_t count, int64_t *bytes) {
    *dst = nullptr;
    const size_t sz = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = cudaMalloc((void **)dst, sz);
    if (e == cudaSuccess)
        *bytes += (int64_t)sz;
    return e;
}

}  // namespace

// the values and vectors of one level in one precision
template <typename T>
struct LevelVals {
    T *a_val = nullptr, *d = nullptr, *wd = nullptr, *p_val = nullptr, *r_val = nullptr;
    T *t = nullptr, *r = nullptr;   // smoothed iterate, residual
    T *x = nullptr, *b = nullptr;   // level >= 1: cycle output and input
};

// one level above the coarsest
struct amg_level {
    int64_t n = 0, nnz = 0;
    double w = 0.0;
    // A's off-diagonal part: sliced ELL on level 0 (a_sp, a_sw), CSR on
    // coarser levels (a_ptr)
    int *a_sp = nullptr, *a_sw = nullptr, *a_ptr = nullptr, *a_col = nullptr;
    short *a_c16 = nullptr;                   // sliced ELL's columns as offsets from the row (float cycle)
    int *p_ptr = nullptr, *p_col = nullptr;   // P: n x n_next
    int *r_ptr = nullptr, *r_col = nullptr;   // R = P^T: n_next x n
    int a_lpr = 1, p_lpr = 1, r_lpr = 1;      // lanes per row of the CSR reads
    bool a_sell = false;                      // A in sliced ELL (else CSR)
    int64_t r_rows = 0;                       // rows of R (= next level's)
    LevelVals<double> v64;
    LevelVals<float> v32;
    int *agg = nullptr;                       // aggregate of every row (device)
    template <typename T>
    const LevelVals<T> &v() const;
    template <typename T>
    DSell<T> A() const {
        return DSell<T>{(int)n, a_sp, a_sw, a_col, v<T>().a_val,
                        std::is_same<T, float>::value ? a_c16 : nullptr};
    }
    template <typename T>
    DCsr<T> Acsr() const { return DCsr<T>{(int)n, a_ptr, a_col, v<T>().a_val}; }
    template <typename T>
    DCsr<T> P() const { return DCsr<T>{(int)n, p_ptr, p_col, v<T>().p_val}; }
    template <typename T>
    DCsr<T> R() const { return DCsr<T>{(int)r_rows, r_ptr, r_col, v<T>().r_val}; }
};
template <>
const LevelVals<double> &amg_level::v<double>() const { return v64; }
template <>
const LevelVals<float> &amg_level::v<float>() const { return v32; }

template <typename T>
struct CoarseVals {
    T *inv = nullptr, *x = nullptr, *b = nullptr;
};

struct ldu_amg {
    int device = 0;
    int64_t n = 0;
    std::vector<amg_level> lev;     // every level that has a prolongator
    // the fine matrix in double for the outer CG (level 0's when it exists)
    int *f_sp = nullptr, *f_sw = nullptr, *f_col = nullptr;
    double *f_val = nullptr, *f_d = nullptr;
    int64_t nc = 0, c_nnz = 0;      // coarsest rows and non-zeros
    CoarseVals<double> c64;         // coarsest dense inverse (row-major), vectors
    CoarseVals<float> c32;
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    float *r32 = nullptr, *z32 = nullptr;   // float cycle's input and output
    double *pv[7] = {};             // pipelined CG: u, w, m, n, z, q, s (allocated on first use)
    // one outer iteration captured as a CUDA graph per loop kind (CG with the
    // float cycle, CG with the FP64 cycle, pipelined), keyed by the caller's x
    cudaStream_t cap = nullptr;     // private stream the iterations are captured on
    cudaGraphExec_t body[3] = {};
    const void *body_x[3] = {};
    double *part = nullptr;
    unsigned *count = nullptr;
    AmgScalars *S = nullptr;        // device
    AmgScalars *S_host = nullptr;   // pinned
    int64_t device_bytes = 0;
    template <typename T>
    const CoarseVals<T> &c() const;
    DSell<double> fine() const {
        return lev.empty() ? DSell<double>{(int)n, f_sp, f_sw, f_col, f_val} : lev[0].A<double>();
    }
    const double *fine_d() const { return lev.empty() ? f_d : lev[0].v64.d; }
};
template <>
const CoarseVals<double> &ldu_amg::c<double>() const { return c64; }
template <>
const CoarseVals<float> &ldu_amg::c<float>() const { return c32; }

namespace {

template <typename T>
void free_vals(LevelVals<T> &v) {
    void *ptrs[] = {v.a_val, v.d, v.wd, v.p_val, v.r_val, v.t, v.r, v.x, v.b};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
}

void free_amg(ldu_amg *M) {
    if (!M)
        return;
    for (auto &L : M->lev) {
        void *ptrs[] = {L.a_sp,  L.a_sw,  L.a_ptr, L.a_col, L.a_c16,
                        L.p_ptr, L.p_col, L.r_ptr, L.r_col, L.agg};
        for (void *p : ptrs)
            if (p)
                cudaFree(p);
        free_vals(L.v64);
        free_vals(L.v32);
    }
    void *ptrs[] = {M->f_sp,   M->f_sw,   M->f_col,  M->f_val, M->f_d,    M->c64.inv, M->c64.x,
                    M->c64.b,  M->c32.inv, M->c32.x, M->c32.b, M->r,      M->z,       M->p,
                    M->q,      M->r32,    M->z32,   M->part,   M->count,   M->S};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    for (double *v : M->pv)
        if (v)
            cudaFree(v);
    for (cudaGraphExec_t g : M->body)
        if (g)
            cudaGraphExecDestroy(g);
    if (M->cap)
        cudaStreamDestroy(M->cap);
    if (M->S_host)
        cudaFreeHost(M->S_host);
    delete M;
}

// x = V(b) from level l down, in precision T.  On entry the level's t holds
// (w/d) b (the producer of b wrote it).  Level 0's b and x are the caller's;
// with DOT the last kernel also reduces the outer PCG's dot products from
// the double residual r64 (PR: the flexible-CG beta).
template <typename T>
int vcycle(ldu_amg *M, size_t l, const T *b, T *x, bool dot, const int *skip, cudaStream_t st) {
    constexpr bool pr = std::is_same<T, float>::value;
    if (l == M->lev.size()) {
        const CoarseVals<T> &C = M->c<T>();
        const int g = grid_warps(M->nc);
        if (!dot)
            k_amg_dense<T, false, false><<<g, kThreads, 0, st>>>((int)M->nc, C.inv, b, x, skip,
                                                                 nullptr, nullptr, nullptr);
        else
            k_amg_dense<T, true, pr><<<g, kThreads, 0, st>>>((int)M->nc, C.inv, b, x, skip, M->S,
                                                             M->part, M->count);
        return cuda_status(cudaGetLastError());
    }
    const amg_level &L = M->lev[l];
    const LevelVals<T> &V = L.v<T>();
    if (L.a_sell)
        k_amg_pre<T><<<grid_rows(L.n), kThreads, 0, st>>>(L.A<T>(), V.d, b, V.t, V.r, skip);
    else
        launch_pre_csr<T>(L.a_lpr, grid_lpr(L.n, L.a_lpr), st, L.Acsr<T>(), (const T *)V.d, b,
                          (const T *)V.t, V.r, skip);
    const bool last = l + 1 == M->lev.size();
    T *bn = last ? M->c<T>().b : M->lev[l + 1].v<T>().b;
    T *xn = last ? M->c<T>().x : M->lev[l + 1].v<T>().x;
    const T *wdn = last ? nullptr : M->lev[l + 1].v<T>().wd;
    T *tn = last ? nullptr : M->lev[l + 1].v<T>().t;
    launch_restrict<T>(L.r_lpr, grid_lpr(L.r_rows, L.r_lpr), st, L.R<T>(), (const T *)V.r, wdn, bn,
                       tn, skip);
    const int rc = vcycle<T>(M, l + 1, bn, xn, false, skip, st);
    if (rc != LDU_OK)
        return rc;
    launch_prolong<T>(L.p_lpr, grid_lpr(L.n, L.p_lpr), st, L.P<T>(), (const T *)xn, V.t, skip);
    if (L.a_sell) {
        const int g = grid_rows(L.n);
        if (!dot)
            k_amg_post<T, false, false><<<g, kThreads, 0, st>>>(L.A<T>(), V.d, V.wd, b, V.t, x,
                                                                skip, nullptr, nullptr, nullptr);
        else
            k_amg_post<T, true, pr><<<g, kThreads, 0, st>>>(L.A<T>(), V.d, V.wd, b, V.t, x, skip,
                                                            M->S, M->part, M->count);
    } else {
        launch_post_csr<T>(L.a_lpr, grid_lpr(L.n, L.a_lpr), st, L.Acsr<T>(), (const T *)V.d,
                           (const T *)V.wd, b, (const T *)V.t, x, skip);
    }
    return cuda_status(cudaGetLastError());
}

// The graph of one outer iteration of loop `kind` for the caller's x: the
// cached one when x is the same, else the launches `body` makes on the
// private stream are captured and replace the cached graph's parameters (or
// a new graph is instantiated).  Every kernel of an iteration returns at once
// when the scalars say the loop has stopped, so the graph can be launched
// for a whole batch of iterations.
template <typename F>
int iteration_graph(ldu_amg *M, int kind, const void *x, F body, cudaGraphExec_t *out) {
    if (M->body[kind] && M->body_x[kind] == x) {
        *out = M->body[kind];
        return LDU_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(M->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return cuda_status(e);
    const int rc = body(M->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(M->cap, &graph);
    if (rc != LDU_OK || e != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc != LDU_OK ? rc : cuda_status(e);
    }
    bool updated = false;
    if (M->body[kind]) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(M->body[kind], graph, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();   // clear the update's error state
            cudaGraphExecDestroy(M->body[kind]);
            M->body[kind] = nullptr;
        }
    }
    if (!updated)
        e = cudaGraphInstantiate(&M->body[kind], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        M->body[kind] = nullptr;
        M->body_x[kind] = nullptr;
        return cuda_status(e);
    }
    M->body_x[kind] = x;
    *out = M->body[kind];
    return LDU_OK;
}

// the outer scalars to the pinned host copy (synchronises st)
int read_scalars(ldu_amg *M, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(M->S_host, M->S, sizeof(AmgScalars), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

// The outer loop shared by AMG-PCG and AMG-PipeCG.  residual(mode) queues
// r = b - A x with the cycle's input (mode 0 also sets bn2 and the
// threshold, see k_amg_residual); resume() queues the restart of the search
// from that residual; body(stream) queues one iteration (captured once as a
// graph, see iteration_graph).  The host starts the loop, launches the
// iteration graph in batches, and when the recursive residual meets the
// tolerance confirms it with the true residual (restarting from it when it
// disagrees); the relative true residual at exit goes to relres.
template <typename Res, typename Resume, typename Body>
int outer_loop(ldu_amg *M, int kind, double *x, double tol, int maxit, Res residual,
               Resume resume, Body body, int *iters, double *relres, cudaStream_t st) {
    AmgScalars *S = M->S, *H = M->S_host;
    std::memset(H, 0, sizeof(AmgScalars));
    H->tol2 = tol * tol;
    H->maxit = maxit;
    H->status = LDU_OK;
    cudaError_t e = cudaMemcpyAsync(S, H, sizeof(AmgScalars), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return cuda_status(e);
    int rc = residual(0);
    if (rc == LDU_OK)
        rc = resume();
    if (rc == LDU_OK)
        rc = read_scalars(M, st);
    if (rc != LDU_OK)
        return rc;
    int status = LDU_NOT_CONVERGED, it = 0;
    bool confirmed = false;   // H->rr holds the true residual of the final x
    const double bn2 = H->bn2, thr2 = H->thr2;
    if (bn2 == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * (size_t)M->n, st);
        status = LDU_OK;
    } else if (H->rr <= thr2) {
        status = LDU_OK;
        confirmed = true;
    } else if (maxit > 0) {
        cudaGraphExec_t step = nullptr;
        if ((rc = iteration_graph(M, kind, x, body, &step)) != LDU_OK)
            return rc;
        // iterations in batches between host reads, sized from the observed
        // convergence rate so that few kernels run past the stopping point
        double rr_prev = H->rr;
        int it_prev = 0, batch = 4;
        for (;;) {
            for (int g = 0; g < batch; ++g) {
                const cudaError_t eg = cudaGraphLaunch(step, st);
                if (eg != cudaSuccess)
                    return cuda_status(eg);
            }
            if ((rc = read_scalars(M, st)) != LDU_OK)
                return rc;
            it = H->it;
            if (H->status == LDU_ERR_NOT_SPD) {
                status = LDU_ERR_NOT_SPD;
                break;
            }
            if (H->conv) {
                // confirm with the true residual; restart the search if it disagrees
                if ((rc = residual(1)) != LDU_OK || (rc = read_scalars(M, st)) != LDU_OK)
                    return rc;
                if (H->rr <= thr2) {
                    status = LDU_OK;
                    confirmed = true;
                    break;
                }
                if (it >= maxit)
                    break;
                if ((rc = resume()) != LDU_OK)
                    return rc;
                continue;
            }
            if (H->status == LDU_NOT_CONVERGED)
                break;
            // remaining iterations from the mean contraction of ||r||^2
            const double rho = std::pow(H->rr / rr_prev, 1.0 / std::max(1, it - it_prev));
            double left = 8.0;
            if (rho > 0.0 && rho < 1.0)
                left = std::min(8.0, std::log(thr2 / H->rr) / std::log(rho));
            batch = std::min(maxit - it, std::max(1, (int)std::lround(left)));
            rr_prev = H->rr;
            it_prev = it;
        }
    }
    // the true residual at exit
    double tr = 0.0;
    if (bn2 > 0.0) {
        if (!confirmed && ((rc = residual(1)) != LDU_OK || (rc = read_scalars(M, st)) != LDU_OK))
            return rc;
        tr = std::sqrt(H->rr / bn2);
    }
    if (iters)
        *iters = it;
    if (relres)
        *relres = tr;
    return status;
}

// AMG-PCG with the cycle in precision T (double: Saad Alg. 9.1 with z = V(r);
// float: the same with the Polak-Ribiere beta)
template <typename T>
int pcg_loop(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
             double *relres, cudaStream_t st) {
    const bool f32 = std::is_same<T, float>::value;
    const DSell<double> A = M->fine();
    const double *d = M->fine_d();
    const int64_t n = M->n;
    const int ga = grid_rows(n);
    const T *wd0 = M->lev.empty() ? nullptr : M->lev[0].v<T>().wd;   // cycle input t0 = (w/d) r
    T *t0 = M->lev.empty() ? nullptr : M->lev[0].v<T>().t;
    T *bv = f32 ? (T *)M->r32 : nullptr;                  // float cycle: its own copy of r
    const T *cyc_b = f32 ? (const T *)M->r32 : (const T *)M->r;
    T *cyc_z = f32 ? (T *)M->z32 : (T *)M->z;
    AmgScalars *S = M->S;
    auto residual = [&](int mode) {
        k_amg_residual<T><<<ga, kThreads, 0, st>>>(A, d, b, x, M->r, wd0, t0, bv, mode, S,
                                                   M->part, M->count);
        return cuda_status(cudaGetLastError());
    };
    // z = V(r) with (r, z); the next direction is z itself
    auto resume = [&]() { return vcycle<T>(M, 0, cyc_b, cyc_z, true, nullptr, st); };
    auto body = [&](cudaStream_t cs) {
        k_amg_p<T><<<ga, kThreads, 0, cs>>>((int)n, (const T *)cyc_z, M->p, S);
        k_amg_q<<<ga, kThreads, 0, cs>>>(A, d, M->p, M->q, S, M->part, M->count);
        k_amg_xr<T><<<ga, kThreads, 0, cs>>>((int)n, M->p, M->q, x, M->r, wd0, t0, bv, S, M->part,
                                             M->count);
        return vcycle<T>(M, 0, cyc_b, cyc_z, true, &S->done, cs);
    };
    return outer_loop(M, f32 ? 0 : 1, x, tol, maxit, residual, resume, body, iters, relres, st);
}

// pipelined PCG with the FP64 cycle (Table 2's AMG-PipeCG): per step one
// cycle m = V(w), one product n = A m and one update pass that also forms
// the step's three dot products
int pipe_loop(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
              double *relres, cudaStream_t st) {
    const DSell<double> A = M->fine();
    const double *d = M->fine_d();
    const int64_t n = M->n;
    const int ga = grid_rows(n);
    for (double *&v : M->pv)
        if (!v) {
            cudaError_t e = alloc(&v, n, &M->device_bytes);
            if (e != cudaSuccess)
                return cuda_status(e);
        }
    double *u = M->pv[0], *w = M->pv[1], *m = M->pv[2], *nv = M->pv[3];
    const PipeVecs V{m, nv, M->pv[4], M->pv[5], M->pv[6], M->p, x, M->r, u, w};
    const double *wd0 = M->lev.empty() ? nullptr : M->lev[0].v64.wd;
    double *t0 = M->lev.empty() ? nullptr : M->lev[0].v64.t;
    AmgScalars *S = M->S;
    auto residual = [&](int mode) {
        k_amg_residual<double><<<ga, kThreads, 0, st>>>(A, d, b, x, M->r, wd0, t0, nullptr, mode,
                                                        S, M->part, M->count);
        return cuda_status(cudaGetLastError());
    };
    // u = V(r), w = A u with gamma and delta; the recurrences restart
    auto resume = [&]() {
        const int r2 = vcycle<double>(M, 0, M->r, u, false, nullptr, st);
        if (r2 != LDU_OK)
            return r2;
        k_pp_init<<<ga, kThreads, 0, st>>>(A, d, u, M->r, w, wd0, t0, S, M->part, M->count);
        return cuda_status(cudaGetLastError());
    };
    auto body = [&](cudaStream_t cs) {
        const int r2 = vcycle<double>(M, 0, w, m, false, &S->done, cs);
        if (r2 != LDU_OK)
            return r2;
        k_pp_spmv<<<ga, kThreads, 0, cs>>>(A, d, m, nv, S);
        k_pp_update<<<std::min(ga, 152 * kUpdateBlocksPerSm), kThreads, 0, cs>>>(
            (int)n, V, wd0, t0, S, M->part, M->count);
        return cuda_status(cudaGetLastError());
    };
    return outer_loop(M, 2, x, tol, maxit, residual, resume, body, iters, relres, st);
}

// ---- the hierarchy on the device (kernels in amg_setup.cuh) ---------------

// a level's matrix during construction: CSR, the diagonal in every row,
// columns sorted (n x m; ptr has n + 1 entries)
struct GCsr {
    int64_t n = 0, m = 0, nnz = 0;
    int64_t *ptr = nullptr;
    int *col = nullptr;
    double *val = nullptr;
};

// stream-ordered scratch of the construction, released on every path
struct Scratch {
    cudaStream_t st;
    std::vector<void *> live;
    explicit Scratch(cudaStream_t s) : st(s) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    template <typename T>
    cudaError_t get(T **p, int64_t count) {
        *p = nullptr;
        const cudaError_t e =
            cudaMallocAsync((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1), st);
        if (e == cudaSuccess)
            live.push_back((void *)*p);
        return e;
    }
    void put(const void *p) {
        for (size_t k = 0; k < live.size(); ++k)
            if (live[k] == p) {
                cudaFreeAsync(live[k], st);
                live.erase(live.begin() + (long)k);
                return;
            }
    }
    void put(GCsr &A) {
        put(A.ptr);
        put(A.col);
        put(A.val);
        A = GCsr();
    }
    ~Scratch() {
        for (void *p : live)
            cudaFreeAsync(p, st);
    }
};

#define CKS(call)                           \
    do {                                    \
        const cudaError_t e_ = (call);      \
        if (e_ != cudaSuccess)              \
            return cuda_status(e_);         \
    } while (0)
#define LAUNCHED() CKS(cudaGetLastError())

// out = exclusive scan of in[0..n) (n + 1 entries); *total = out[n]
int exscan(Scratch &S, const int64_t *in, int64_t n, int64_t **out, int64_t *total) {
    int64_t *tmp;
    CKS(S.get(out, n + 1));
    CKS(S.get(&tmp, amgs::scan_tmp_items(n)));
    amgs::scan_excl(in, *out, n, tmp, S.st);
    LAUNCHED();
    CKS(cudaMemcpyAsync(total, *out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, S.st));
    CKS(cudaStreamSynchronize(S.st));
    S.put(tmp);
    return LDU_OK;
}

int read_int(Scratch &S, const int *dev, int *host) {
    CKS(cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, S.st));
    CKS(cudaStreamSynchronize(S.st));
    return LDU_OK;
}

// both triangles of an LDU matrix with the diagonal; entries of one column
// (duplicate faces) added in face order
int ldu_to_csr(Scratch &S, int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
               const double *diag, const double *up, const double *lo, GCsr &A) {
    using namespace amgs;
    int64_t *len, *xptr, *xkey, *cur, xnnz = 0;
    int *xcol;
    double *xval;
    CKS(S.get(&len, n));
    k_ones<<<blocks(n), kT, 0, S.st>>>(n, len);
    if (nf > 0)
        k_ldu_len<<<blocks(nf), kT, 0, S.st>>>(nf, own, nbr, len);
    LAUNCHED();
    if (int rc = exscan(S, len, n, &xptr, &xnnz))
        return rc;
    CKS(S.get(&xcol, xnnz));
    CKS(S.get(&xval, xnnz));
    CKS(S.get(&xkey, xnnz));
    CKS(S.get(&cur, n));
    k_ldu_fill_diag<<<blocks(n), kT, 0, S.st>>>(n, xptr, diag, xcol, xval, xkey, cur);
    if (nf > 0)
        k_ldu_fill_faces<<<blocks(nf), kT, 0, S.st>>>(nf, own, nbr, up, lo, xcol, xval, xkey,
                                                       cur);
    k_row_sort_merge<<<blocks(n), kT, 0, S.st>>>(n, xptr, xcol, xval, xkey, len);
    LAUNCHED();
    A.n = A.m = n;
    if (int rc = exscan(S, len, n, &A.ptr, &A.nnz))
        return rc;
    CKS(S.get(&A.col, A.nnz));
    CKS(S.get(&A.val, A.nnz));
    k_pack<<<blocks(n), kT, 0, S.st>>>(n, xptr, xcol, xval, A.ptr, A.col, A.val);
    LAUNCHED();
    for (const void *p : {(const void *)len, (const void *)xptr, (const void *)xkey,
                          (const void *)cur, (const void *)xcol, (const void *)xval})
        S.put(p);
    return LDU_OK;
}

// the rows of n whose len is at least thr: *list (device, *count entries)
int long_rows(Scratch &S, const int64_t *len, int64_t n, int64_t thr, int **list, int64_t *count) {
    using namespace amgs;
    int64_t *flag, *rank;
    CKS(S.get(&flag, n));
    k_flag_long<<<blocks(n), kT, 0, S.st>>>(n, len, thr, flag);
    LAUNCHED();
    if (int rc = exscan(S, flag, n, &rank, count))
        return rc;
    CKS(S.get(list, *count));
    if (*count > 0)
        k_list_long<<<blocks(n), kT, 0, S.st>>>(n, flag, rank, *list);
    LAUNCHED();
    S.put(flag);
    S.put(rank);
    return LDU_OK;
}

__global__ void k_gather_i64(int64_t m, const int *list, const int64_t *a, int64_t *b) {
    const int64_t k = (int64_t)blockIdx.x * amgs::kT + threadIdx.x;
    if (k < m)
        b[k] = a[list[k]];
}

// Z = X Y on the structural pattern, each row's sums independent of the
// order of the threads that form them: a thread per row adding its products
// in expansion order, or, for rows of many products, a block per row with
// fixed-point integer sums
int spgemm(Scratch &S, const GCsr &X, const GCsr &Y, GCsr &Z) {
    using namespace amgs;
    const int n = (int)X.n;
    int64_t *ub, *ts, *tp, *cnt, tsize = 0;
    int *tcol;
    double *tval;
    CKS(S.get(&ub, n));
    CKS(S.get(&ts, n));
    k_gemm_bound<<<blocks(n), kT, 0, S.st>>>(n, X.ptr, X.col, Y.ptr, ub);
    k_gemm_tsize<<<blocks(n), kT, 0, S.st>>>(n, ub, Y.m, ts);
    LAUNCHED();
    if (int rc = exscan(S, ts, n, &tp, &tsize))
        return rc;
    CKS(S.get(&tcol, tsize));
    CKS(S.get(&tval, tsize));
    CKS(S.get(&cnt, n));
    k_gemm_rows<<<blocks(n), kT, 0, S.st>>>(n, X.ptr, X.col, X.val, Y.ptr, Y.col, Y.val, ub, tp,
                                            tcol, tval, cnt);
    LAUNCHED();
    {
        int *list;
        int64_t nlong = 0;
        if (int rc = long_rows(S, ub, n, kLongRow, &list, &nlong))
            return rc;
        if (nlong > 0) {
            int64_t *tsl, *lp, lsize = 0;
            long long *fix;
            CKS(S.get(&tsl, nlong));
            k_gather_i64<<<blocks(nlong), kT, 0, S.st>>>(nlong, list, ts, tsl);
            LAUNCHED();
            if (int rc = exscan(S, tsl, nlong, &lp, &lsize))
                return rc;
            CKS(S.get(&fix, 2 * lsize));
            k_gemm_long_rows<<<(unsigned)nlong, kT, kSortSmem, S.st>>>(
                list, X.ptr, X.col, X.val, Y.ptr, Y.col, Y.val, ub, tp, lp, tcol, tval, fix, cnt);
            LAUNCHED();
            S.put(tsl);
            S.put(lp);
            S.put(fix);
        }
        S.put(list);
    }
    Z.n = X.n;
    Z.m = Y.m;
    if (int rc = exscan(S, cnt, n, &Z.ptr, &Z.nnz))
        return rc;
    CKS(S.get(&Z.col, Z.nnz));
    CKS(S.get(&Z.val, Z.nnz));
    k_pack<<<blocks(n), kT, 0, S.st>>>(n, tp, tcol, tval, Z.ptr, Z.col, Z.val);
    LAUNCHED();
    for (const void *p : {(const void *)ub, (const void *)ts, (const void *)tp, (const void *)cnt,
                          (const void *)tcol, (const void *)tval})
        S.put(p);
    return LDU_OK;
}

// a kept copy (cudaMalloc, counted) of a device array
template <typename T>
int keep_copy(Scratch &S, T **dst, const T *src, int64_t count, int64_t *nb) {
    CKS(alloc(dst, count, nb));
    if (count > 0)
        CKS(cudaMemcpyAsync(*dst, src, sizeof(T) * (size_t)count, cudaMemcpyDeviceToDevice, S.st));
    return LDU_OK;
}

// a kept int32 copy of an int64 array (values checked to fit by the caller)
int keep_i32(Scratch &S, int **dst, const int64_t *src, int64_t count, int64_t *nb) {
    CKS(alloc(dst, count, nb));
    amgs::k_i64_to_i32<<<amgs::blocks(count), amgs::kT, 0, S.st>>>(count, src, *dst);
    LAUNCHED();
    return LDU_OK;
}

// kept double values and their float rounding
int keep_vals(Scratch &S, double **d64, float **d32, const double *src, int64_t count,
              int64_t *nb) {
    if (int rc = keep_copy(S, d64, src, count, nb))
        return rc;
    CKS(alloc(d32, count, nb));
    amgs::k_d2f<<<amgs::blocks(count), amgs::kT, 0, S.st>>>(count, *d64, *d32);
    LAUNCHED();
    return LDU_OK;
}

// A's off-diagonal part in 32-row sliced ELL, kept: slice offsets and widths,
// columns, double values (the float copy is left to the caller) and, when
// every column lies within 16 bits of its row, the offsets; *padded = slots.
// Returns UNSUPPORTED when the slots exceed int32 indexing.  With probe, only
// *padded is computed.
int sell32(Scratch &S, const GCsr &A, const int64_t *olen, bool probe, int64_t *padded,
           int **sp, int **sw, int **col, double **val, short **c16, int64_t *nb) {
    using namespace amgs;
    const int n = (int)A.n;
    const int64_t ns = (A.n + 31) / 32;
    int64_t *swd, *slots, *spd;
    CKS(S.get(&swd, ns));
    CKS(S.get(&slots, ns));
    k_slice32_width<<<blocks(ns), kT, 0, S.st>>>(n, olen, swd);
    k_slice32_slots<<<blocks(ns), kT, 0, S.st>>>((int)ns, swd, slots);
    LAUNCHED();
    if (int rc = exscan(S, slots, ns, &spd, padded))
        return rc;
    if (!probe) {
        if (*padded > INT32_MAX)
            return LDU_ERR_UNSUPPORTED;
        int *flags;
        CKS(S.get(&flags, 1));
        CKS(cudaMemsetAsync(flags, 0, sizeof(int), S.st));
        CKS(alloc(col, *padded, nb));
        CKS(alloc(val, *padded, nb));
        CKS(alloc(c16, *padded, nb));
        k_sell32_fill<<<blocks(ns * 32), kT, 0, S.st>>>(n, A.ptr, A.col, A.val, spd, swd, *col,
                                                        *val, *c16, flags);
        LAUNCHED();
        if (int rc = keep_i32(S, sp, spd, ns + 1, nb))
            return rc;
        if (int rc = keep_i32(S, sw, swd, ns, nb))
            return rc;
        int hf = 0;
        if (int rc = read_int(S, flags, &hf))
            return rc;
        if (hf & 4) {   // some column is beyond 16 bits of its row
            cudaFree(*c16);
            *nb -= (int64_t)sizeof(short) * std::max<int64_t>(*padded, 1);
            *c16 = nullptr;
        }
        S.put(flags);
    }
    S.put(swd);
    S.put(slots);
    S.put(spd);
    return LDU_OK;
}

// One level: its scalars, aggregates, P, R and device layouts (kept in L)
// and its Galerkin matrix Ac.  *stop = true when the aggregation would not
// shrink the level (nothing is kept then).
int build_level(Scratch &S, const GCsr &A, bool first, int lanes, amg_level &L, GCsr &Ac,
                bool *stop, int64_t *nb) {
    using namespace amgs;
    const int n = (int)A.n;
    *stop = false;
    // 1. d, rho, w
    double *d;
    unsigned long long *rho_bits;
    int *flags;
    CKS(S.get(&d, n));
    CKS(S.get(&rho_bits, 1));
    CKS(S.get(&flags, 1));
    CKS(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), S.st));
    CKS(cudaMemsetAsync(flags, 0, sizeof(int), S.st));
    k_diag_rho<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, A.val, d, rho_bits, flags);
    LAUNCHED();
    unsigned long long rb = 0;
    int hf = 0;
    CKS(cudaMemcpyAsync(&rb, rho_bits, sizeof(rb), cudaMemcpyDeviceToHost, S.st));
    if (int rc = read_int(S, flags, &hf))
        return rc;
    if (hf & 1)
        return LDU_ERR_NOT_SPD;
    double rho;
    std::memcpy(&rho, &rb, sizeof(rho));
    const double w = 4.0 / (3.0 * rho);
    // 2. distance-2 maximal independent set
    int *state, *s1, *s2;
    uint64_t *h, *h1, *h2;
    unsigned *left;
    CKS(S.get(&state, n));
    CKS(S.get(&s1, n));
    CKS(S.get(&s2, n));
    CKS(S.get(&h, n));
    CKS(S.get(&h1, n));
    CKS(S.get(&h2, n));
    CKS(S.get(&left, 1));
    k_mis_init<<<blocks(n), kT, 0, S.st>>>(n, state, h);
    for (int round = 0;; ++round) {
        if (round > n + 1)
            return LDU_ERR_UNSUPPORTED;   // every round decides at least one row
        CKS(cudaMemsetAsync(left, 0, sizeof(unsigned), S.st));
        k_pair_max<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, state, h, s1, h1);
        k_pair_max<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, s1, h1, s2, h2);
        k_mis_update<<<blocks(n), kT, 0, S.st>>>(n, state, h, s2, h2, left);
        LAUNCHED();
        unsigned hl = 0;
        CKS(cudaMemcpyAsync(&hl, left, sizeof(hl), cudaMemcpyDeviceToHost, S.st));
        CKS(cudaStreamSynchronize(S.st));
        if (hl == 0)
            break;
    }
    // 3. aggregates
    int64_t *flag, *rank, na = 0;
    CKS(S.get(&flag, n));
    k_root_flags<<<blocks(n), kT, 0, S.st>>>(n, state, flag);
    LAUNCHED();
    if (int rc = exscan(S, flag, n, &rank, &na))
        return rc;
    if (na >= n) {
        *stop = true;
        return LDU_OK;
    }
    int *firsta, *agg;
    CKS(S.get(&firsta, n));
    CKS(alloc(&agg, n, nb));
    L.agg = agg;
    k_agg_roots<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, state, rank, firsta);
    k_agg_rest<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, A.val, firsta, agg, kTie, flags);
    LAUNCHED();
    if (int rc = read_int(S, flags, &hf))
        return rc;
    if (hf & 2)
        return LDU_ERR_UNSUPPORTED;   // a row beyond two steps of every root: not a maximal set
    for (const void *p : {(const void *)state, (const void *)s1, (const void *)s2,
                          (const void *)h, (const void *)h1, (const void *)h2, (const void *)left,
                          (const void *)flag, (const void *)rank, (const void *)firsta})
        S.put(p);
    // 4. P = (I - w D^-1 A) P_t on the pattern of (I + A) P_t
    GCsr P;
    {
        int *xcol;
        double *xval;
        int64_t *xkey, *cnt;
        CKS(S.get(&xcol, A.nnz));
        CKS(S.get(&xval, A.nnz));
        CKS(S.get(&xkey, A.nnz));
        CKS(S.get(&cnt, n));
        k_p_expand<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, A.val, agg, xcol, xval, xkey);
        k_row_sort_merge<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, xcol, xval, xkey, cnt);
        k_p_values<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, cnt, xcol, xval, agg, d, w);
        LAUNCHED();
        P.n = n;
        P.m = na;
        if (int rc = exscan(S, cnt, n, &P.ptr, &P.nnz))
            return rc;
        CKS(S.get(&P.col, P.nnz));
        CKS(S.get(&P.val, P.nnz));
        k_pack<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, xcol, xval, P.ptr, P.col, P.val);
        LAUNCHED();
        for (const void *p : {(const void *)xcol, (const void *)xval, (const void *)xkey,
                              (const void *)cnt})
            S.put(p);
    }
    if (P.nnz > INT32_MAX)
        return LDU_ERR_UNSUPPORTED;
    // 5. R = P^T (rows in increasing order within each of its rows)
    GCsr R;
    {
        int64_t *rlen, *cur, *rkey;
        CKS(S.get(&rlen, na));
        CKS(cudaMemsetAsync(rlen, 0, sizeof(int64_t) * (size_t)na, S.st));
        k_col_count<<<blocks(P.nnz), kT, 0, S.st>>>(P.nnz, P.col, rlen);
        LAUNCHED();
        R.n = na;
        R.m = n;
        if (int rc = exscan(S, rlen, na, &R.ptr, &R.nnz))
            return rc;
        CKS(S.get(&cur, na));
        CKS(S.get(&R.col, R.nnz));
        CKS(S.get(&R.val, R.nnz));
        CKS(S.get(&rkey, R.nnz));
        k_copy_i64<<<blocks(na), kT, 0, S.st>>>(na, R.ptr, cur);
        k_transpose_fill<<<blocks(n), kT, 0, S.st>>>(n, P.ptr, P.col, P.val, cur, R.col, R.val,
                                                      rkey);
        // short rows by a thread each, long ones by a block each (the rows
        // of a transpose hold distinct columns: sorting is all they need)
        k_row_sort_merge<<<blocks(na), kT, 0, S.st>>>(na, R.ptr, R.col, R.val, rkey, rlen,
                                                      kLongSort - 1);
        LAUNCHED();
        {
            int *list;
            int64_t nlong = 0;
            if (int rc = long_rows(S, rlen, na, kLongSort, &list, &nlong))
                return rc;
            if (nlong > 0)
                k_sort_long_rows<<<(unsigned)nlong, kT, kSortSmem, S.st>>>(list, R.ptr, R.col,
                                                                           R.val);
            LAUNCHED();
            S.put(list);
        }
        for (const void *p : {(const void *)rlen, (const void *)cur, (const void *)rkey})
            S.put(p);
    }
    // 6. Ac = R (A P)
    {
        GCsr AP;
        if (int rc = spgemm(S, A, P, AP))
            return rc;
        if (int rc = spgemm(S, R, AP, Ac))
            return rc;
        S.put(AP);
    }
    // 7. the level's device layouts
    L.n = A.n;
    L.nnz = A.nnz;
    L.w = w;
    int64_t *olen;
    CKS(S.get(&olen, n));
    k_offdiag_len<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, olen);
    LAUNCHED();
    const int64_t off_nnz = A.nnz - A.n;
    int64_t padded = 0;
    if (int rc = sell32(S, A, olen, true, &padded, nullptr, nullptr, nullptr, nullptr, nullptr, nb))
        return rc;
    L.a_sell = first || (double)padded <= kSellPad * (double)off_nnz;
    if (L.a_sell) {
        if (int rc = sell32(S, A, olen, false, &padded, &L.a_sp, &L.a_sw, &L.a_col, &L.v64.a_val,
                            &L.a_c16, nb))
            return rc;
        CKS(alloc(&L.v32.a_val, padded, nb));
        k_d2f<<<blocks(padded), kT, 0, S.st>>>(padded, L.v64.a_val, L.v32.a_val);
        LAUNCHED();
    } else {
        int64_t *optr, ototal = 0;
        if (int rc = exscan(S, olen, n, &optr, &ototal))
            return rc;
        if (ototal > INT32_MAX)
            return LDU_ERR_UNSUPPORTED;
        CKS(alloc(&L.a_col, ototal, nb));
        CKS(alloc(&L.v64.a_val, ototal, nb));
        k_offdiag_csr<<<blocks(n), kT, 0, S.st>>>(n, A.ptr, A.col, A.val, optr, L.a_col,
                                                   L.v64.a_val);
        LAUNCHED();
        if (int rc = keep_i32(S, &L.a_ptr, optr, n + 1, nb))
            return rc;
        CKS(alloc(&L.v32.a_val, ototal, nb));
        k_d2f<<<blocks(ototal), kT, 0, S.st>>>(ototal, L.v64.a_val, L.v32.a_val);
        LAUNCHED();
        L.a_lpr = lanes ? lanes : lpr_for(A.n, ototal);
        S.put(optr);
    }
    S.put(olen);
    {
        double *wd;
        CKS(S.get(&wd, n));
        k_wd<<<blocks(n), kT, 0, S.st>>>(n, d, w, wd);
        LAUNCHED();
        if (int rc = keep_vals(S, &L.v64.d, &L.v32.d, d, n, nb))
            return rc;
        if (int rc = keep_vals(S, &L.v64.wd, &L.v32.wd, wd, n, nb))
            return rc;
        S.put(wd);
    }
    if (int rc = keep_i32(S, &L.p_ptr, P.ptr, P.n + 1, nb))
        return rc;
    if (int rc = keep_copy(S, &L.p_col, P.col, P.nnz, nb))
        return rc;
    if (int rc = keep_vals(S, &L.v64.p_val, &L.v32.p_val, P.val, P.nnz, nb))
        return rc;
    if (int rc = keep_i32(S, &L.r_ptr, R.ptr, R.n + 1, nb))
        return rc;
    if (int rc = keep_copy(S, &L.r_col, R.col, R.nnz, nb))
        return rc;
    if (int rc = keep_vals(S, &L.v64.r_val, &L.v32.r_val, R.val, R.nnz, nb))
        return rc;
    L.p_lpr = lpr_for(P.n, P.nnz);
    L.r_lpr = lanes ? lanes : lpr_for(R.n, R.nnz);
    L.r_rows = R.n;
    S.put(P);
    S.put(R);
    S.put(d);
    S.put(rho_bits);
    S.put(flags);
    return LDU_OK;
}

// a device CSR copied to the host (for the coarsest level's dense inverse)
int to_host(Scratch &S, const GCsr &A, HCsr &H) {
    H.n = A.n;
    H.m = A.m;
    H.ptr.resize((size_t)A.n + 1);
    H.col.resize((size_t)A.nnz);
    H.val.resize((size_t)A.nnz);
    CKS(cudaMemcpyAsync(H.ptr.data(), A.ptr, sizeof(int64_t) * H.ptr.size(),
                        cudaMemcpyDeviceToHost, S.st));
    if (A.nnz > 0) {
        CKS(cudaMemcpyAsync(H.col.data(), A.col, sizeof(int) * H.col.size(),
                            cudaMemcpyDeviceToHost, S.st));
        CKS(cudaMemcpyAsync(H.val.data(), A.val, sizeof(double) * H.val.size(),
                            cudaMemcpyDeviceToHost, S.st));
    }
    CKS(cudaStreamSynchronize(S.st));
    return LDU_OK;
}

#undef LAUNCHED
#undef CKS

}  // namespace

extern "C" {

int ldu_amg_create(int64_t n, int64_t nf, const int32_t *owner, const int32_t *neighbour,
                   const double *diag, const double *upper, const double *lower,
                   const amg_opts *aopt, ldu_stream_t stream, ldu_amg **out) {
    if (!out)
        return LDU_ERR_BAD_ARG;
    *out = nullptr;
    if (n <= 0 || nf < 0 || !diag || (nf > 0 && (!owner || !neighbour || !upper || !lower)))
        return LDU_ERR_BAD_ARG;
    int max_coarse = 500, max_levels = 12, lanes = 0;
    if (aopt) {
        if (aopt->max_coarse)
            max_coarse = aopt->max_coarse;
        if (aopt->max_levels)
            max_levels = aopt->max_levels;
        lanes = aopt->lanes_per_row;
    }
    if (max_coarse < 1 || max_coarse > kMaxCoarse || max_levels < 1 || max_levels > 64 ||
        lanes < 0 || lanes > 32 || (lanes & (lanes - 1)) != 0)
        return LDU_ERR_BAD_ARG;
    if (n > INT32_MAX / 2 || nf > INT32_MAX / 2)
        return LDU_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    ldu_amg *M = new ldu_amg();
    int rc = LDU_OK;
    {
        Scratch S(st);
#define CKA(call)                              \
    do {                                       \
        const cudaError_t e_ = (call);         \
        if (e_ != cudaSuccess) {               \
            rc = cuda_status(e_);              \
            goto done;                         \
        }                                      \
    } while (0)
#define RCA(call)                              \
    do {                                       \
        rc = (call);                           \
        if (rc != LDU_OK)                      \
            goto done;                         \
    } while (0)
        int64_t *nb = &M->device_bytes;
        GCsr A;
        std::vector<double> inv;
        HCsr C;
        CKA(cudaGetDevice(&M->device));
        M->n = n;
        {
            // validation on the device, as ldu_create does
            int *deg, *flags;
            CKA(S.get(&deg, n));
            CKA(S.get(&flags, 4));
            CKA(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)n, st));
            CKA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
            if (nf > 0)
                k_validate_count<<<amgs::blocks(nf), 256, 0, st>>>(nf, (int)n, owner, neighbour,
                                                                    deg, flags);
            k_validate_values<<<amgs::blocks(std::max(n, nf)), 256, 0, st>>>(n, nf, diag, upper,
                                                                              lower, flags);
            CKA(cudaGetLastError());
            int hf = 0;
            RCA(read_int(S, flags, &hf));
            if (hf & (kFlagBadIndex | kFlagBadOrder)) {
                rc = LDU_ERR_BAD_ADDRESSING;
                goto done;
            }
            if (hf & (kFlagBadDiag | kFlagNonFinite)) {
                rc = LDU_ERR_NOT_SPD;
                goto done;
            }
            S.put(deg);
            S.put(flags);
        }
        RCA(ldu_to_csr(S, n, nf, owner, neighbour, diag, upper, lower, A));
        // coarsen while the level is above max_coarse rows and aggregation shrinks it
        while (A.n > max_coarse && (int)M->lev.size() < max_levels) {
            M->lev.emplace_back();
            GCsr Ac;
            bool stop = false;
            RCA(build_level(S, A, M->lev.size() == 1, lanes, M->lev.back(), Ac, &stop, nb));
            if (stop) {
                M->lev.pop_back();
                break;
            }
            amg_level &L = M->lev.back();
            CKA(alloc(&L.v64.t, L.n, nb));
            CKA(alloc(&L.v64.r, L.n, nb));
            CKA(alloc(&L.v32.t, L.n, nb));
            CKA(alloc(&L.v32.r, L.n, nb));
            if (M->lev.size() > 1) {
                CKA(alloc(&L.v64.x, L.n, nb));
                CKA(alloc(&L.v64.b, L.n, nb));
                CKA(alloc(&L.v32.x, L.n, nb));
                CKA(alloc(&L.v32.b, L.n, nb));
            }
            S.put(A);
            A = Ac;
        }
        if (M->lev.empty()) {
            // the fine matrix is the coarsest: keep its SpMV form for the outer loop
            int64_t *olen, padded = 0;
            short *c16 = nullptr;
            CKA(S.get(&olen, A.n));
            amgs::k_offdiag_len<<<amgs::blocks(A.n), amgs::kT, 0, st>>>((int)A.n, A.ptr, A.col,
                                                                         olen);
            CKA(cudaGetLastError());
            RCA(sell32(S, A, olen, false, &padded, &M->f_sp, &M->f_sw, &M->f_col, &M->f_val,
                       &c16, nb));
            if (c16) {
                cudaFree(c16);
                *nb -= (int64_t)sizeof(short) * std::max<int64_t>(padded, 1);
            }
            unsigned long long *rho_bits;
            int *flags;
            CKA(S.get(&rho_bits, 1));
            CKA(S.get(&flags, 1));
            CKA(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), st));
            CKA(cudaMemsetAsync(flags, 0, sizeof(int), st));
            CKA(alloc(&M->f_d, A.n, nb));
            amgs::k_diag_rho<<<amgs::blocks(A.n), amgs::kT, 0, st>>>((int)A.n, A.ptr, A.col, A.val,
                                                                      M->f_d, rho_bits, flags);
            CKA(cudaGetLastError());
            S.put(olen);
        }
        // the coarsest level, applied through its dense inverse
        if (A.n > kMaxCoarse) {
            rc = LDU_ERR_UNSUPPORTED;   // coarsening stopped above what a dense inverse allows
            goto done;
        }
        M->nc = A.n;
        M->c_nnz = A.nnz;
        RCA(to_host(S, A, C));
        if (!dense_inverse(C, inv)) {
            rc = LDU_ERR_NOT_SPD;
            goto done;
        }
        CKA(upload2(&M->c64.inv, &M->c32.inv, inv, nb));
        CKA(alloc(&M->c64.x, A.n, nb));
        CKA(alloc(&M->c64.b, A.n, nb));
        CKA(alloc(&M->c32.x, A.n, nb));
        CKA(alloc(&M->c32.b, A.n, nb));
        CKA(alloc(&M->r, n, nb));
        CKA(alloc(&M->z, n, nb));
        CKA(alloc(&M->p, n, nb));
        CKA(alloc(&M->q, n, nb));
        CKA(alloc(&M->r32, n, nb));
        CKA(alloc(&M->z32, n, nb));
        CKA(alloc(&M->part, 3 * kMaxBlocks, nb));
        CKA(alloc(&M->count, 1, nb));
        CKA(cudaMemset(M->count, 0, sizeof(unsigned)));
        CKA(alloc(&M->S, 1, nb));
        CKA(cudaMallocHost((void **)&M->S_host, sizeof(AmgScalars)));
        CKA(cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking));
#undef CKA
#undef RCA
    done:;
    }   // the scratch is released here (stream-ordered)
    if (rc == LDU_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            rc = cuda_status(e);
    }
    if (rc != LDU_OK) {
        cudaStreamSynchronize(st);
        free_amg(M);
        return rc;
    }
    *out = M;
    return LDU_OK;
}

void ldu_amg_destroy(ldu_amg *M) {
    if (!M)
        return;
    cudaDeviceSynchronize();
    free_amg(M);
}

int ldu_amg_info(const ldu_amg *M, int *levels, int64_t *rows, int64_t *nnz, int max_levels) {
    if (!M || !levels || max_levels < 0)
        return LDU_ERR_BAD_ARG;
    const int count = (int)M->lev.size();   // levels with a prolongator, then the coarsest
    *levels = count + 1;
    for (int l = 0; l <= count && l < max_levels; ++l) {
        if (rows)
            rows[l] = l < count ? M->lev[(size_t)l].n : M->nc;
        if (nnz)
            nnz[l] = l < count ? M->lev[(size_t)l].nnz : M->c_nnz;
    }
    return LDU_OK;
}

int ldu_amg_aggregates(const ldu_amg *M, int level, int32_t *agg) {
    if (!M || !agg || level < 0 || level >= (int)M->lev.size())
        return LDU_ERR_BAD_ARG;
    const amg_level &L = M->lev[(size_t)level];
    const cudaError_t e =
        cudaMemcpy(agg, L.agg, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int ldu_amg_vcycle(ldu_amg *M, int precision, const void *b, void *x, ldu_stream_t stream) {
    if (!M || !b || !x || b == x || (precision != LDU_FP64 && precision != LDU_FP32))
        return LDU_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int g = grid_rows(M->n);
    if (precision == LDU_FP64) {
        if (!M->lev.empty())
            k_amg_scale<double><<<g, kThreads, 0, st>>>((int)M->n, M->lev[0].v64.wd,
                                                        (const double *)b, M->lev[0].v64.t);
        return vcycle<double>(M, 0, (const double *)b, (double *)x, false, nullptr, st);
    }
    if (!M->lev.empty())
        k_amg_scale<float><<<g, kThreads, 0, st>>>((int)M->n, M->lev[0].v32.wd, (const float *)b,
                                                   M->lev[0].v32.t);
    return vcycle<float>(M, 0, (const float *)b, (float *)x, false, nullptr, st);
}

int amg_pcg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int precision,
                  int *iters, double *relres, ldu_stream_t stream) {
    if (!M || !b || !x || b == x || maxit < 0 || !(tol >= 0.0) ||
        (precision != LDU_FP64 && precision != LDU_MIXED))
        return LDU_ERR_BAD_ARG;
    if (precision == LDU_FP64)
        return pcg_loop<double>(M, b, x, tol, maxit, iters, relres, (cudaStream_t)stream);
    return pcg_loop<float>(M, b, x, tol, maxit, iters, relres, (cudaStream_t)stream);
}

int amg_pipecg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
                     double *relres, ldu_stream_t stream) {
    if (!M || !b || !x || b == x || maxit < 0 || !(tol >= 0.0))
        return LDU_ERR_BAD_ARG;
    return pipe_loop(M, b, x, tol, maxit, iters, relres, (cudaStream_t)stream);
}

}  // extern "C"
