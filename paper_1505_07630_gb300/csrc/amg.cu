// amg.cu -- aggregation-AMG preconditioned CG (Sec. 5; Table 2's AMG-CG).
//
// The paper preconditions its CG with a V-cycle of an aggregation-based AMG
// (aggregates around a distance-2 maximal independent set, weighted-Jacobi
// smoother with omega = 4/3).  The reading implemented here:
//   aggregation   rows in increasing order; phase 1: a row whose neighbours
//                 are all free becomes a root and takes them (roots form a
//                 greedy distance-2 independent set); phase 2: every free row
//                 joins the phase-1 aggregate of its strongest neighbour
//                 (largest |a_ij|, strengths within a relative 1e-12 tie and
//                 go to the lower aggregate); phase 3: isolated rows alone;
//   prolongator   P = (I - w D^-1 A) P_t, w = 4 / (3 rho), rho the Gershgorin
//                 bound of D^-1 A (max_i sum_j |a_ij| / a_ii);
//   coarse        A_c = P^T A P until a level has at most max_coarse rows,
//                 whose dense inverse is applied;
//   cycle         V(1,1) with the same weighted Jacobi, from zero;
//   outer         PCG (Saad Alg. 9.1) with z = V(r), stopping on the
//                 recursive ||r|| and confirming with the true residual.
// The hierarchy is built on the host (it runs once per matrix); every step of
// a solve runs in the kernels below, the scalars of the outer PCG staying on
// the device, so that the host only reads them between batches of iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ldupcg_impl.cuh"

using namespace ldu;

namespace {

constexpr double kTie = 1e-12;
constexpr int kMaxCoarse = 4096;   // largest coarsest level (dense inverse: 128 MiB)

// ---- host sparse matrices ----------------------------------------------------

struct HCsr {
    int64_t n = 0, m = 0;           // rows, columns
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;       // sorted within each row
    std::vector<double> val;
};

// both triangles of an LDU matrix, rows sorted, duplicate entries summed
HCsr csr_from_ldu(int64_t n, int64_t nf, const int32_t *own, const int32_t *nbr,
                  const double *diag, const double *up, const double *lo) {
    std::vector<std::vector<std::pair<int32_t, double>>> rows((size_t)n);
    for (int64_t i = 0; i < n; ++i)
        rows[(size_t)i].push_back({(int32_t)i, diag[i]});
    for (int64_t f = 0; f < nf; ++f) {
        rows[(size_t)own[f]].push_back({nbr[f], up[f]});
        rows[(size_t)nbr[f]].push_back({own[f], lo[f]});
    }
    HCsr A;
    A.n = A.m = n;
    A.ptr.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        auto &r = rows[(size_t)i];
        std::sort(r.begin(), r.end(),
                  [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                      return a.first < b.first;
                  });
        for (size_t k = 0; k < r.size(); ++k) {
            if (k > 0 && r[k].first == A.col.back()) {
                A.val.back() += r[k].second;
                continue;
            }
            A.col.push_back(r[k].first);
            A.val.push_back(r[k].second);
        }
        A.ptr[(size_t)i + 1] = (int64_t)A.col.size();
        std::vector<std::pair<int32_t, double>>().swap(r);
    }
    return A;
}

double diag_of(const HCsr &A, int64_t i) {
    for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k)
        if (A.col[(size_t)k] == i)
            return A.val[(size_t)k];
    return 0.0;
}

// phases 1-3 of the aggregation; returns the number of aggregates
int64_t aggregate(const HCsr &A, std::vector<int32_t> &agg) {
    const int64_t n = A.n;
    agg.assign((size_t)n, -1);
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {   // phase 1
        if (agg[(size_t)i] >= 0)
            continue;
        bool any = false, free_all = true;
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k) {
            const int32_t j = A.col[(size_t)k];
            if (j == i)
                continue;
            any = true;
            if (agg[(size_t)j] >= 0) {
                free_all = false;
                break;
            }
        }
        if (!any || !free_all)
            continue;
        agg[(size_t)i] = (int32_t)na;
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k)
            agg[(size_t)A.col[(size_t)k]] = (int32_t)na;
        ++na;
    }
    const std::vector<int32_t> phase1 = agg;
    for (int64_t i = 0; i < n; ++i) {   // phase 2
        if (phase1[(size_t)i] >= 0)
            continue;
        int32_t best = -1;
        double best_v = -1.0;
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k) {
            const int32_t j = A.col[(size_t)k];
            if (j == i || phase1[(size_t)j] < 0)
                continue;
            const double a = std::fabs(A.val[(size_t)k]);
            if (best < 0 || a > best_v * (1.0 + kTie)) {
                best = phase1[(size_t)j];
                best_v = a;
            } else if (a >= best_v * (1.0 - kTie) && phase1[(size_t)j] < best) {
                best = phase1[(size_t)j];
                best_v = std::max(a, best_v);
            }
        }
        agg[(size_t)i] = best;
    }
    for (int64_t i = 0; i < n; ++i)     // phase 3
        if (agg[(size_t)i] < 0)
            agg[(size_t)i] = (int32_t)na++;
    return na;
}

// w = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii
double jacobi_weight(const HCsr &A) {
    double rho = 0.0;
    for (int64_t i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k)
            s += std::fabs(A.val[(size_t)k]);
        rho = std::max(rho, s / diag_of(A, i));
    }
    return 4.0 / (3.0 * rho);
}

// P = (I - w D^-1 A) P_t: row i holds, for every aggregate J touched by row
// i of A, [J == agg(i)] - w (1/a_ii) sum_{j in J} a_ij; exact zeros dropped
HCsr prolongator(const HCsr &A, const std::vector<int32_t> &agg, int64_t na, double w) {
    HCsr P;
    P.n = A.n;
    P.m = na;
    P.ptr.assign((size_t)A.n + 1, 0);
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < A.n; ++i) {
        row.clear();
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k) {
            const int32_t J = agg[(size_t)A.col[(size_t)k]];
            auto it = std::find_if(row.begin(), row.end(),
                                   [J](const std::pair<int32_t, double> &e) { return e.first == J; });
            if (it == row.end())
                row.push_back({J, A.val[(size_t)k]});
            else
                it->second += A.val[(size_t)k];
        }
        const double inv_d = 1.0 / diag_of(A, i);
        const int32_t own_agg = agg[(size_t)i];
        bool has_own = false;
        for (auto &e : row) {
            const double t = w * (inv_d * e.second);
            e.second = (e.first == own_agg ? 1.0 : 0.0) - t;
            has_own |= e.first == own_agg;
        }
        if (!has_own)
            row.push_back({own_agg, 1.0});
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                      return a.first < b.first;
                  });
        for (auto &e : row)
            if (e.second != 0.0) {
                P.col.push_back(e.first);
                P.val.push_back(e.second);
            }
        P.ptr[(size_t)i + 1] = (int64_t)P.col.size();
    }
    return P;
}

HCsr transpose(const HCsr &P) {
    HCsr R;
    R.n = P.m;
    R.m = P.n;
    R.ptr.assign((size_t)R.n + 1, 0);
    for (int32_t c : P.col)
        ++R.ptr[(size_t)c + 1];
    for (int64_t I = 0; I < R.n; ++I)
        R.ptr[(size_t)I + 1] += R.ptr[(size_t)I];
    R.col.resize(P.col.size());
    R.val.resize(P.val.size());
    std::vector<int64_t> at(R.ptr.begin(), R.ptr.end() - 1);
    for (int64_t i = 0; i < P.n; ++i)   // rows in increasing order: columns of R sorted
        for (int64_t k = P.ptr[(size_t)i]; k < P.ptr[(size_t)i + 1]; ++k) {
            const int64_t dst = at[(size_t)P.col[(size_t)k]]++;
            R.col[(size_t)dst] = (int32_t)i;
            R.val[(size_t)dst] = P.val[(size_t)k];
        }
    return R;
}

// A_c = R A P with R = P^T, one coarse row at a time through a dense
// accumulator; exact zeros dropped
HCsr galerkin(const HCsr &A, const HCsr &P, const HCsr &R) {
    HCsr Ac;
    Ac.n = Ac.m = P.m;
    Ac.ptr.assign((size_t)Ac.n + 1, 0);
    std::vector<double> acc((size_t)Ac.n, 0.0);
    std::vector<char> used((size_t)Ac.n, 0);
    std::vector<int32_t> touched;
    for (int64_t I = 0; I < Ac.n; ++I) {
        touched.clear();
        for (int64_t a = R.ptr[(size_t)I]; a < R.ptr[(size_t)I + 1]; ++a) {
            const int32_t i = R.col[(size_t)a];
            const double r = R.val[(size_t)a];
            for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k) {
                const int32_t j = A.col[(size_t)k];
                const double ra = r * A.val[(size_t)k];
                for (int64_t q = P.ptr[(size_t)j]; q < P.ptr[(size_t)j + 1]; ++q) {
                    const int32_t J = P.col[(size_t)q];
                    if (!used[(size_t)J]) {
                        used[(size_t)J] = 1;
                        touched.push_back(J);
                    }
                    acc[(size_t)J] += ra * P.val[(size_t)q];
                }
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int32_t J : touched) {
            if (acc[(size_t)J] != 0.0) {
                Ac.col.push_back(J);
                Ac.val.push_back(acc[(size_t)J]);
            }
            acc[(size_t)J] = 0.0;
            used[(size_t)J] = 0;
        }
        Ac.ptr[(size_t)I + 1] = (int64_t)Ac.col.size();
    }
    return Ac;
}

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
// Every level keeps A's off-diagonal part in sliced ELL with 32-row slices
// (one warp per slice, one thread per row, slot k of row s*32+i at
// sp[s] + 32k + i; padding slots hold column 0 and value 0), its diagonal d
// and w/d; P as CSR read one thread per row (3-5 entries a row); R = P^T as
// CSR read one warp per row (tens to hundreds of entries a row).

struct DSell {
    int n;
    const int *sp, *sw, *col;
    const double *val;
};

struct DCsr {
    int n;
    const int *ptr, *col;
    const double *val;
};

// scalars of the outer PCG, resident on the device between kernels
struct AmgScalars {
    double tol2, bn2, thr2, rr, rz, pq, alpha, beta;
    int it, maxit;
    int done;      // 1: the remaining kernels of the iteration return at once
    int conv;      // 1: the recursive residual met the tolerance
    int status;    // LDU_OK, LDU_NOT_CONVERGED or LDU_ERR_NOT_SPD
    int restart;   // 1: the next search direction is z itself
};

constexpr int kWarps = 8;                 // warps (slices) per block
constexpr int kThreads = kWarps * 32;
constexpr int kMaxBlocks = 152 * 8;       // grid cap: 8 resident blocks on each of 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
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
// only (r, z) when the search restarts
__device__ __forceinline__ void set_rz(AmgScalars *S, double rz) {
    if (S->restart) {
        S->rz = rz;
    } else {
        S->beta = rz / S->rz;
        S->rz = rz;
    }
}

// sum over the off-diagonal slots of row `row` (slice s, lane i) of a_ij f(j)
template <typename F>
__device__ __forceinline__ double sell_row(const DSell &A, int s, int i, F f) {
    const int w = A.sw[s];
    const int base = A.sp[s] + i;
    double acc = 0.0;
    int k = 0;
    for (; k + 2 <= w; k += 2) {
        const int c0 = __ldg(A.col + base + k * 32), c1 = __ldg(A.col + base + (k + 1) * 32);
        const double v0 = __ldcs(A.val + base + k * 32), v1 = __ldcs(A.val + base + (k + 1) * 32);
        const double f0 = f(c0), f1 = f(c1);
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

// pre-smoothing from zero and the residual, in one pass:
//   t = (w/d) b;  r = b - A t, with t_j formed from b_j on the fly
__global__ void __launch_bounds__(kThreads) k_amg_pre(DSell A, const double *__restrict__ d,
                                                      const double *__restrict__ wd,
                                                      const double *__restrict__ b,
                                                      double *__restrict__ t,
                                                      double *__restrict__ r, const int *skip) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const bool in = row < A.n;
        const double off = sell_row(A, s, lane, [&](int c) { return wd[c] * b[c]; });
        if (in) {
            const double bi = b[row], ti = wd[row] * bi;
            t[row] = ti;
            r[row] = bi - fma(d[row], ti, off);
        }
    }
}

// post-smoothing: x = t + (w/d) (b - A t); with DOT, also (b, x) reduced
// into the outer PCG's scalars (b = r and x = z of the outer iteration)
template <bool DOT>
__global__ void __launch_bounds__(kThreads) k_amg_post(DSell A, const double *__restrict__ d,
                                                       const double *__restrict__ wd,
                                                       const double *__restrict__ b,
                                                       const double *__restrict__ t,
                                                       double *__restrict__ x, const int *skip,
                                                       AmgScalars *S, double *part,
                                                       unsigned *count) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    double dot = 0.0;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off = sell_row(A, s, lane, [&](int c) { return t[c]; });
        if (row < A.n) {
            const double bi = b[row], ti = t[row];
            const double xi = fma(wd[row], bi - fma(d[row], ti, off), ti);
            x[row] = xi;
            if (DOT)
                dot = fma(bi, xi, dot);
        }
    }
    if (DOT) {
        double v[1] = {dot}, tot[1];
        if (grid_sum_last<1>(v, part, count, tot) && threadIdx.x == 0)
            set_rz(S, tot[0]);
    }
}

// b_c = R r, one warp per coarse row (fixed lane split and shuffle tree)
__global__ void __launch_bounds__(kThreads) k_amg_restrict(DCsr R, const double *__restrict__ r,
                                                           double *__restrict__ bc,
                                                           const int *skip) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * kWarps + (threadIdx.x >> 5); row < R.n;
         row += gridDim.x * kWarps) {
        double acc = 0.0;
        for (int k = R.ptr[row] + lane; k < R.ptr[row + 1]; k += 32)
            acc = fma(__ldcs(R.val + k), r[__ldcs(R.col + k)], acc);
        acc = warp_sum(acc);
        if (lane == 0)
            bc[row] = acc;
    }
}

// t += P x_c, one thread per fine row
__global__ void __launch_bounds__(kThreads) k_amg_prolong(DCsr P, const double *__restrict__ xc,
                                                          double *__restrict__ t,
                                                          const int *skip) {
    if (skip && *skip)
        return;
    for (int row = blockIdx.x * kThreads + threadIdx.x; row < P.n; row += gridDim.x * kThreads) {
        double acc = t[row];
        for (int k = P.ptr[row]; k < P.ptr[row + 1]; ++k)
            acc = fma(__ldcs(P.val + k), xc[__ldcs(P.col + k)], acc);
        t[row] = acc;
    }
}

// x = Minv b on the coarsest level, one warp per row; with DOT (a system
// that is its own coarsest level) also (b, x) into the outer scalars
template <bool DOT>
__global__ void __launch_bounds__(kThreads) k_amg_dense(int n, const double *__restrict__ Minv,
                                                        const double *__restrict__ b,
                                                        double *__restrict__ x, const int *skip,
                                                        AmgScalars *S, double *part,
                                                        unsigned *count) {
    if (skip && *skip)
        return;
    const int lane = threadIdx.x & 31;
    double dot = 0.0;
    for (int row = blockIdx.x * kWarps + (threadIdx.x >> 5); row < n; row += gridDim.x * kWarps) {
        double s = 0.0;
        for (int k = lane; k < n; k += 32)
            s = fma(Minv[(size_t)row * n + k], b[k], s);
        s = warp_sum(s);
        if (lane == 0) {
            x[row] = s;
            if (DOT)
                dot = fma(b[row], s, dot);
        }
    }
    if (DOT) {
        double v[1] = {dot}, tot[1];
        if (grid_sum_last<1>(v, part, count, tot) && threadIdx.x == 0)
            set_rz(S, tot[0]);
    }
}

// r = b - A x with (r, r) and (b, b) reduced: mode 0 starts a solve
// (bn2, thr2, rr; the next direction restarts), mode 1 confirms a
// converged recursive residual (rr only)
__global__ void __launch_bounds__(kThreads) k_amg_residual(DSell A, const double *__restrict__ d,
                                                           const double *__restrict__ b,
                                                           const double *__restrict__ x,
                                                           double *__restrict__ r, int mode,
                                                           AmgScalars *S, double *part,
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

__device__ __forceinline__ double next_p(double z, double beta, double p, int restart) {
    return restart ? z : fma(beta, p, z);
}

// p' = z + beta p (p' = z after a restart) and q = A p', p'_j formed on the
// fly from z_j and p_j; (p', q) reduced into alpha
__global__ void __launch_bounds__(kThreads) k_amg_q(DSell A, const double *__restrict__ d,
                                                    const double *__restrict__ z,
                                                    const double *__restrict__ p,
                                                    double *__restrict__ pn,
                                                    double *__restrict__ q, AmgScalars *S,
                                                    double *part, unsigned *count) {
    if (S->done)
        return;
    const int restart = S->restart;
    const double beta = S->beta;
    const int lane = threadIdx.x & 31;
    double pq = 0.0;
    FOR_SLICES(A) {
        const int row = s * 32 + lane;
        const double off =
            sell_row(A, s, lane, [&](int c) { return next_p(z[c], beta, p[c], restart); });
        if (row < A.n) {
            const double pi = next_p(z[row], beta, p[row], restart);
            const double qi = fma(d[row], pi, off);
            pn[row] = pi;
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

// x += alpha p; r -= alpha q; (r, r) reduced; the iteration is counted and
// the loop stops when the recursive residual meets the tolerance or maxit
// iterations have run
__global__ void __launch_bounds__(kThreads) k_amg_xr(int n, const double *__restrict__ p,
                                                     const double *__restrict__ q,
                                                     double *__restrict__ x,
                                                     double *__restrict__ r, AmgScalars *S,
                                                     double *part, unsigned *count) {
    if (S->done)
        return;
    const double alpha = S->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
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

int grid_rows(int64_t n) {   // blocks for one warp per 32-row slice (or per row)
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, kMaxBlocks));
}

int grid_warps(int64_t n) {  // blocks for one warp per row
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kWarps - 1) / kWarps, kMaxBlocks));
}

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

template <typename T>
cudaError_t alloc(T **dst, int64_t count, int64_t *bytes) {
    *dst = nullptr;
    const size_t sz = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = cudaMalloc((void **)dst, sz);
    if (e == cudaSuccess)
        *bytes += (int64_t)sz;
    return e;
}

// host sliced-ELL image of A's off-diagonal part
struct HSell {
    std::vector<int> sp, sw, col;
    std::vector<double> val;
};

// false when the padded slot count does not fit an int
bool sell_of(const HCsr &A, HSell &S) {
    const int64_t ns = (A.n + 31) / 32;
    S.sp.assign((size_t)ns + 1, 0);
    S.sw.assign((size_t)ns, 0);
    int64_t total = 0;
    for (int64_t s = 0; s < ns; ++s) {
        int w = 0;
        for (int64_t row = s * 32; row < std::min<int64_t>(A.n, s * 32 + 32); ++row) {
            int len = 0;
            for (int64_t k = A.ptr[(size_t)row]; k < A.ptr[(size_t)row + 1]; ++k)
                len += A.col[(size_t)k] != row;
            w = std::max(w, len);
        }
        S.sw[(size_t)s] = w;
        total += 32 * (int64_t)w;
        if (total > INT32_MAX)
            return false;
        S.sp[(size_t)s + 1] = (int)total;
    }
    S.col.assign((size_t)S.sp.back(), 0);
    S.val.assign((size_t)S.sp.back(), 0.0);
    for (int64_t row = 0; row < A.n; ++row) {
        const int64_t s = row / 32, i = row % 32;
        int k = 0;
        for (int64_t e = A.ptr[(size_t)row]; e < A.ptr[(size_t)row + 1]; ++e) {
            if (A.col[(size_t)e] == row)
                continue;
            const size_t at = (size_t)S.sp[(size_t)s] + (size_t)k * 32 + (size_t)i;
            S.col[at] = A.col[(size_t)e];
            S.val[at] = A.val[(size_t)e];
            ++k;
        }
    }
    return true;
}

}  // namespace

// one level above the coarsest
struct amg_level {
    int64_t n = 0, nnz = 0;
    double w = 0.0;
    int *a_sp = nullptr, *a_sw = nullptr, *a_col = nullptr;   // A off-diagonal, sliced ELL
    double *a_val = nullptr, *d = nullptr, *wd = nullptr;      // values, diagonal, w / diagonal
    int *p_ptr = nullptr, *p_col = nullptr;                    // P: n x n_next
    double *p_val = nullptr;
    int *r_ptr = nullptr, *r_col = nullptr;                    // R = P^T: n_next x n
    double *r_val = nullptr;
    double *t = nullptr, *r = nullptr;                         // smoothed iterate, residual
    double *x = nullptr, *b = nullptr;                         // level >= 1: cycle output, input
    std::vector<int32_t> agg;                                  // host copy, for inspection
    DSell A() const { return DSell{(int)n, a_sp, a_sw, a_col, a_val}; }
};

struct ldu_amg {
    int device = 0;
    int64_t n = 0;
    std::vector<amg_level> lev;     // every level that has a prolongator
    // the fine matrix when it is itself the coarsest (no prolongator)
    int *f_sp = nullptr, *f_sw = nullptr, *f_col = nullptr;
    double *f_val = nullptr, *f_d = nullptr;
    int64_t nc = 0, c_nnz = 0;      // coarsest rows and non-zeros
    double *cinv = nullptr;         // coarsest dense inverse (row-major)
    double *cx = nullptr, *cb = nullptr;
    double *r = nullptr, *z = nullptr, *p[2] = {nullptr, nullptr}, *q = nullptr;
    double *part = nullptr;
    unsigned *count = nullptr;
    AmgScalars *S = nullptr;        // device
    AmgScalars *S_host = nullptr;   // pinned
    int64_t device_bytes = 0;
    DSell fine() const {
        return lev.empty() ? DSell{(int)n, f_sp, f_sw, f_col, f_val} : lev[0].A();
    }
    const double *fine_d() const { return lev.empty() ? f_d : lev[0].d; }
};

namespace {

void free_amg(ldu_amg *M) {
    if (!M)
        return;
    for (auto &L : M->lev) {
        void *ptrs[] = {L.a_sp, L.a_sw, L.a_col, L.a_val, L.d,     L.wd, L.p_ptr, L.p_col,
                        L.p_val, L.r_ptr, L.r_col, L.r_val, L.t, L.r,  L.x,     L.b};
        for (void *p : ptrs)
            if (p)
                cudaFree(p);
    }
    void *ptrs[] = {M->f_sp, M->f_sw, M->f_col, M->f_val, M->f_d, M->cinv, M->cx, M->cb,
                    M->r,    M->z,    M->p[0],  M->p[1],  M->q,   M->part, M->count, M->S};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (M->S_host)
        cudaFreeHost(M->S_host);
    delete M;
}

// x = V(b) from level l down (level 0: b and x are the caller's); with DOT the
// last kernel also reduces (b, x) into the outer scalars
int vcycle(ldu_amg *M, size_t l, const double *b, double *x, bool dot, const int *skip,
           cudaStream_t st) {
    if (l == M->lev.size()) {
        if (dot)
            k_amg_dense<true><<<grid_warps(M->nc), kThreads, 0, st>>>((int)M->nc, M->cinv, b, x,
                                                                      skip, M->S, M->part,
                                                                      M->count);
        else
            k_amg_dense<false><<<grid_warps(M->nc), kThreads, 0, st>>>(
                (int)M->nc, M->cinv, b, x, skip, nullptr, nullptr, nullptr);
        return cuda_status(cudaGetLastError());
    }
    const amg_level &L = M->lev[l];
    const DSell A = L.A();
    const int ga = grid_rows(L.n);
    k_amg_pre<<<ga, kThreads, 0, st>>>(A, L.d, L.wd, b, L.t, L.r, skip);
    const bool last = l + 1 == M->lev.size();
    const int64_t nn = last ? M->nc : M->lev[l + 1].n;
    double *bn = last ? M->cb : M->lev[l + 1].b;
    double *xn = last ? M->cx : M->lev[l + 1].x;
    k_amg_restrict<<<grid_warps(nn), kThreads, 0, st>>>(DCsr{(int)nn, L.r_ptr, L.r_col, L.r_val},
                                                         L.r, bn, skip);
    const int rc = vcycle(M, l + 1, bn, xn, false, skip, st);
    if (rc != LDU_OK)
        return rc;
    k_amg_prolong<<<grid_rows(L.n), kThreads, 0, st>>>(DCsr{(int)L.n, L.p_ptr, L.p_col, L.p_val},
                                                        xn, L.t, skip);
    if (dot)
        k_amg_post<true><<<ga, kThreads, 0, st>>>(A, L.d, L.wd, b, L.t, x, skip, M->S, M->part,
                                                  M->count);
    else
        k_amg_post<false><<<ga, kThreads, 0, st>>>(A, L.d, L.wd, b, L.t, x, skip, nullptr,
                                                   nullptr, nullptr);
    return cuda_status(cudaGetLastError());
}

// the outer scalars to the pinned host copy (synchronises st)
int read_scalars(ldu_amg *M, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(M->S_host, M->S, sizeof(AmgScalars), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

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
    int max_coarse = 500, max_levels = 12;
    if (aopt) {
        if (aopt->max_coarse)
            max_coarse = aopt->max_coarse;
        if (aopt->max_levels)
            max_levels = aopt->max_levels;
    }
    if (max_coarse < 1 || max_coarse > kMaxCoarse || max_levels < 1 || max_levels > 64)
        return LDU_ERR_BAD_ARG;
    if (n > INT32_MAX / 2 || nf > INT32_MAX / 2)
        return LDU_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    // a host copy of the fine matrix, validated as ldu_create does
    std::vector<int32_t> ho((size_t)nf), hn((size_t)nf);
    std::vector<double> hd((size_t)n), hu((size_t)nf), hl((size_t)nf);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && nf > 0) {
        e = cudaMemcpy(ho.data(), owner, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hn.data(), neighbour, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hu.data(), upper, sizeof(double) * nf, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hl.data(), lower, sizeof(double) * nf, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(hd.data(), diag, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_status(e);
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t o = ho[(size_t)f], b = hn[(size_t)f];
        if (o < 0 || b < 0 || o >= n || b >= n || o >= b)
            return LDU_ERR_BAD_ADDRESSING;
        if (!std::isfinite(hu[(size_t)f]) || !std::isfinite(hl[(size_t)f]))
            return LDU_ERR_NOT_SPD;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(hd[(size_t)i]) || !(hd[(size_t)i] > 0.0))
            return LDU_ERR_NOT_SPD;
    HCsr A = csr_from_ldu(n, nf, ho.data(), hn.data(), hd.data(), hu.data(), hl.data());
    std::vector<int32_t>().swap(ho);
    std::vector<int32_t>().swap(hn);

    ldu_amg *M = new ldu_amg();
    cudaGetDevice(&M->device);
    M->n = n;
#define CKA(call)                  \
    do {                           \
        e = (call);                \
        if (e != cudaSuccess) {    \
            free_amg(M);           \
            return cuda_status(e); \
        }                          \
    } while (0)
    bool fine_uploaded = false;
    // coarsen while the level is above max_coarse rows and aggregation shrinks it
    while (A.n > max_coarse && (int)M->lev.size() < max_levels) {
        std::vector<int32_t> agg;
        const int64_t na = aggregate(A, agg);
        if (na >= A.n)
            break;
        M->lev.emplace_back();
        amg_level &L = M->lev.back();
        L.n = A.n;
        L.nnz = (int64_t)A.col.size();
        L.w = jacobi_weight(A);
        HCsr P = prolongator(A, agg, na, L.w);
        HCsr R = transpose(P);
        if ((int64_t)P.col.size() > INT32_MAX) {
            free_amg(M);
            return LDU_ERR_UNSUPPORTED;
        }
        HCsr Ac = galerkin(A, P, R);
        L.agg = std::move(agg);
        HSell S;
        if (!sell_of(A, S)) {
            free_amg(M);
            return LDU_ERR_UNSUPPORTED;
        }
        std::vector<double> d((size_t)A.n), wd((size_t)A.n);
        for (int64_t i = 0; i < A.n; ++i) {
            d[(size_t)i] = diag_of(A, i);
            wd[(size_t)i] = L.w / d[(size_t)i];
        }
        std::vector<int> pp(P.ptr.begin(), P.ptr.end()), rp(R.ptr.begin(), R.ptr.end());
        CKA(upload(&L.a_sp, S.sp, &M->device_bytes));
        CKA(upload(&L.a_sw, S.sw, &M->device_bytes));
        CKA(upload(&L.a_col, S.col, &M->device_bytes));
        CKA(upload(&L.a_val, S.val, &M->device_bytes));
        CKA(upload(&L.d, d, &M->device_bytes));
        CKA(upload(&L.wd, wd, &M->device_bytes));
        CKA(upload(&L.p_ptr, pp, &M->device_bytes));
        CKA(upload(&L.p_col, P.col, &M->device_bytes));
        CKA(upload(&L.p_val, P.val, &M->device_bytes));
        CKA(upload(&L.r_ptr, rp, &M->device_bytes));
        CKA(upload(&L.r_col, R.col, &M->device_bytes));
        CKA(upload(&L.r_val, R.val, &M->device_bytes));
        CKA(alloc(&L.t, L.n, &M->device_bytes));
        CKA(alloc(&L.r, L.n, &M->device_bytes));
        if (M->lev.size() > 1) {
            CKA(alloc(&L.x, L.n, &M->device_bytes));
            CKA(alloc(&L.b, L.n, &M->device_bytes));
        }
        fine_uploaded = true;
        A = std::move(Ac);
    }
    if (!fine_uploaded) {
        // the fine matrix is the coarsest: keep its SpMV form for the outer loop
        HSell S;
        if (!sell_of(A, S)) {
            free_amg(M);
            return LDU_ERR_UNSUPPORTED;
        }
        std::vector<double> d((size_t)A.n);
        for (int64_t i = 0; i < A.n; ++i)
            d[(size_t)i] = diag_of(A, i);
        CKA(upload(&M->f_sp, S.sp, &M->device_bytes));
        CKA(upload(&M->f_sw, S.sw, &M->device_bytes));
        CKA(upload(&M->f_col, S.col, &M->device_bytes));
        CKA(upload(&M->f_val, S.val, &M->device_bytes));
        CKA(upload(&M->f_d, d, &M->device_bytes));
    }
    // the coarsest level, applied through its dense inverse
    if (A.n > kMaxCoarse) {
        free_amg(M);   // coarsening stopped above what a dense inverse allows
        return LDU_ERR_UNSUPPORTED;
    }
    M->nc = A.n;
    M->c_nnz = (int64_t)A.col.size();
    std::vector<double> inv;
    if (!dense_inverse(A, inv)) {
        free_amg(M);
        return LDU_ERR_NOT_SPD;
    }
    CKA(upload(&M->cinv, inv, &M->device_bytes));
    CKA(alloc(&M->cx, A.n, &M->device_bytes));
    CKA(alloc(&M->cb, A.n, &M->device_bytes));
    CKA(alloc(&M->r, n, &M->device_bytes));
    CKA(alloc(&M->z, n, &M->device_bytes));
    CKA(alloc(&M->p[0], n, &M->device_bytes));
    CKA(alloc(&M->p[1], n, &M->device_bytes));
    CKA(alloc(&M->q, n, &M->device_bytes));
    CKA(alloc(&M->part, 2 * kMaxBlocks, &M->device_bytes));
    CKA(alloc(&M->count, 1, &M->device_bytes));
    CKA(cudaMemset(M->count, 0, sizeof(unsigned)));
    CKA(alloc(&M->S, 1, &M->device_bytes));
    CKA(cudaMallocHost((void **)&M->S_host, sizeof(AmgScalars)));
#undef CKA
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
    const auto &a = M->lev[(size_t)level].agg;
    std::memcpy(agg, a.data(), sizeof(int32_t) * a.size());
    return LDU_OK;
}

int ldu_amg_vcycle(ldu_amg *M, const double *b, double *x, ldu_stream_t stream) {
    if (!M || !b || !x || b == x)
        return LDU_ERR_BAD_ARG;
    return vcycle(M, 0, b, x, false, nullptr, (cudaStream_t)stream);
}

int amg_pcg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
                  double *relres, ldu_stream_t stream) {
    if (!M || !b || !x || b == x || maxit < 0 || !(tol >= 0.0))
        return LDU_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const DSell A = M->fine();
    const double *d = M->fine_d();
    const int64_t n = M->n;
    const int ga = grid_rows(n);
    AmgScalars *S = M->S, *H = M->S_host;
    std::memset(H, 0, sizeof(AmgScalars));
    H->tol2 = tol * tol;
    H->maxit = maxit;
    H->status = LDU_OK;
    cudaError_t e = cudaMemcpyAsync(S, H, sizeof(AmgScalars), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return cuda_status(e);
    int rc = LDU_OK;
    // r = b - A x0, then z = V(r) and (r, z)
    k_amg_residual<<<ga, kThreads, 0, st>>>(A, d, b, x, M->r, 0, S, M->part, M->count);
    if ((rc = vcycle(M, 0, M->r, M->z, true, nullptr, st)) != LDU_OK)
        return rc;
    if ((rc = read_scalars(M, st)) != LDU_OK)
        return rc;
    int status = LDU_NOT_CONVERGED, it = 0, cur = 0;
    bool confirmed = false;   // H->rr holds the true residual of the final x
    const double bn2 = H->bn2, thr2 = H->thr2;
    if (bn2 == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st);
        status = LDU_OK;
    } else if (H->rr <= thr2) {
        status = LDU_OK;
    } else if (maxit == 0) {
        status = LDU_NOT_CONVERGED;
    } else {
        // iterations in batches between host reads, sized from the observed
        // convergence rate so that few kernels run past the stopping point
        double rr_prev = H->rr;
        int it_prev = 0, batch = 4;
        for (;;) {
            for (int g = 0; g < batch; ++g) {
                k_amg_q<<<ga, kThreads, 0, st>>>(A, d, M->z, M->p[cur], M->p[cur ^ 1], M->q, S,
                                                 M->part, M->count);
                cur ^= 1;
                k_amg_xr<<<grid_rows(n), kThreads, 0, st>>>((int)n, M->p[cur], M->q, x, M->r, S,
                                                            M->part, M->count);
                if ((rc = vcycle(M, 0, M->r, M->z, true, &S->done, st)) != LDU_OK)
                    return rc;
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
                k_amg_residual<<<ga, kThreads, 0, st>>>(A, d, b, x, M->r, 1, S, M->part, M->count);
                if ((rc = read_scalars(M, st)) != LDU_OK)
                    return rc;
                if (H->rr <= thr2) {
                    status = LDU_OK;
                    confirmed = true;
                    break;
                }
                if ((rc = vcycle(M, 0, M->r, M->z, true, nullptr, st)) != LDU_OK)
                    return rc;
                if (it >= maxit)
                    break;
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
    if (bn2 > 0.0 && (confirmed || (status == LDU_OK && it == 0))) {
        tr = std::sqrt(H->rr / bn2);
    } else if (bn2 > 0.0) {
        k_amg_residual<<<ga, kThreads, 0, st>>>(A, d, b, x, M->r, 1, S, M->part, M->count);
        if ((rc = read_scalars(M, st)) != LDU_OK)
            return rc;
        tr = std::sqrt(H->rr / bn2);
    }
    if (iters)
        *iters = it;
    if (relres)
        *relres = tr;
    return status;
}

}  // extern "C"
