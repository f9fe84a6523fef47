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
// a solve runs in the kernels below and the levels' SpMV kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ldupcg_impl.cuh"
#include "setup_kernels.cuh"

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

double entry(const HCsr &A, int64_t i, int32_t j) {
    const int32_t *b = A.col.data() + A.ptr[(size_t)i], *e = A.col.data() + A.ptr[(size_t)i + 1];
    const int32_t *p = std::lower_bound(b, e, j);
    return (p != e && *p == j) ? A.val[(size_t)(p - A.col.data())] : 0.0;
}

// LDU arrays of a CSR matrix: faces are the upper-triangle entries
void ldu_of(const HCsr &A, std::vector<int32_t> &own, std::vector<int32_t> &nbr,
            std::vector<double> &diag, std::vector<double> &up, std::vector<double> &lo) {
    diag.assign((size_t)A.n, 0.0);
    own.clear();
    nbr.clear();
    up.clear();
    lo.clear();
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.ptr[(size_t)i]; k < A.ptr[(size_t)i + 1]; ++k) {
            const int32_t j = A.col[(size_t)k];
            if (j == i) {
                diag[(size_t)i] = A.val[(size_t)k];
            } else if (j > i) {
                own.push_back((int32_t)i);
                nbr.push_back(j);
                up.push_back(A.val[(size_t)k]);
                lo.push_back(entry(A, j, (int32_t)i));
            }
        }
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

// ---- device kernels of a V-cycle and of the outer PCG -------------------------

#define GRID_STRIDE(i, n)                                                                \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// x = w b / d (the first Jacobi sweep from zero)
__global__ void k_amg_jacobi0(int64_t n, double w, const double *b, const double *d, double *x) {
    GRID_STRIDE(i, n) x[i] = w * b[i] / d[i];
}

// r = b - y
__global__ void k_amg_sub(int64_t n, const double *b, const double *y, double *r) {
    GRID_STRIDE(i, n) r[i] = b[i] - y[i];
}

// x += w (b - y) / d
__global__ void k_amg_post(int64_t n, double w, const double *b, const double *y,
                           const double *d, double *x) {
    GRID_STRIDE(i, n) x[i] += w * (b[i] - y[i]) / d[i];
}

// y = M x (add = 0) or y += M x (add = 1), M in CSR, one thread per row
__global__ void k_csr_mv(int64_t n, const int *ptr, const int *col, const double *val,
                         const double *x, double *y, int add) {
    GRID_STRIDE(i, n) {
        double s = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            s = fma(val[k], x[col[k]], s);
        y[i] = add ? y[i] + s : s;
    }
}

// x = Minv b for the small dense coarsest matrix: one warp per row
__global__ void k_dense_mv(int n, const double *Minv, const double *b, double *x) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n)
        return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32)
        s = fma(Minv[(size_t)warp * n + k], b[k], s);
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_down_sync(kFullMask, s, o);
    if (lane == 0)
        x[warp] = s;
}

constexpr int kDotBlocks = 256;

// partial dot products (u, v) and (u2, v2) of each block's fixed range
__global__ void k_dot2(int64_t n, const double *u, const double *v, const double *u2,
                       const double *v2, double *part) {
    __shared__ double sm[2][32];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = std::min<int64_t>(n, lo + per);
    double a = 0.0, c = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        a = fma(u[i], v[i], a);
        if (u2)
            c = fma(u2[i], v2[i], c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFullMask, a, o);
        c += __shfl_down_sync(kFullMask, c, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sm[0][warp] = a;
        sm[1][warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += sm[0][k];
            s1 += sm[1][k];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

// the block partials summed in block order (one thread: 256 pairs)
__global__ void k_dot_total(int nb, const double *part, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < nb; ++k) {
            s0 += part[2 * k];
            s1 += part[2 * k + 1];
        }
        out[0] = s0;
        out[1] = s1;
    }
}

// x += a p ; r -= a q
__global__ void k_amg_xr(int64_t n, double a, const double *p, const double *q, double *x,
                         double *r) {
    GRID_STRIDE(i, n) {
        x[i] = fma(a, p[i], x[i]);
        r[i] = fma(-a, q[i], r[i]);
    }
}

// p = z + beta p
__global__ void k_amg_p(int64_t n, double beta, const double *z, double *p) {
    GRID_STRIDE(i, n) p[i] = fma(beta, p[i], z[i]);
}

int blocks_of(int64_t n, int t = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 4096));
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

}  // namespace

// one level above the coarsest: its matrix handle, weight, transfers, vectors
struct amg_level {
    ldu_matrix *A = nullptr;   // level 0: the fine handle (owned by ldu_amg::fine)
    int64_t n = 0, nnz = 0;
    double w = 0.0;
    int *p_ptr = nullptr, *p_col = nullptr;    // P: n x n_next
    double *p_val = nullptr;
    int *r_ptr = nullptr, *r_col = nullptr;    // R = P^T: n_next x n
    double *r_val = nullptr;
    double *x = nullptr, *b = nullptr;         // level vectors (null on level 0: the caller's)
    double *y = nullptr;                       // A x and residuals
    std::vector<int32_t> agg;                  // host copy, for inspection
};

struct ldu_amg {
    int device = 0;
    ldu_matrix *fine = nullptr;
    std::vector<amg_level> lev;     // every level that has a prolongator
    int64_t nc = 0, c_nnz = 0;      // coarsest rows and non-zeros
    double *cinv = nullptr;         // coarsest dense inverse (row-major)
    double *cx = nullptr, *cb = nullptr;
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;   // outer PCG vectors
    double *part = nullptr, *dots = nullptr, *dots_host = nullptr;   // reductions (host: pinned)
    int64_t device_bytes = 0;
};

namespace {

void free_amg(ldu_amg *M) {
    if (!M)
        return;
    for (size_t l = 0; l < M->lev.size(); ++l) {
        amg_level &L = M->lev[l];
        if (l > 0 && L.A)
            ldu_destroy(L.A);
        void *ptrs[] = {L.p_ptr, L.p_col, L.p_val, L.r_ptr, L.r_col, L.r_val, L.x, L.b, L.y};
        for (void *p : ptrs)
            if (p)
                cudaFree(p);
    }
    if (M->fine)
        ldu_destroy(M->fine);
    void *ptrs[] = {M->cinv, M->cx, M->cb, M->r, M->z, M->p, M->q, M->part, M->dots};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (M->dots_host)
        cudaFreeHost(M->dots_host);
    delete M;
}

// a device handle of a coarse matrix (its LDU arrays staged through the device)
int coarse_handle(const HCsr &A, ldu_stream_t stream, ldu_matrix **out) {
    std::vector<int32_t> co, cn;
    std::vector<double> cd, cu, cl;
    ldu_of(A, co, cn, cd, cu, cl);
    int32_t *d_o = nullptr, *d_n = nullptr;
    double *d_d = nullptr, *d_u = nullptr, *d_l = nullptr;
    int64_t tmp = 0;
    int rc = LDU_OK;
    cudaError_t e = upload(&d_o, co, &tmp);
    if (e == cudaSuccess)
        e = upload(&d_n, cn, &tmp);
    if (e == cudaSuccess)
        e = upload(&d_d, cd, &tmp);
    if (e == cudaSuccess)
        e = upload(&d_u, cu, &tmp);
    if (e == cudaSuccess)
        e = upload(&d_l, cl, &tmp);
    if (e != cudaSuccess) {
        rc = cuda_status(e);
    } else {
        ldu_opts o{};
        o.slice_rows = 32;   // coarse rows have wide, uneven stencils
        o.staging = -1;
        rc = ldu_create(A.n, (int64_t)co.size(), d_o, d_n, d_d, d_u, d_l, &o, stream, out);
        cudaStreamSynchronize((cudaStream_t)stream);
    }
    void *ptrs[] = {d_o, d_n, d_d, d_u, d_l};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    return rc;
}

// z = V(b) on level l (level 0: b and x given)
int vcycle(ldu_amg *M, size_t l, const double *b, double *x, cudaStream_t st) {
    if (l == M->lev.size()) {
        k_dense_mv<<<(int)((M->nc * 32 + 255) / 256), 256, 0, st>>>((int)M->nc, M->cinv, b, x);
        return cuda_status(cudaGetLastError());
    }
    amg_level &L = M->lev[l];
    const int64_t n = L.n;
    const int gb = blocks_of(n);
    ldu_matrix *A = L.A;
    const int sp = (int)((n + 255) / 256);
    k_amg_jacobi0<<<gb, 256, 0, st>>>(n, L.w, b, A->dg, x);
    k_spmv<double><<<sp, 256, 0, st>>>((int)n, A->C, A->slice_ptr, A->slice_w, A->col, A->val64,
                                       A->sd, x, L.y);
    k_amg_sub<<<gb, 256, 0, st>>>(n, b, L.y, L.y);
    const int64_t nn = l + 1 < M->lev.size() ? M->lev[l + 1].n : M->nc;
    double *bn = l + 1 < M->lev.size() ? M->lev[l + 1].b : M->cb;
    double *xn = l + 1 < M->lev.size() ? M->lev[l + 1].x : M->cx;
    k_csr_mv<<<blocks_of(nn), 256, 0, st>>>(nn, L.r_ptr, L.r_col, L.r_val, L.y, bn, 0);
    int rc = vcycle(M, l + 1, bn, xn, st);
    if (rc != LDU_OK)
        return rc;
    k_csr_mv<<<gb, 256, 0, st>>>(n, L.p_ptr, L.p_col, L.p_val, xn, x, 1);
    k_spmv<double><<<sp, 256, 0, st>>>((int)n, A->C, A->slice_ptr, A->slice_w, A->col, A->val64,
                                       A->sd, x, L.y);
    k_amg_post<<<gb, 256, 0, st>>>(n, L.w, b, L.y, A->dg, x);
    return cuda_status(cudaGetLastError());
}

// (u, v) and (u2, v2) to the pinned host pair dots_host (synchronises st)
int dot2(ldu_amg *M, int64_t n, const double *u, const double *v, const double *u2,
         const double *v2, cudaStream_t st, double &a, double &c) {
    k_dot2<<<kDotBlocks, 256, 0, st>>>(n, u, v, u2, v2, M->part);
    k_dot_total<<<1, 32, 0, st>>>(kDotBlocks, M->part, M->dots);
    cudaError_t e = cudaMemcpyAsync(M->dots_host, M->dots, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_status(e);
    a = M->dots_host[0];
    c = M->dots_host[1];
    return LDU_OK;
}

}  // namespace

extern "C" {

int ldu_amg_create(int64_t n, int64_t nf, const int32_t *owner, const int32_t *neighbour,
                   const double *diag, const double *upper, const double *lower,
                   const ldu_opts *opt, const amg_opts *aopt, ldu_stream_t stream,
                   ldu_amg **out) {
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
    cudaStream_t st = (cudaStream_t)stream;
    ldu_amg *M = new ldu_amg();
    cudaGetDevice(&M->device);
    int rc = ldu_create(n, nf, owner, neighbour, diag, upper, lower, opt, stream, &M->fine);
    if (rc != LDU_OK) {
        free_amg(M);
        return rc;
    }
    cudaError_t e = cudaSuccess;
#define CKA(call)                \
    do {                         \
        e = (call);              \
        if (e != cudaSuccess) {  \
            free_amg(M);         \
            return cuda_status(e); \
        }                        \
    } while (0)
    // a host copy of the fine matrix (the handle validated its addressing)
    std::vector<int32_t> ho((size_t)nf), hn((size_t)nf);
    std::vector<double> hd((size_t)n), hu((size_t)nf), hl((size_t)nf);
    CKA(cudaStreamSynchronize(st));
    if (nf > 0) {
        CKA(cudaMemcpy(ho.data(), owner, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost));
        CKA(cudaMemcpy(hn.data(), neighbour, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost));
        CKA(cudaMemcpy(hu.data(), upper, sizeof(double) * nf, cudaMemcpyDeviceToHost));
        CKA(cudaMemcpy(hl.data(), lower, sizeof(double) * nf, cudaMemcpyDeviceToHost));
    }
    CKA(cudaMemcpy(hd.data(), diag, sizeof(double) * n, cudaMemcpyDeviceToHost));
    HCsr A = csr_from_ldu(n, nf, ho.data(), hn.data(), hd.data(), hu.data(), hl.data());
    std::vector<int32_t>().swap(ho);
    std::vector<int32_t>().swap(hn);
    // coarsen while the level is above max_coarse rows and aggregation shrinks it
    ldu_matrix *handle = M->fine;
    while (A.n > max_coarse && (int)M->lev.size() < max_levels) {
        std::vector<int32_t> agg;
        const int64_t na = aggregate(A, agg);
        if (na >= A.n)
            break;
        if (!handle) {
            rc = coarse_handle(A, stream, &handle);
            if (rc != LDU_OK) {
                free_amg(M);
                return rc;
            }
        }
        M->lev.emplace_back();
        amg_level &L = M->lev.back();
        L.A = handle;
        handle = nullptr;
        L.n = A.n;
        L.nnz = (int64_t)A.col.size();
        L.w = jacobi_weight(A);
        HCsr P = prolongator(A, agg, na, L.w);
        HCsr R = transpose(P);
        HCsr Ac = galerkin(A, P, R);
        L.agg = std::move(agg);
        std::vector<int> pp(P.ptr.begin(), P.ptr.end()), rp(R.ptr.begin(), R.ptr.end());
        const std::vector<double> zeros((size_t)L.n, 0.0);
        CKA(upload(&L.p_ptr, pp, &M->device_bytes));
        CKA(upload(&L.p_col, P.col, &M->device_bytes));
        CKA(upload(&L.p_val, P.val, &M->device_bytes));
        CKA(upload(&L.r_ptr, rp, &M->device_bytes));
        CKA(upload(&L.r_col, R.col, &M->device_bytes));
        CKA(upload(&L.r_val, R.val, &M->device_bytes));
        CKA(upload(&L.y, zeros, &M->device_bytes));
        if (M->lev.size() > 1) {
            CKA(upload(&L.x, zeros, &M->device_bytes));
            CKA(upload(&L.b, zeros, &M->device_bytes));
        }
        A = std::move(Ac);
    }
    // the coarsest level, applied through its dense inverse
    if (A.n > kMaxCoarse) {
        free_amg(M);   // coarsening stalled above what a dense inverse allows
        return LDU_ERR_UNSUPPORTED;
    }
    M->nc = A.n;
    M->c_nnz = (int64_t)A.col.size();
    std::vector<double> inv;
    if (!dense_inverse(A, inv)) {
        free_amg(M);
        return LDU_ERR_NOT_SPD;
    }
    const std::vector<double> zc((size_t)A.n, 0.0), zn((size_t)n, 0.0);
    CKA(upload(&M->cinv, inv, &M->device_bytes));
    CKA(upload(&M->cx, zc, &M->device_bytes));
    CKA(upload(&M->cb, zc, &M->device_bytes));
    CKA(upload(&M->r, zn, &M->device_bytes));
    CKA(upload(&M->z, zn, &M->device_bytes));
    CKA(upload(&M->p, zn, &M->device_bytes));
    CKA(upload(&M->q, zn, &M->device_bytes));
    CKA(upload(&M->part, std::vector<double>(2 * kDotBlocks, 0.0), &M->device_bytes));
    CKA(upload(&M->dots, std::vector<double>(2, 0.0), &M->device_bytes));
    CKA(cudaMallocHost((void **)&M->dots_host, 2 * sizeof(double)));
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
    if (!M || !b || !x)
        return LDU_ERR_BAD_ARG;
    return vcycle(M, 0, b, x, (cudaStream_t)stream);
}

int amg_pcg_solve(ldu_amg *M, const double *b, double *x, double tol, int maxit, int *iters,
                  double *relres, ldu_stream_t stream) {
    if (!M || !b || !x || maxit < 0 || !(tol >= 0.0))
        return LDU_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const ldu_matrix *A = M->fine;
    const int64_t n = A->n;
    const int gb = blocks_of(n), sp = (int)((n + 255) / 256);
    auto spmv = [&](const double *v, double *y) {
        k_spmv<double><<<sp, 256, 0, st>>>((int)n, A->C, A->slice_ptr, A->slice_w, A->col,
                                           A->val64, A->sd, v, y);
    };
    auto precond = [&](const double *r, double *z) {
        return ldu_amg_vcycle(M, r, z, stream);
    };
    double bn2 = 0.0, unused = 0.0;
    int rc = dot2(M, n, b, b, nullptr, nullptr, st, bn2, unused);
    if (rc != LDU_OK)
        return rc;
    int it = 0, status = LDU_NOT_CONVERGED;
    double rr = 0.0, rz = 0.0;
    if (bn2 == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st);
        status = LDU_OK;
    } else {
        const double thr2 = tol * tol * bn2;
        spmv(x, M->q);                                          // r = b - A x0
        k_amg_sub<<<gb, 256, 0, st>>>(n, b, M->q, M->r);
        if ((rc = precond(M->r, M->z)) != LDU_OK)
            return rc;
        if ((rc = dot2(M, n, M->r, M->z, M->r, M->r, st, rz, rr)) != LDU_OK)
            return rc;
        cudaMemcpyAsync(M->p, M->z, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        if (rr <= thr2)
            status = LDU_OK;
        while (status != LDU_OK && it < maxit) {
            spmv(M->p, M->q);
            double pq = 0.0;
            if ((rc = dot2(M, n, M->p, M->q, nullptr, nullptr, st, pq, unused)) != LDU_OK)
                return rc;
            if (!(pq > 0.0) || !(rz > 0.0)) {
                status = LDU_ERR_NOT_SPD;
                break;
            }
            const double alpha = rz / pq;
            k_amg_xr<<<gb, 256, 0, st>>>(n, alpha, M->p, M->q, x, M->r);
            ++it;
            if ((rc = precond(M->r, M->z)) != LDU_OK)
                return rc;
            double rz_new = 0.0;
            if ((rc = dot2(M, n, M->r, M->z, M->r, M->r, st, rz_new, rr)) != LDU_OK)
                return rc;
            if (rr <= thr2) {
                // confirm with the true residual; restart the search if it disagrees
                spmv(x, M->q);
                k_amg_sub<<<gb, 256, 0, st>>>(n, b, M->q, M->r);
                if ((rc = precond(M->r, M->z)) != LDU_OK)
                    return rc;
                if ((rc = dot2(M, n, M->r, M->z, M->r, M->r, st, rz, rr)) != LDU_OK)
                    return rc;
                if (rr <= thr2) {
                    status = LDU_OK;
                    break;
                }
                cudaMemcpyAsync(M->p, M->z, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice,
                                st);
                continue;
            }
            k_amg_p<<<gb, 256, 0, st>>>(n, rz_new / rz, M->z, M->p);
            rz = rz_new;
        }
    }
    // the true residual at exit
    double tr2 = 0.0;
    if (bn2 > 0.0) {
        spmv(x, M->q);
        k_amg_sub<<<gb, 256, 0, st>>>(n, b, M->q, M->r);
        if ((rc = dot2(M, n, M->r, M->r, nullptr, nullptr, st, tr2, unused)) != LDU_OK)
            return rc;
    }
    if (iters)
        *iters = it;
    if (relres)
        *relres = bn2 > 0.0 ? std::sqrt(tr2 / bn2) : 0.0;
    return status;
}

}  // extern "C"
