// amg_setup.cuh -- device construction of the aggregation-AMG hierarchy
// (Sec. 5; Table 2's AMG-CG, whose AMG the paper takes from CUSP, where the
// aggregation forms a distance-2 maximal independent set in parallel: Bell,
// Dalton & Olson, SIAM J. Sci. Comput. 34 (2012)).  Included by amg.cu.
//
// Every level is a CSR matrix on the device (rows with their diagonal,
// columns sorted).  Per level:
//   1. d = diag(A), rho = max_i sum_j |a_ij| / a_ii, w = 4 / (3 rho);
//   2. distance-2 MIS by rounds: every row holds (state, h_i), state 0
//      excluded, 1 undecided, 2 root, h_i = mix64((i + 1) * golden) (the
//      SplitMix64 output of counter i + 1, Steele, Lea & Flood 2014);
//      two sweeps of "largest pair over the row and its neighbours" give the
//      largest pair within distance 2; an undecided row whose largest pair is
//      its own becomes a root, one whose largest pair is a root's is excluded;
//   3. aggregates: roots numbered in row order; a row next to a root joins it;
//      the others join the assigned neighbour of largest |a_ij| (ties within
//      1e-12 of the row's largest |a_ij| go to the lower aggregate);
//   4. P = (I - w D^-1 A) P_t on the structural pattern of (I + A) P_t;
//   5. R = P^T; A P and A_c = R (A P), structural patterns (entries that
//      cancel are kept), each row's sums formed in a fixed order so the
//      result is the same on every run.
// Sparse products expand each output row's candidate entries into a hash
// table of its own (open addressing in a device scratch sized by an upper
// bound of the row's entries), one thread per row adding them in expansion
// order; the occupied entries are then sorted by column and packed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

namespace amgs {

constexpr int kT = 256;   // threads per block of the setup kernels
constexpr int64_t kLongRow = 2048;   // products of a row of C = X Y from which it takes a block
constexpr int64_t kLongSort = 256;   // entries of a transpose's row from which it takes a block
constexpr int kSortMax = 2048;       // largest row a block sorts in shared memory (24 KB)
constexpr size_t kSortSmem = (size_t)kSortMax * (sizeof(int) + sizeof(double));
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// the SplitMix64 finaliser (Steele, Lea & Flood 2014)
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

__device__ __forceinline__ uint64_t prio(int64_t i) { return mix64((uint64_t)(i + 1) * kGolden); }

inline int blocks(int64_t work) {
    const int64_t b = (work + kT - 1) / kT;
    return (int)(b < 1 ? 1 : (b > (1 << 30) ? (1 << 30) : b));
}

// ---- exclusive scan of int64 values (three passes, recursive over block sums)

constexpr int kScanItems = 1024;   // items per block: 256 threads x 4

// block-local exclusive scan of items [0, m) (in[] read as 0 at and past n);
// bsum[b] = the block's total
__global__ void k_scan_block(const int64_t *in, int64_t n, int64_t m, int64_t *out,
                             int64_t *bsum) {
    __shared__ int64_t sm[kT];
    const int64_t base = (int64_t)blockIdx.x * kScanItems + 4 * threadIdx.x;
    int64_t v[4], t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    sm[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < kT; o <<= 1) {   // inclusive scan of the thread totals
        const int64_t a = threadIdx.x >= (unsigned)o ? sm[threadIdx.x - o] : 0;
        __syncthreads();
        sm[threadIdx.x] += a;
        __syncthreads();
    }
    int64_t run = sm[threadIdx.x] - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < m)
            out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kT - 1)
        bsum[blockIdx.x] = sm[kT - 1];
}

__global__ void k_scan_add(int64_t *out, const int64_t *boff, int64_t m) {
    const int64_t add = boff[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t j = base + (int64_t)k * kT;
        if (j < m)
            out[j] += add;
    }
}

// scratch items scan_excl needs for n inputs
inline int64_t scan_tmp_items(int64_t n) {
    const int64_t nb = (n + 1 + kScanItems - 1) / kScanItems;
    return nb > 1 ? 2 * nb + 1 + scan_tmp_items(nb) : nb;
}

// out[i] = in[0] + ... + in[i - 1] for i = 0..n (out[n] is the total); in
// and out must not alias; tmp holds scan_tmp_items(n) items
inline void scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                      cudaStream_t st) {
    const int64_t m = n + 1;
    const int64_t nb = (m + kScanItems - 1) / kScanItems;
    int64_t *bsum = tmp;
    k_scan_block<<<(unsigned)nb, kT, 0, st>>>(in, n, m, out, bsum);
    if (nb > 1) {
        int64_t *boff = tmp + nb;   // nb + 1 entries
        scan_excl(bsum, boff, nb, boff + nb + 1, st);
        k_scan_add<<<(unsigned)nb, kT, 0, st>>>(out, boff, m);
    }
}

// ---- the level-0 CSR from LDU faces -------------------------------------

__global__ void k_ldu_len(int64_t nf, const int32_t *own, const int32_t *nbr, int64_t *len) {
    const int64_t f = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (f < nf) {
        atomicAdd((unsigned long long *)&len[own[f]], 1ull);
        atomicAdd((unsigned long long *)&len[nbr[f]], 1ull);
    }
}

__global__ void k_ones(int64_t n, int64_t *len) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n)
        len[i] = 1;
}

// entry slots of the expanded rows: (column, value, order key); the diagonal
// first, then each face's two entries at atomically claimed slots (their
// order key is the face number, so the sort below restores face order)
__global__ void k_ldu_fill_diag(int64_t n, const int64_t *ptr, const double *diag, int *col,
                                double *val, int64_t *key, int64_t *cur) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n) {
        const int64_t at = ptr[i];
        col[at] = (int)i;
        val[at] = diag[i];
        key[at] = -1;
        cur[i] = at + 1;
    }
}

__global__ void k_ldu_fill_faces(int64_t nf, const int32_t *own, const int32_t *nbr,
                                 const double *up, const double *lo, int *col, double *val,
                                 int64_t *key, int64_t *cur) {
    const int64_t f = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (f < nf) {
        const int o = own[f], b = nbr[f];
        const int64_t a1 = (int64_t)atomicAdd((unsigned long long *)&cur[o], 1ull);
        col[a1] = b;
        val[a1] = up[f];
        key[a1] = f;
        const int64_t a2 = (int64_t)atomicAdd((unsigned long long *)&cur[b], 1ull);
        col[a2] = o;
        val[a2] = lo[f];
        key[a2] = f;
    }
}

// In-place sort of m entries (column c, order key q, value v) by (c, q),
// every (c, q) pair distinct, so the result does not depend on the method:
// insertion sort for the short rows of a mesh, heapsort (m log m) for the
// long rows of transposes and coarse levels.
__device__ __forceinline__ bool entry_less(const int *c, const int64_t *q, int64_t a, int64_t b) {
    return c[a] < c[b] || (c[a] == c[b] && (q ? q[a] < q[b] : false));
}

__device__ __forceinline__ void entry_swap(int *c, int64_t *q, double *v, int64_t a, int64_t b) {
    const int tc = c[a];
    c[a] = c[b];
    c[b] = tc;
    const double tv = v[a];
    v[a] = v[b];
    v[b] = tv;
    if (q) {
        const int64_t tq = q[a];
        q[a] = q[b];
        q[b] = tq;
    }
}

__device__ void sort_entries(int *c, int64_t *q, double *v, int64_t m) {
    if (m <= 32) {
        for (int64_t k = 1; k < m; ++k)
            for (int64_t j = k; j > 0 && entry_less(c, q, j, j - 1); --j)
                entry_swap(c, q, v, j, j - 1);
        return;
    }
    auto sift = [&](int64_t root, int64_t end) {   // max-heap on [0, end)
        for (;;) {
            int64_t child = 2 * root + 1;
            if (child >= end)
                return;
            if (child + 1 < end && entry_less(c, q, child, child + 1))
                ++child;
            if (!entry_less(c, q, root, child))
                return;
            entry_swap(c, q, v, root, child);
            root = child;
        }
    };
    for (int64_t r = m / 2 - 1; r >= 0; --r)
        sift(r, m);
    for (int64_t end = m - 1; end > 0; --end) {
        entry_swap(c, q, v, 0, end);
        sift(0, end);
    }
}

// sort each row's entries by (column, key) in place, add entries of equal
// column in key order, and write the number of distinct columns to cnt[i];
// the merged entries are left at the front of the row
__global__ void k_row_sort_merge(int64_t n, const int64_t *ptr, int *col, double *val,
                                 int64_t *key, int64_t *cnt, int64_t max_len = INT64_MAX) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    const int64_t b = ptr[i], e = ptr[i + 1];
    if (e - b > max_len)
        return;   // a long row: sorted by k_sort_long_rows (distinct keys, no merging)
    sort_entries(col + b, key + b, val + b, e - b);
    int64_t w = b;
    for (int64_t k = b; k < e; ++k) {
        if (k > b && col[k] == col[w - 1]) {
            val[w - 1] += val[k];
            continue;
        }
        col[w] = col[k];
        val[w] = val[k];
        ++w;
    }
    cnt[i] = w - b;
}

// copy the first cnt entries of every expanded row into the packed CSR
__global__ void k_pack(int64_t n, const int64_t *xptr, const int *xcol, const double *xval,
                       const int64_t *ptr, int *col, double *val) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    const int64_t s = xptr[i];
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        col[k] = xcol[s + (k - ptr[i])];
        val[k] = xval[s + (k - ptr[i])];
    }
}

// ---- per-level scalars and the independent set --------------------------

// d_i and max_i sum_j |a_ij| / a_ii (non-negative doubles order as their bits);
// flags |= 1 when a diagonal is missing, non-positive or not finite
__global__ void k_diag_rho(int n, const int64_t *ptr, const int *col, const double *val, double *d,
                           unsigned long long *rho_bits, int *flags) {
    const int i = blockIdx.x * kT + threadIdx.x;
    unsigned long long rb = 0;   // bits of this row's ratio (0 for no row)
    if (i < n) {
        double di = 0.0, s = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            s += fabs(val[k]);
            if (col[k] == i)
                di = val[k];
        }
        d[i] = di;
        if (!(di > 0.0) || !isfinite(di) || !isfinite(s))
            atomicOr(flags, 1);
        else
            rb = (unsigned long long)__double_as_longlong(s / di);
    }
    // the warp's largest first, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, rb, o);
        rb = t > rb ? t : rb;
    }
    if ((threadIdx.x & 31) == 0 && rb != 0)
        atomicMax(rho_bits, rb);
}

__device__ __forceinline__ bool pair_less(int sa, uint64_t ha, int sb, uint64_t hb) {
    return sa < sb || (sa == sb && ha < hb);
}

// the largest (state, h) over row i and its neighbours
__global__ void k_pair_max(int n, const int64_t *ptr, const int *col, const int *s_in,
                           const uint64_t *h_in, int *s_out, uint64_t *h_out) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    int bs = s_in[i];
    uint64_t bh = h_in[i];
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int j = col[k];
        const int sj = s_in[j];
        const uint64_t hj = h_in[j];
        if (pair_less(bs, bh, sj, hj)) {
            bs = sj;
            bh = hj;
        }
    }
    s_out[i] = bs;
    h_out[i] = bh;
}

__global__ void k_mis_init(int n, int *state, uint64_t *h) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n) {
        state[i] = 1;
        h[i] = prio(i);
    }
}

// one round's decisions; *left counts rows still undecided afterwards
__global__ void k_mis_update(int n, int *state, const uint64_t *h, const int *s2,
                             const uint64_t *h2, unsigned *left) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    if (state[i] != 1)
        return;
    if (s2[i] == 1 && h2[i] == h[i]) {
        state[i] = 2;
    } else if (s2[i] == 2) {
        state[i] = 0;
    } else {
        atomicAdd(left, 1u);
    }
}

__global__ void k_root_flags(int n, const int *state, int64_t *flag) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n)
        flag[i] = state[i] == 2 ? 1 : 0;
}

// roots: their number; other rows: the root they are next to, else -1
__global__ void k_agg_roots(int n, const int64_t *ptr, const int *col, const int *state,
                            const int64_t *rank, int *first) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    if (state[i] == 2) {
        first[i] = (int)rank[i];
        return;
    }
    int a = -1;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int j = col[k];
        if (j != i && state[j] == 2)
            a = (int)rank[j];
    }
    first[i] = a;
}

// rows not yet assigned: the assigned neighbour of largest |a_ij|, ties
// within TIE of the row's largest |a_ij| going to the lower aggregate;
// flags |= 2 when a row has no assigned neighbour
__global__ void k_agg_rest(int n, const int64_t *ptr, const int *col, const double *val,
                           const int *first, int *agg, double tie, int *flags) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    if (first[i] >= 0) {
        agg[i] = first[i];
        return;
    }
    double mx = 0.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
        if (col[k] != i)
            mx = fmax(mx, fabs(val[k]));
    const double tol = tie * mx;
    int best = -1;
    double best_v = -1.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int j = col[k];
        if (j == i || first[j] < 0)
            continue;
        const double a = fabs(val[k]);
        if (best < 0 || a > best_v + tol) {
            best = first[j];
            best_v = a;
        } else if (a >= best_v - tol && first[j] < best) {
            best = first[j];
            best_v = fmax(a, best_v);
        }
    }
    if (best < 0)
        atomicOr(flags, 2);
    agg[i] = best < 0 ? 0 : best;
}

// ---- prolongator ----------------------------------------------------------

// expand row i of P: (agg(j), a_ij) for every stored entry of row i of A, in
// A's slot order (the key), into the row's own slots of the expansion
__global__ void k_p_expand(int n, const int64_t *ptr, const int *col, const double *val,
                           const int *agg, int *xcol, double *xval, int64_t *xkey) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        xcol[k] = agg[col[k]];
        xval[k] = val[k];
        xkey[k] = k;
    }
}

// the merged row of D^-1 A P_t into P's values: [J == agg(i)] - w/d_i sum
__global__ void k_p_values(int n, const int64_t *xptr, const int64_t *cnt, int *xcol,
                           double *xval, const int *agg, const double *d, double w) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    const double s = w / d[i];
    const int own = agg[i];
    for (int64_t k = xptr[i]; k < xptr[i] + cnt[i]; ++k)
        xval[k] = (xcol[k] == own ? 1.0 : 0.0) - s * xval[k];
}

// ---- transpose --------------------------------------------------------------

__global__ void k_col_count(int64_t nnz, const int *col, int64_t *len) {
    const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (k < nnz)
        atomicAdd((unsigned long long *)&len[col[k]], 1ull);
}

__global__ void k_transpose_fill(int n, const int64_t *ptr, const int *col, const double *val,
                                 int64_t *cur, int *tcol, double *tval, int64_t *tkey) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int64_t at = (int64_t)atomicAdd((unsigned long long *)&cur[col[k]], 1ull);
        tcol[at] = i;
        tval[at] = val[k];
        tkey[at] = 0;
    }
}

__global__ void k_copy_i64(int64_t n, const int64_t *a, int64_t *b) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n)
        b[i] = a[i];
}

// ---- sparse product C = X Y (structural pattern, fixed summation order) ----

// upper bound of row i's entries: sum over X's row of the lengths of Y's rows
__global__ void k_gemm_bound(int n, const int64_t *xp, const int *xc, const int64_t *yp,
                             int64_t *ub) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    int64_t t = 0;
    for (int64_t k = xp[i]; k < xp[i + 1]; ++k)
        t += yp[xc[k] + 1] - yp[xc[k]];
    ub[i] = t;
}

// table size of row i: the smallest power of two above the row's possible
// distinct columns, at most min(ub, m) with m the columns of the product
// (0 for an empty row), so that a probe always finds a free slot
__global__ void k_gemm_tsize(int n, const int64_t *ub, int64_t m, int64_t *ts) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    const int64_t d = ub[i] < m ? ub[i] : m;
    int64_t s = 0;
    if (d > 0) {
        s = 2;
        while (s <= d)
            s <<= 1;
    }
    ts[i] = s;
}

__device__ __forceinline__ uint32_t slot_hash(int c) { return (uint32_t)c * 2654435761u; }

// row i of C: every x_ik y_kj added into the row's own hash table in the
// order (k, j) of the two rows; the occupied slots then sorted by column
// into the front of the table and their number written to cnt[i]
__global__ void k_gemm_rows(int n, const int64_t *xp, const int *xc, const double *xv,
                            const int64_t *yp, const int *yc, const double *yv,
                            const int64_t *ub, const int64_t *tp, int *tcol, double *tval,
                            int64_t *cnt) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    if (ub[i] >= kLongRow)
        return;   // k_gemm_long_rows forms this row
    const int64_t base = tp[i], size = tp[i + 1] - base;
    int *tc = tcol + base;
    double *tv = tval + base;
    for (int64_t s = 0; s < size; ++s)
        tc[s] = -1;
    const uint64_t mask = (uint64_t)size - 1;
    int64_t used = 0;
    for (int64_t k = xp[i]; k < xp[i + 1]; ++k) {
        const int r = xc[k];
        const double a = xv[k];
        for (int64_t q = yp[r]; q < yp[r + 1]; ++q) {
            const int c = yc[q];
            uint64_t h = slot_hash(c) & mask;
            while (tc[h] != -1 && tc[h] != c)
                h = (h + 1) & mask;
            if (tc[h] == -1) {
                tc[h] = c;
                tv[h] = a * yv[q];
                ++used;
            } else {
                tv[h] += a * yv[q];
            }
        }
    }
    // pack the occupied slots to the front, then sort them by column
    int64_t w = 0;
    for (int64_t s = 0; s < size; ++s)
        if (tc[s] != -1) {
            tc[w] = tc[s];
            tv[w] = tv[s];
            ++w;
        }
    sort_entries(tc, nullptr, tv, w);   // columns are distinct
    cnt[i] = used;
}

// ---- long rows: a block per row -----------------------------------------------
//
// Rows with many entries (the transposes and products of the coarse levels:
// thousands of entries in a few thousand rows) take a block of kT threads
// each instead of one thread.


__global__ void k_flag_long(int64_t n, const int64_t *len, int64_t thr, int64_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n)
        flag[i] = len[i] >= thr ? 1 : 0;
}

// list[rank[i]] = i for the flagged rows (rank: the exclusive scan of flag)
__global__ void k_list_long(int64_t n, const int64_t *flag, const int64_t *rank, int *list) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n && flag[i])
        list[rank[i]] = (int)i;
}

// the block's bitonic sort of m <= kSortMax (column, value) pairs with
// distinct columns, in place in global memory, through shared memory
__device__ void block_sort_pairs(int *col, double *val, int m) {
    extern __shared__ __align__(16) unsigned char sort_smem[];
    int *sc = reinterpret_cast<int *>(sort_smem);
    double *sv = reinterpret_cast<double *>(sort_smem + sizeof(int) * kSortMax);
    int p = 1;
    while (p < m)
        p <<= 1;
    for (int t = threadIdx.x; t < p; t += blockDim.x) {
        sc[t] = t < m ? col[t] : INT_MAX;
        sv[t] = t < m ? val[t] : 0.0;
    }
    __syncthreads();
    for (int k = 2; k <= p; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < p; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    if ((sc[t] > sc[u]) == up) {
                        const int c = sc[t];
                        sc[t] = sc[u];
                        sc[u] = c;
                        const double v = sv[t];
                        sv[t] = sv[u];
                        sv[u] = v;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        col[t] = sc[t];
        val[t] = sv[t];
    }
    __syncthreads();
}

// sort the long rows of a CSR (distinct columns) by column, a block per row
__global__ void k_sort_long_rows(const int *list, const int64_t *ptr, int *col, double *val) {
    const int i = list[blockIdx.x];
    const int64_t b = ptr[i], m = ptr[i + 1] - b;
    if (m <= kSortMax) {
        block_sort_pairs(col + b, val + b, (int)m);
    } else if (threadIdx.x == 0) {
        sort_entries(col + b, nullptr, val + b, m);
    }
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double red[kT / 32];
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// Row i of C = X Y for a long row, a block per row.  The products are added
// in parallel, so that the result is the same whatever the order, each one
// is split into two 64-bit fixed-point parts relative to the row's largest
// product (about 90 significant bits in all, more than an FP64 sum keeps)
// and the parts are summed with integer atomics, which are associative.
// The occupied slots are then packed in slot order, converted back to
// double and sorted by column.  hi, lo: the row's fixed-point scratch.
__global__ void k_gemm_long_rows(const int *list, const int64_t *xp, const int *xc, const double *xv,
                                 const int64_t *yp, const int *yc, const double *yv,
                                 const int64_t *ub, const int64_t *tp, const int64_t *lp,
                                 int *tcol, double *tval, long long *fix, int64_t *cnt) {
    const int i = list[blockIdx.x];
    const int64_t base = tp[i], size = tp[i + 1] - base;
    int *tc = tcol + base;
    double *tv = tval + base;
    long long *hi = fix + 2 * lp[blockIdx.x];
    long long *lo = hi + size;
    for (int64_t s2 = threadIdx.x; s2 < size; s2 += blockDim.x) {
        tc[s2] = -1;
        hi[s2] = 0;
        lo[s2] = 0;
    }
    // largest |product| of the row
    double mx = 0.0;
    for (int64_t k = xp[i] + threadIdx.x; k < xp[i + 1]; k += blockDim.x) {
        const double a = fabs(xv[k]);
        const int r = xc[k];
        for (int64_t q = yp[r]; q < yp[r + 1]; ++q)
            mx = fmax(mx, a * fabs(yv[q]));
    }
    mx = block_max(mx);   // ends with a barrier: the table is initialised
    int L = 1;
    while (((int64_t)1 << L) <= ub[i])
        ++L;
    // |p 2^s1| < 2^(61 - L): a sum of ub parts cannot overflow
    const int s1 = mx > 0.0 ? 61 - L - (ilogb(mx) + 1) : 0;
    const int s2s = 61 - L;
    const uint64_t mask = (uint64_t)size - 1;
    for (int64_t k = xp[i] + threadIdx.x; k < xp[i + 1]; k += blockDim.x) {
        const double a = xv[k];
        const int r = xc[k];
        for (int64_t q = yp[r]; q < yp[r + 1]; ++q) {
            const int c = yc[q];
            const double sc = ldexp(a * yv[q], s1);
            const long long hv = (long long)sc;                    // integer part (exact)
            const long long lv = llrint(ldexp(sc - (double)hv, s2s));   // fraction, 61 - L bits
            uint64_t h = slot_hash(c) & mask;
            for (;;) {
                const int t = atomicCAS(tc + h, -1, c);
                if (t == -1 || t == c)
                    break;
                h = (h + 1) & mask;
            }
            atomicAdd(reinterpret_cast<unsigned long long *>(hi + h), (unsigned long long)hv);
            atomicAdd(reinterpret_cast<unsigned long long *>(lo + h), (unsigned long long)lv);
        }
    }
    __syncthreads();
    // pack the occupied slots to the front in slot order, as doubles
    __shared__ int s_total;
    __shared__ int s_warp[kT / 32];
    if (threadIdx.x == 0)
        s_total = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < size; c0 += blockDim.x) {
        const int64_t s3 = c0 + threadIdx.x;
        const bool occ = s3 < size && tc[s3] != -1;
        int cv = 0;
        double vv = 0.0;
        if (occ) {
            cv = tc[s3];
            vv = ldexp((double)hi[s3] + ldexp((double)lo[s3], -s2s), -s1);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, occ);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0)
            s_warp[wid] = __popc(bal);
        __syncthreads();   // every thread has read its slot before any is written
        int off = s_total;
        for (int w = 0; w < wid; ++w)
            off += s_warp[w];
        off += __popc(bal & ((1u << lane) - 1u));
        if (occ) {
            tc[off] = cv;
            tv[off] = vv;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                s_total += s_warp[w];
        __syncthreads();
    }
    const int used = s_total;
    if (used <= kSortMax)
        block_sort_pairs(tc, tv, used);
    else if (threadIdx.x == 0)
        sort_entries(tc, nullptr, tv, used);
    if (threadIdx.x == 0)
        cnt[i] = used;
}

// ---- the level's device layouts --------------------------------------------

__global__ void k_offdiag_len(int n, const int64_t *ptr, const int *col, int64_t *len) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    int64_t t = 0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
        t += col[k] != i;
    len[i] = t;
}

// widest off-diagonal row of each 32-row slice
__global__ void k_slice32_width(int n, const int64_t *len, int64_t *sw) {
    const int s = blockIdx.x * kT + threadIdx.x;
    if (s >= (n + 31) / 32)
        return;
    int64_t w = 0;
    for (int r = s * 32; r < min(n, s * 32 + 32); ++r)
        w = max(w, len[r]);
    sw[s] = w;
}

__global__ void k_slice32_slots(int ns, const int64_t *sw, int64_t *slots) {
    const int s = blockIdx.x * kT + threadIdx.x;
    if (s < ns)
        slots[s] = 32 * sw[s];
}

// A's off-diagonal part in 32-row sliced ELL (padding: column 0, value 0;
// 16-bit offsets: 0, the row itself) and whether every offset fits 16 bits
__global__ void k_sell32_fill(int n, const int64_t *ptr, const int *col, const double *val,
                              const int64_t *sp, const int64_t *sw, int *scol, double *sval,
                              short *c16, int *flags) {
    const int row = blockIdx.x * kT + threadIdx.x;
    if (row >= (n + 31) / 32 * 32)
        return;
    const int s = row >> 5, i = row & 31;
    int k = 0;
    if (row < n)
        for (int64_t e = ptr[row]; e < ptr[row + 1]; ++e) {
            const int c = col[e];
            if (c == row)
                continue;
            const int64_t at = sp[s] + (int64_t)k * 32 + i;
            scol[at] = c;
            sval[at] = val[e];
            const int off = c - row;
            if (off < -32768 || off > 32767)
                atomicOr(flags, 4);
            c16[at] = (short)off;
            ++k;
        }
    for (; k < sw[s]; ++k) {
        const int64_t at = sp[s] + (int64_t)k * 32 + i;
        scol[at] = 0;
        sval[at] = 0.0;
        c16[at] = 0;
    }
}

// A's off-diagonal part in CSR (int32 row pointers)
__global__ void k_offdiag_csr(int n, const int64_t *ptr, const int *col, const double *val,
                              const int64_t *optr, int *oc, double *ov) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n)
        return;
    int64_t w = optr[i];
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
        if (col[k] != i) {
            oc[w] = col[k];
            ov[w] = val[k];
            ++w;
        }
}

__global__ void k_i64_to_i32(int64_t n, const int64_t *a, int *b) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n)
        b[i] = (int)a[i];
}

__global__ void k_d2f(int64_t n, const double *a, float *b) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n)
        b[i] = (float)a[i];
}

__global__ void k_wd(int n, const double *d, double w, double *wd) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n)
        wd[i] = w / d[i];
}

}  // namespace amgs
