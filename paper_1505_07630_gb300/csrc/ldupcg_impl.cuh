// ldupcg_impl.cuh -- internal types and device helpers of libldupcg.
//
// Device layout of a handle (all arrays padded to n_pad = n_slices * C rows):
//   sliced ELL (SELL-C, sigma = 1): slice s holds rows [s*C, s*C + C); its
//   width w_s is the longest off-diagonal row in it; entry k of row
//   s*C + i sits at slice_ptr[s] + k*C + i ("column-major in the slice"), so
//   a warp reads C consecutive values per k.  A lane owns R = C/32
//   consecutive rows and reads them with one R-wide vector load.  Padding
//   slots hold col = own row, value 0.
//   Values are stored symmetrically scaled, Ahat = D^-1/2 A D^-1/2 (unit
//   diagonal, not stored), in double (val64) and float (val32), sharing one
//   int32 column array.  sd = sqrt(diag), isd = 1/sd, dg = diag (double).
//   fid[] maps each slot to its face (bit 31 set when the slot is the
//   face's lower coefficient), so values can be refreshed without a repack.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ldupcg.h"

namespace ldu {

constexpr int kWarp = 32;
constexpr int kNumDots = 4;            // doubles per block in a reduction slot
constexpr unsigned kFullMask = 0xffffffffu;
constexpr uint32_t kLowerBit = 0x80000000u;
constexpr uint32_t kPadFid = 0xffffffffu;
constexpr int kMetaSmemMax = 32 * 1024;   // dynamic shared memory for slice metadata
constexpr int kDefaultMinSlices = 8;      // ldu_opts.min_slices when 0

// error bits raised by device-side validation
enum : int {
    kFlagBadIndex = 1,
    kFlagBadOrder = 2,
    kFlagBadDiag = 4,
    kFlagNonFinite = 8,
    kFlagOverflow = 16,
};

// device status words written by the persistent kernels
enum : int {
    kDevOk = 0,
    kDevNotConverged = 1,
    kDevNotSpd = 2,
    kDevTimeout = 3,
};

struct SolveOut {
    int status;
    int iters;
    int replacements;
    int pad;
    double relres;
    double bnorm;
};

// Read-only view of the repacked matrix, passed by value to kernels.
struct SellView {
    int n;             // real rows
    int n_pad;         // padded rows
    int n_slices;
    int C;             // rows per slice
    const int *slice_ptr;   // [n_slices + 1], in slots
    const int *slice_w;     // [n_slices]
    const int *col;         // [nnz_pad]
    const short *col16;     // [nnz_pad] column minus row of each slot when every slot
                            // fits in 16 bits (null otherwise); read by staged sweeps
    const double *val64;    // [nnz_pad]
    const float *val32;     // [nnz_pad]
    const double *sd;       // [n_pad]
    const double *isd;      // [n_pad]
    const double *dg;       // [n_pad]
    int meta_smem;          // 1: each block keeps its slices' (offset, width) in shared memory
    int meta_cap;           // slice entries reserved for that metadata in shared memory
    int stage_w;            // > 0: float sweeps stage (col, val32) slices of width <= stage_w
                            // into shared memory with bulk copies; 0: plain global loads
    int stages;             // pipeline depth per warp when staging (2..kMaxStages)
};

// Barrier state shared by the blocks of one persistent launch.
struct GridSync {
    unsigned *count;        // arrivals, reset to 0 before each launch
    int *err;               // first error code raised
    unsigned long long timeout_ns;
};

}  // namespace ldu

// Host-side handle.  Plain struct: every pointer is a device allocation owned
// by the handle unless noted.
struct ldu_matrix {
    int device;
    int num_sms;
    int64_t n, nf, n_pad, nnz_pad, n_slices;
    int64_t n_cells;           // caller's cells (n for a single system; without padding rows for a batch)
    int *row_cell;             // batched handles: caller cell of each row, -1 between systems
    int C;
    int max_w;
    int block_threads;
    int blocks_per_sm;
    int staging;               // 0 auto, -1 off
    int min_slices;            // at most one block per min_slices slices (<= 0: no limit)
    int64_t device_bytes;
    // structure
    int *slice_ptr, *slice_w, *col;
    short *col16;              // 16-bit column offsets (null when some offset does not fit)
    uint32_t *fid;
    int32_t *owner, *neighbour;
    // values
    double *val64, *sd, *isd, *dg;
    float *sdf;                // (float)sd: the scaling factors of the float product
    float *val32;
    // work vectors
    double *v64[10];
    float *v32[10];
    double *slots;          // [2][max_grid][kNumDots]
    int max_grid;
    unsigned *bar_count;
    int *bar_err;
    ldu::SolveOut *out_dev;
    ldu::SolveOut *out_host;   // pinned host
    int *flags_dev;            // validation flags
    double *rhs;               // right-hand side of ldu_heat_steps (allocated on first use)
    ldu_solve_stats last;
    struct ldu_batch *batch;   // systems of a batched handle (NULL otherwise)
};

namespace ldu {

ldu::SellView view_of(const ldu_matrix *A);
int cuda_status(cudaError_t e);
int launch_persistent(const void *kernel, int grid, int block, void **args, size_t smem,
                      cudaStream_t s);
int grid_for_smem(const ldu_matrix *A, const void *kernel, int block, size_t smem, int *grid);
int meta_smem_bytes(int64_t n_slices, int blocks, size_t *bytes);
int grid_cap(const ldu_matrix *A);

// ---------------------------------------------------------------------------
// device helpers

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over `members` blocks of a cooperative launch (all of them, or a
// team that solves one system of a batch).  `epoch` counts the barriers
// this block has passed; arrivals accumulate in one counter that is never
// reset during the launch.  Arrival is a release-add by thread 0 after the
// block's __syncthreads (cumulative over the block's writes); the wait is an
// acquire-load spin, so the block's later reads see every write made before
// any block's arrival.  Every spin is bounded: after timeout_ns the block
// records kDevTimeout and leaves, and every other spinning block sees the
// record within a few polls and leaves too.  Returns false when the launch
// must stop.
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// lead = false: the caller has already passed a __syncthreads after its
// threads' last global writes (a block reduction), so thread 0's release
// covers them without another one.
__device__ __forceinline__ bool team_sync(const GridSync &g, unsigned &epoch, unsigned members,
                                          bool lead = true) {
    __shared__ int s_fail;
    if (lead)
        __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * members;
        red_release_add_u32(g.count, 1u);
        int fail = 0;
        unsigned polls = 0;
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire_u32(g.count) - target) < 0) {
            // every 16 polls: leave at once if any block has already failed
            // (so a failure in one team of a batch does not leave the others
            // waiting out their own time limits one after another)
            if ((++polls & 15u) == 0 && *(volatile int *)g.err != 0) {
                fail = 1;
                break;
            }
            if (global_ns() - t0 > g.timeout_ns) {
                atomicCAS(g.err, 0, kDevTimeout);
                fail = 1;
                break;
            }
        }
        s_fail = fail;
    }
    __syncthreads();
    return s_fail == 0;
}

template <int K>
__device__ __forceinline__ void warp_sum(double (&v)[K]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k)
            v[k] += __shfl_down_sync(kFullMask, v[k], o);
}

// Sum K doubles over the block (fixed order) and store them in slot[0..K).
template <int K>
__device__ __forceinline__ void block_sum_to_slot(double (&v)[K], double *slot) {
    __shared__ double sm[32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    warp_sum<K>(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] = lane < nwarps ? sm[lane][k] : 0.0;
        warp_sum<K>(t);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < K; ++k)
                slot[k] = t[k];
    }
}

// After a barrier: every block sums the per-block slots in the same fixed
// order (thread t takes slots t, t + blockDim, ...; then a fixed tree), so
// all blocks hold bitwise-identical totals.  All slot loads of a thread are
// independent, so the sum costs about one L2 round trip.
struct NoTail {
    template <int K>
    __device__ __forceinline__ void operator()(const double (&)[K]) const {}
};

// tail(totals) runs in thread 0 before the totals are published to the
// block, so that the same barrier also publishes what it decides.
template <int K, typename Tail = NoTail>
__device__ __forceinline__ void grid_total(const double *slots, double (&out)[K], int members,
                                           Tail tail = Tail()) {
    __shared__ double sm[32][K];
    __shared__ double res[K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    double t[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        t[k] = 0.0;
    for (int c = threadIdx.x; c < members; c += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] += __ldcg(slots + (size_t)c * kNumDots + k);
    warp_sum<K>(t);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            sm[warp][k] = t[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] = lane < nwarps ? sm[lane][k] : 0.0;
        warp_sum<K>(t);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                res[k] = t[k];
            tail(res);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
        out[k] = res[k];
}

// ---- float-pair ("double-float") sums ---------------------------------------
// FP64 instructions are scarce on this GPU (a warp-wide FP64 add occupies the
// pipe for on the order of a hundred cycles), so per-iteration reductions
// carry each value as an unevaluated sum hi + lo of two floats, combined
// with Knuth's TwoSum: about 48 significant bits, all in FP32 instructions.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    const float h = s.hi + e;
    return {h, e - (h - s.hi)};
}

__device__ __forceinline__ FF ff_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double ff_value(FF a) { return (double)a.hi + (double)a.lo; }

// Compensated (Kahan) float accumulation: a thread sums its share of a dot
// product in float with a running correction term, so the per-thread sum
// keeps close to double accuracy without FP64 instructions in the sweep.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ FF ff() const { return ff_two_sum(s, -c); }
};

template <int K>
__device__ __forceinline__ void warp_sum_ff(FF (&v)[K]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            FF t;
            t.hi = __shfl_down_sync(kFullMask, v[k].hi, o);
            t.lo = __shfl_down_sync(kFullMask, v[k].lo, o);
            v[k] = ff_add(v[k], t);
        }
}

// Float-pair block sum into slot[0..K) (one float2 per value), fixed order.
template <int K>
__device__ __forceinline__ void block_sum_ff(FF (&v)[K], float2 *slot) {
    __shared__ FF sm[32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    warp_sum_ff<K>(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        FF t[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] = lane < nwarps ? sm[lane][k] : FF{0.0f, 0.0f};
        warp_sum_ff<K>(t);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < K; ++k)
                slot[k] = make_float2(t[k].hi, t[k].lo);
    }
}

// Float-pair grid total after a barrier (same fixed order in every block).
template <int K, typename Tail = NoTail>
__device__ __forceinline__ void grid_total_ff(const float2 *slots, double (&out)[K], int members,
                                              Tail tail = Tail()) {
    __shared__ FF sm[32][K];
    __shared__ double res[K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    FF t[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        t[k] = FF{0.0f, 0.0f};
    for (int c = threadIdx.x; c < members; c += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 v = __ldcg(slots + (size_t)c * kNumDots + k);
            t[k] = ff_add(t[k], FF{v.x, v.y});
        }
    warp_sum_ff<K>(t);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            sm[warp][k] = t[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] = lane < nwarps ? sm[lane][k] : FF{0.0f, 0.0f};
        warp_sum_ff<K>(t);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                res[k] = ff_value(t[k]);
            tail(res);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
        out[k] = res[k];
}

// ---- R-wide vector loads / stores of consecutive rows ----------------------

template <typename T, int R>
struct Rows {
    T v[R];
};

template <int R>
__device__ __forceinline__ void ld_rows(const float *p, float (&o)[R]) {
    if constexpr (R == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (R == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else {
        o[0] = *p;
    }
}

template <int R>
__device__ __forceinline__ void st_rows(float *p, const float (&o)[R]) {
    if constexpr (R == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (R == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    } else {
        *p = o[0];
    }
}

template <int R>
__device__ __forceinline__ void ld_rows(const int *p, int (&o)[R]) {
    if constexpr (R == 4) {
        int4 t = *reinterpret_cast<const int4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (R == 2) {
        int2 t = *reinterpret_cast<const int2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else {
        o[0] = *p;
    }
}

template <int R>
__device__ __forceinline__ void ld_rows(const short *p, int (&o)[R]) {
    if constexpr (R == 4) {
        short4 t = *reinterpret_cast<const short4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (R == 2) {
        short2 t = *reinterpret_cast<const short2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else {
        o[0] = *p;
    }
}

template <int R>
__device__ __forceinline__ void ld_rows(const double *p, double (&o)[R]) {
    if constexpr (R >= 2) {
#pragma unroll
        for (int j = 0; j < R; j += 2) {
            double2 t = *reinterpret_cast<const double2 *>(p + j);
            o[j] = t.x;
            o[j + 1] = t.y;
        }
    } else {
        o[0] = *p;
    }
}

template <int R>
__device__ __forceinline__ void st_rows(double *p, const double (&o)[R]) {
    if constexpr (R >= 2) {
#pragma unroll
        for (int j = 0; j < R; j += 2)
            *reinterpret_cast<double2 *>(p + j) = make_double2(o[j], o[j + 1]);
    } else {
        *p = o[0];
    }
}

// streaming (evict-first) loads for the matrix, which is read once per pass
template <int R>
__device__ __forceinline__ void ld_stream(const int *p, int (&o)[R]) {
    if constexpr (R == 4) {
        int4 t = __ldcs(reinterpret_cast<const int4 *>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (R == 2) {
        int2 t = __ldcs(reinterpret_cast<const int2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else {
        o[0] = __ldcs(p);
    }
}

template <int R>
__device__ __forceinline__ void ld_stream(const float *p, float (&o)[R]) {
    if constexpr (R == 4) {
        float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (R == 2) {
        float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else {
        o[0] = __ldcs(p);
    }
}

template <int R>
__device__ __forceinline__ void ld_stream(const double *p, double (&o)[R]) {
    if constexpr (R >= 2) {
#pragma unroll
        for (int j = 0; j < R; j += 2) {
            double2 t = __ldcs(reinterpret_cast<const double2 *>(p + j));
            o[j] = t.x;
            o[j + 1] = t.y;
        }
    } else {
        o[0] = __ldcs(p);
    }
}

template <typename T>
__device__ __forceinline__ const T *vals_of(const SellView &A);
template <>
__device__ __forceinline__ const double *vals_of<double>(const SellView &A) { return A.val64; }
template <>
__device__ __forceinline__ const float *vals_of<float>(const SellView &A) { return A.val32; }

// acc[j] += sum_k Ahat[row0 + j, col] * x[col] over the off-diagonal slots
// of this lane's R rows in the slice described by m = (first slot, width).
// Slots are taken KB at a time: all column and value loads of a batch are
// issued before its gathers.
template <typename T, int R, int KB>
__device__ __forceinline__ void sell_accum(const SellView &A, int2 m, int lane,
                                           const T *__restrict__ x, T (&acc)[R]) {
    const int w = m.y;
    const int C = A.C;
    const int base = m.x + R * lane;
    const T *__restrict__ val = vals_of<T>(A);
    for (int k0 = 0; k0 < w; k0 += KB) {
        int c[KB][R];
        T v[KB][R];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k0 + k < w) {
                ld_stream<R>(A.col + base + (k0 + k) * C, c[k]);
                ld_stream<R>(val + base + (k0 + k) * C, v[k]);
            }
        }
        T g[KB][R];
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int j = 0; j < R; ++j)
                g[k][j] = (k0 + k < w) ? x[c[k][j]] : T(0);
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (k0 + k < w)
                    acc[j] = fma(v[k][j], g[k][j], acc[j]);
    }
}

// Same, for two vectors gathered through the same slots (y1 = Ahat x1,
// y2 = Ahat x2 share one read of the matrix).
template <typename T, int R, int KB>
__device__ __forceinline__ void sell_accum2(const SellView &A, int2 m, int lane,
                                            const T *__restrict__ x1, const T *__restrict__ x2,
                                            T (&acc1)[R], T (&acc2)[R]) {
    const int w = m.y;
    const int C = A.C;
    const int base = m.x + R * lane;
    const T *__restrict__ val = vals_of<T>(A);
    for (int k0 = 0; k0 < w; k0 += KB) {
        int c[KB][R];
        T v[KB][R];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k0 + k < w) {
                ld_stream<R>(A.col + base + (k0 + k) * C, c[k]);
                ld_stream<R>(val + base + (k0 + k) * C, v[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (k0 + k < w) {
                    acc1[j] = fma(v[k][j], x1[c[k][j]], acc1[j]);
                    acc2[j] = fma(v[k][j], x2[c[k][j]], acc2[j]);
                }
    }
}

// acc64 += Ahat64 x64 (double values) and acc32 += Ahat32 x32 (float values)
// through the same slots: one read of the columns serves an FP64 and a float
// product, each accumulated in slot order as sell_accum does.
template <int R, int KB>
__device__ __forceinline__ void sell_accum_df(const SellView &A, int2 m, int lane,
                                              const double *__restrict__ x64,
                                              const float *__restrict__ x32, double (&acc64)[R],
                                              float (&acc32)[R]) {
    const int w = m.y;
    const int C = A.C;
    const int base = m.x + R * lane;
    for (int k0 = 0; k0 < w; k0 += KB) {
        int c[KB][R];
        double v[KB][R];
        float u[KB][R];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k0 + k < w) {
                ld_stream<R>(A.col + base + (k0 + k) * C, c[k]);
                ld_stream<R>(A.val64 + base + (k0 + k) * C, v[k]);
                ld_stream<R>(A.val32 + base + (k0 + k) * C, u[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (k0 + k < w) {
                    acc64[j] = fma(v[k][j], x64[c[k][j]], acc64[j]);
                    acc32[j] = fmaf(u[k][j], x32[c[k][j]], acc32[j]);
                }
    }
}

// Slices of the calling block: a contiguous range, warps interleaved in it.
struct SliceRange {
    int begin, end;
};

__device__ __forceinline__ SliceRange block_slices(int n_slices) {
    const long long b = blockIdx.x, G = gridDim.x;
    SliceRange r;
    r.begin = (int)((b * n_slices) / G);
    r.end = (int)(((b + 1) * n_slices) / G);
    return r;
}

// ---- bulk-copy staging of matrix slices (copy engine + mbarrier) -----------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// An L2 policy that marks lines evict-first: the matrix is read once per
// sweep and must not push the (re-used) vectors out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// An L2 policy that marks lines evict-last: the float vectors of the mixed
// sweep (about 59 MB at 128^3) are read and written every iteration and
// should stay in the 129 MB L2 while the matrix streams past them.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// R consecutive floats with an L2 cache policy (load and store)
template <int R>
__device__ __forceinline__ void ld_rows_pol(const float *p, float (&o)[R], uint64_t pol) {
    if constexpr (R == 4) {
        asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
                     : "l"(p), "l"(pol));
    } else if constexpr (R == 2) {
        asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                     : "=f"(o[0]), "=f"(o[1])
                     : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(o[0]) : "l"(p), "l"(pol));
    }
}

template <int R>
__device__ __forceinline__ void st_rows_pol(float *p, const float (&o)[R], uint64_t pol) {
    if constexpr (R == 4) {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p),
                     "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]), "l"(pol)
                     : "memory");
    } else if constexpr (R == 2) {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(o[0]),
                     "f"(o[1]), "l"(pol)
                     : "memory");
    } else {
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(o[0]), "l"(pol)
                     : "memory");
    }
}

// bytes from global src to shared dst, completing on bar (both 16-byte
// aligned, bytes a multiple of 16), with L2 policy pol
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes to the same buffer
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Dynamic shared memory of the persistent kernels: (first slot, width) of
// each slice the block owns, loaded once per launch, so the sweeps do not
// wait on a global load before every slice's matrix loads.
extern __shared__ __align__(128) int2 ldu_slice_meta[];

__device__ __forceinline__ void load_slice_meta(const SellView &A, const SliceRange &range) {
    if (A.meta_smem) {
        for (int s = range.begin + (int)threadIdx.x; s < range.end; s += blockDim.x)
            ldu_slice_meta[s - range.begin] = make_int2(A.slice_ptr[s], A.slice_w[s]);
        __syncthreads();
    }
}

__device__ __forceinline__ int2 slice_meta(const SellView &A, int s, const SliceRange &range) {
    if (A.meta_smem)
        return ldu_slice_meta[s - range.begin];
    return make_int2(A.slice_ptr[s], A.slice_w[s]);
}

}  // namespace ldu

namespace ldu {

// ---- per-warp pipeline of matrix slices in shared memory -----------------
// Dynamic shared memory: [slice metadata, meta_cap int2, padded to 128 B]
// [stages: nwarps x nst x stage_bytes][mbarriers: nwarps x nst].  A stage
// holds a slice's columns (16-bit offsets, else int32) followed by its float
// values (stage_w x C each).  While a warp works on one slice from shared
// memory, the copy engine brings its next nst - 1 slices, so the DRAM
// latency of the matrix stream leaves the dependency chain; only the
// (mostly L2-resident) gathers remain.  Each sweep consumes exactly the
// copies it issues, so the mbarrier phases stay in step across sweeps.
constexpr int kMaxStages = 2;

struct SlicePipe {
    char *buf;
    uint64_t *bar;
    unsigned stage_bytes;
    unsigned val_off;
    unsigned phase;   // bit k: parity the next wait on stage k expects
    int nst;          // stages per warp
    // the sweep in progress: this warp's k-th slice is first + k * nwarps
    int first, nk, k, cur;
    bool primed;      // the next sweep's first slices are already in flight
};

__host__ __device__ __forceinline__ size_t stage_area_offset(int meta_cap) {
    return ((size_t)meta_cap * sizeof(int2) + 127) & ~(size_t)127;
}

// bytes of one stage: col_bytes per column (2 or 4) plus a float per slot
__host__ __device__ __forceinline__ size_t stage_bytes(int stage_w, int C, int col_bytes) {
    return (size_t)stage_w * C * (size_t)(col_bytes + 4);
}

__host__ __device__ __forceinline__ size_t staged_smem_bytes(int meta_cap, int nwarps, int stage_w,
                                                             int C, int col_bytes, int nst) {
    return stage_area_offset(meta_cap) + (size_t)nwarps * nst * stage_bytes(stage_w, C, col_bytes) +
           (size_t)nwarps * nst * sizeof(uint64_t);
}

__device__ __forceinline__ SlicePipe pipe_open(const SellView &A, int warp, int nwarps, int lane) {
    char *base = reinterpret_cast<char *>(ldu_slice_meta) + stage_area_offset(A.meta_cap);
    const int cb = A.col16 ? 2 : 4;
    SlicePipe pp;
    pp.nst = A.stages;
    pp.stage_bytes = (unsigned)stage_bytes(A.stage_w, A.C, cb);
    pp.val_off = (unsigned)A.stage_w * A.C * (unsigned)cb;
    pp.buf = base + (size_t)warp * pp.nst * pp.stage_bytes;
    pp.bar = reinterpret_cast<uint64_t *>(base + (size_t)nwarps * pp.nst * pp.stage_bytes) +
             pp.nst * warp;
    pp.phase = 0;
    pp.first = pp.nk = pp.k = pp.cur = 0;
    pp.primed = false;
    if (lane == 0) {
        for (int j = 0; j < pp.nst; ++j)
            mbar_init(pp.bar + j, 1);
        mbar_init_fence();
    }
    __syncwarp();
    return pp;
}

// lane 0 asks the copy engine for slice m into stage st: its columns (16-bit
// offsets when the handle has them, else int32) and its float values.  Slot
// offsets are multiples of C >= 32, so every source address, destination
// offset and size is a multiple of 64 bytes.
__device__ __forceinline__ void pipe_issue(const SellView &A, SlicePipe &pp, int st, int2 m,
                                           int lane) {
    if (lane == 0) {
        const unsigned vbytes = (unsigned)m.y * A.C * 4u;
        const unsigned cbytes = A.col16 ? vbytes / 2u : vbytes;
        mbar_expect_tx(pp.bar + st, cbytes + vbytes);
        if (vbytes) {
            char *dst = pp.buf + (size_t)st * pp.stage_bytes;
            const uint64_t pol = l2_evict_first_policy();
            const void *csrc = A.col16 ? (const void *)(A.col16 + m.x) : (const void *)(A.col + m.x);
            bulk_copy_g2s(dst, csrc, cbytes, pp.bar + st, pol);
            bulk_copy_g2s(dst + pp.val_off, A.val32 + m.x, vbytes, pp.bar + st, pol);
        }
    }
}

// every lane waits for stage st (bounded); the warp agrees on the outcome.
// The expected parity advances only on success, so that a drain after a
// timeout waits for the same phase again.
__device__ __forceinline__ bool pipe_wait(SlicePipe &pp, int st, unsigned long long timeout_ns) {
    const unsigned par = (pp.phase >> st) & 1u;
    bool ok = mbar_try_wait(pp.bar + st, par);
    if (!ok) {
        const unsigned long long t0 = global_ns();
        while (!(ok = mbar_try_wait(pp.bar + st, par)))
            if (global_ns() - t0 > timeout_ns)
                break;
    }
    ok = __all_sync(kFullMask, ok);
    if (ok)
        pp.phase ^= (1u << st);
    return ok;
}

// fill the pipeline with the first slices of a sweep over this warp's
// slices of range (every staged sweep visits the same slices in the same
// order, and the matrix does not change during a solve)
__device__ __forceinline__ void pipe_fill(const SellView &A, SlicePipe &pp,
                                         const SliceRange &range, int warp, int nwarps,
                                         int lane) {
    pp.first = range.begin + warp;
    pp.nk = pp.first < range.end ? (range.end - pp.first + nwarps - 1) / nwarps : 0;
    pp.k = 0;
    pp.cur = 0;
    const int fill = pp.nk < pp.nst ? pp.nk : pp.nst;
    for (int j = 0; j < fill; ++j)
        pipe_issue(A, pp, j, slice_meta(A, pp.first + j * nwarps, range), lane);
}

// start a sweep: fill the pipeline unless the end of the previous sweep did
__device__ __forceinline__ void pipe_begin(const SellView &A, SlicePipe &pp,
                                          const SliceRange &range, int warp, int nwarps,
                                          int lane) {
    if (!pp.primed)
        pipe_fill(A, pp, range, warp, nwarps, lane);
    pp.primed = false;
}

// end of a sweep whose slices have all been consumed: start the copies of
// the next sweep's first slices, so that their latency overlaps the grid
// reduction that follows
__device__ __forceinline__ void pipe_prime(const SellView &A, SlicePipe &pp,
                                          const SliceRange &range, int warp, int nwarps,
                                          int lane) {
    pipe_fill(A, pp, range, warp, nwarps, lane);
    pp.primed = true;
}

// wait for the warp's current slice; returns its stage, or null on timeout
__device__ __forceinline__ const char *pipe_front(SlicePipe &pp, unsigned long long timeout_ns) {
    if (!pipe_wait(pp, pp.cur, timeout_ns))
        return nullptr;
    return pp.buf + (size_t)pp.cur * pp.stage_bytes;
}

// the current stage has been read: order those reads before the copy
// engine's next write into it, refill it with slice k + nst, advance
__device__ __forceinline__ void pipe_pop(const SellView &A, SlicePipe &pp, const SliceRange &range,
                                        int nwarps, int lane) {
    fence_proxy_async_smem();
    __syncwarp();
    if (pp.k + pp.nst < pp.nk)
        pipe_issue(A, pp, pp.cur, slice_meta(A, pp.first + (pp.k + pp.nst) * nwarps, range),
                   lane);
    ++pp.k;
    pp.cur = pp.cur + 1 == pp.nst ? 0 : pp.cur + 1;
}

// wait (bounded) for every copy still in flight, so that none lands in
// shared memory after the block has left; the pipeline is empty afterwards
__device__ __forceinline__ void pipe_drain(SlicePipe &pp, unsigned long long timeout_ns) {
    const int left = pp.nk - pp.k;
    const int n = left < pp.nst ? left : pp.nst;
    int st = pp.cur;
    for (int j = 0; j < n; ++j) {
        pipe_wait(pp, st, timeout_ns);
        st = st + 1 == pp.nst ? 0 : st + 1;
    }
    pp.k = pp.nk;
    pp.primed = false;
}

// Drains the pipeline when the solve body returns, on every path.
struct PipeGuard {
    SlicePipe *pp;
    unsigned long long timeout_ns;
    __device__ __forceinline__ ~PipeGuard() {
        if (pp)
            pipe_drain(*pp, timeout_ns);
    }
};

// Column of a staged slot of row `row`, clamped into the padded matrix: one
// unsigned min per gather (about 1 % of the solve), so that no value read
// from shared memory can address outside the vectors.  A correct stage is
// never clamped.
template <typename CT>
__device__ __forceinline__ int staged_col(int c, int row, int n_pad) {
    if constexpr (sizeof(CT) == 2)
        c += row;
    return (int)min((unsigned)c, (unsigned)(n_pad - 1));
}

// acc[j] += sum_k val * x[col] for this lane's R rows, slots taken from a
// staged slice in shared memory (same order of operations as sell_accum);
// KS slots' gathers are in flight per batch.  CT = short: the stage holds
// column minus row, and row0 is the lane's first row.
template <int R, int KS, typename CT>
__device__ __forceinline__ void sell_accum_staged(const char *stage, unsigned val_off, int w, int C,
                                                  int lane, int row0, int n_pad,
                                                  const float *__restrict__ x, float (&acc)[R]) {
    const CT *scol = reinterpret_cast<const CT *>(stage);
    const float *sval = reinterpret_cast<const float *>(stage + val_off);
    for (int k0 = 0; k0 < w; k0 += KS) {
        float g[KS][R];
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (k0 + k < w) {
                int c[R];
                ld_rows<R>(scol + (k0 + k) * C + R * lane, c);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    g[k][j] = x[staged_col<CT>(c[j], row0 + j, n_pad)];
            }
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (k0 + k < w) {
                float v[R];
                ld_rows<R>(sval + (k0 + k) * C + R * lane, v);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    acc[j] = fmaf(v[j], g[k][j], acc[j]);
            }
    }
}

// Same for two vectors through the same staged slots (acc1 += Ahat x1,
// acc2 += Ahat x2), in slot order.
template <int R, int KS, typename CT>
__device__ __forceinline__ void sell_accum2_staged(const char *stage, unsigned val_off, int w, int C,
                                                   int lane, int row0, int n_pad,
                                                   const float *__restrict__ x1,
                                                   const float *__restrict__ x2, float (&acc1)[R],
                                                   float (&acc2)[R]) {
    const CT *scol = reinterpret_cast<const CT *>(stage);
    const float *sval = reinterpret_cast<const float *>(stage + val_off);
    for (int k0 = 0; k0 < w; k0 += KS) {
        float g1[KS][R], g2[KS][R];
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (k0 + k < w) {
                int c[R];
                ld_rows<R>(scol + (k0 + k) * C + R * lane, c);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const int cj = staged_col<CT>(c[j], row0 + j, n_pad);
                    g1[k][j] = x1[cj];
                    g2[k][j] = x2[cj];
                }
            }
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (k0 + k < w) {
                float v[R];
                ld_rows<R>(sval + (k0 + k) * C + R * lane, v);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    acc1[j] = fmaf(v[j], g1[k][j], acc1[j]);
                    acc2[j] = fmaf(v[j], g2[k][j], acc2[j]);
                }
            }
    }
}

}  // namespace ldu
