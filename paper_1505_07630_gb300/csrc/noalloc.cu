// noalloc.cu -- pcg_solve_ldu_noalloc: Jacobi-PCG on a small LDU system
// without any device allocation.
//
// Who needs it: a caller whose device memory is owned by another allocator
// (a framework's caching pool that has reserved the GPU, a fixed-budget
// embedded runtime) or that must not take cudaMalloc's implicit device
// synchronisation in a latency-critical loop cannot call ldu_create, which
// allocates the repacked matrix and work vectors.  This entry point takes
// the caller's LDU arrays directly, repacks them and runs the same FP64
// Jacobi-PCG kernel as pcg_solve, with every intermediate array in one
// file-scope __device__ array of fixed size (kScratchBytes, 8,130,816 bytes (7.75 MiB))
// that each GPU loading the library holds until the process exits.
//
// The scratch is shared by all calls on a device and keeps whatever the last
// call left in it; everything a call relies on starting at zero is cleared
// by that call.  Calls whose work overlaps on the GPU (two streams, two
// host threads) race on the scratch.  The scratch's device address is looked
// up once per device, by the first call on it, and kept for the life of the
// process: after a cudaDeviceReset (which unloads the module and frees the
// array) this entry point must not be called again in the same process.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ldupcg_impl.cuh"
#include "setup_kernels.cuh"
#include "solve_kernels.cuh"

using namespace ldu;

namespace {

constexpr int kNoallocC = 128;                       // rows per slice, as pcg_solve's default
constexpr int kNoallocBlock = 256;                   // threads per block, as pcg_solve's default
constexpr int64_t kMaxCells = 32768;                 // e.g. a 32^3 mesh
constexpr int64_t kMaxFaces = 131072;
constexpr int64_t kMaxRows = kMaxCells;              // already a multiple of 128
constexpr int64_t kMaxSlices = kMaxRows / kNoallocC;
constexpr int64_t kMaxSlots = 8 * kMaxRows;          // off-diagonal slots incl. padding
constexpr int64_t kMaxGrid = 8192;                   // reduction slots: blocks of the launch

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// byte offsets of the arrays inside the scratch
constexpr size_t kOffDeg = 0;
constexpr size_t kOffCursor = kOffDeg + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffSliceW = kOffCursor + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffSlicePtr = kOffSliceW + align256(sizeof(int) * kMaxSlices);
constexpr size_t kOffCol = kOffSlicePtr + align256(sizeof(int) * (kMaxSlices + 1));
constexpr size_t kOffFid = kOffCol + align256(sizeof(int) * kMaxSlots);
constexpr size_t kOffVal64 = kOffFid + align256(sizeof(uint32_t) * kMaxSlots);
constexpr size_t kOffVal32 = kOffVal64 + align256(sizeof(double) * kMaxSlots);
constexpr size_t kOffSd = kOffVal32 + align256(sizeof(float) * kMaxSlots);
constexpr size_t kOffIsd = kOffSd + align256(sizeof(double) * kMaxRows);
constexpr size_t kOffDg = kOffIsd + align256(sizeof(double) * kMaxRows);
constexpr size_t kOffVec = kOffDg + align256(sizeof(double) * kMaxRows);   // 5 FP64 vectors
constexpr size_t kOffSlots = kOffVec + 5 * align256(sizeof(double) * kMaxRows);
constexpr size_t kOffWords = kOffSlots + align256(sizeof(double) * 2 * kMaxGrid * kNumDots);
// words (byte offsets): 0 barrier count, 256 barrier error, 512 flags,
// 768 slot total, 1024 SolveOut
constexpr size_t kWordsBytes = 2048;
constexpr size_t kScratchBytes = kOffWords + kWordsBytes;

static_assert(kScratchBytes == 8130816, "the scratch size is stated in ldupcg.h");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// host copy of g_scratch's device address, one per device ordinal
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// One thread: slot offsets from the slice widths; flags an overflow of the
// scratch's slot capacity instead of writing past it.
__global__ void k_noalloc_scan(int n_slices, int C, const int *slice_w, int *slice_ptr,
                               int *flags, int *total) {
    if (blockIdx.x != 0 || threadIdx.x != 0)
        return;
    long long acc = 0;
    for (int s = 0; s < n_slices; ++s) {
        slice_ptr[s] = (int)acc;
        acc += (long long)slice_w[s] * C;
        if (acc > kMaxSlots) {
            atomicOr(flags, kFlagOverflow);
            acc = kMaxSlots;
        }
    }
    slice_ptr[n_slices] = (int)acc;
    *total = (int)acc;
}

int noalloc_blocks(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

}  // namespace

extern "C" int pcg_solve_ldu_noalloc(int64_t n, int64_t nFaces, const int32_t *owner,
                                     const int32_t *neighbour, const double *diag,
                                     const double *upper, const double *lower, const double *b,
                                     double *x, double tol, int maxit, int *iters,
                                     double *relres, ldu_stream_t stream) {
    if (n < 0 || nFaces < 0 || maxit < 0 || !(tol >= 0.0) || (n > 0 && (!diag || !b || !x)) ||
        (nFaces > 0 && (!owner || !neighbour || !upper || !lower)))
        return LDU_ERR_BAD_ARG;
    if (n > kMaxCells || nFaces > kMaxFaces)
        return LDU_ERR_UNSUPPORTED;   // beyond the fixed scratch: use ldu_create + pcg_solve
    if (n == 0) {
        if (iters)
            *iters = 0;
        if (relres)
            *relres = 0.0;
        return LDU_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices)
        return LDU_ERR_UNSUPPORTED;
    unsigned char *base;
    {
        // set-up, once per device, with that device current: the host-side
        // name g_scratch is not a device address, so look the address up
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess)
                return cuda_status(e);
            g_scratch_addr[dev] = (unsigned char *)p;
        }
        base = g_scratch_addr[dev];
    }
    int *deg = (int *)(base + kOffDeg);
    int *cursor = (int *)(base + kOffCursor);
    int *slice_w = (int *)(base + kOffSliceW);
    int *slice_ptr = (int *)(base + kOffSlicePtr);
    int *col = (int *)(base + kOffCol);
    uint32_t *fid = (uint32_t *)(base + kOffFid);
    double *val64 = (double *)(base + kOffVal64);
    float *val32 = (float *)(base + kOffVal32);
    double *sd = (double *)(base + kOffSd);
    double *isd = (double *)(base + kOffIsd);
    double *dg = (double *)(base + kOffDg);
    double *slots = (double *)(base + kOffSlots);
    unsigned char *words = base + kOffWords;
    unsigned *bar_count = (unsigned *)(words + 0);
    int *bar_err = (int *)(words + 256);
    int *flags = (int *)(words + 512);
    int *total = (int *)(words + 768);
    SolveOut *out = (SolveOut *)(words + 1024);

    const int C = kNoallocC;
    const int64_t n_slices = (n + C - 1) / C;
    const int64_t n_pad = n_slices * C;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_status(e);

    // what must start at zero: degree counts, scatter cursors, flags, barrier words
#define CK(call)                                  \
    do {                                          \
        if ((e = (call)) != cudaSuccess)          \
            return cuda_status(e);                \
    } while (0)
    CK(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)n, st));
    CK(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)n, st));
    CK(cudaMemsetAsync(words, 0, kWordsBytes, st));
    // the result block reads as "no result" (status -1) until the kernel
    // writes it, so a launch that ends without writing it is an error
    CK(cudaMemsetAsync(out, 0xff, sizeof(SolveOut), st));

    if (nFaces > 0)
        k_validate_count<<<noalloc_blocks(nFaces, 256), 256, 0, st>>>(nFaces, (int)n, owner,
                                                                      neighbour, deg, flags);
    k_validate_values<<<noalloc_blocks(std::max(n, nFaces), 256), 256, 0, st>>>(
        n, nFaces, diag, upper, lower, flags);
    k_slice_width<<<noalloc_blocks(n_slices, 128), 128, 0, st>>>((int)n, (int)n_slices, C, deg,
                                                                  slice_w);
    k_noalloc_scan<<<1, 1, 0, st>>>((int)n_slices, C, slice_w, slice_ptr, flags, total);
    CK(cudaGetLastError());
    int host_flags = 0;
    CK(cudaMemcpyAsync(&host_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (host_flags & (kFlagBadIndex | kFlagBadOrder))
        return LDU_ERR_BAD_ADDRESSING;
    if (host_flags & (kFlagBadDiag | kFlagNonFinite))
        return LDU_ERR_NOT_SPD;
    if (host_flags & kFlagOverflow)
        return LDU_ERR_UNSUPPORTED;   // rows too long for the scratch's slot capacity

    k_fill_pad<<<noalloc_blocks(n_pad, 256), 256, 0, st>>>((int)n_pad, C, slice_ptr, slice_w, col,
                                                            fid);
    if (nFaces > 0)
        k_scatter_faces<<<noalloc_blocks(nFaces, 256), 256, 0, st>>>(nFaces, C, owner, neighbour,
                                                                     slice_ptr, cursor, col, fid);
    k_sort_rows<<<noalloc_blocks(n, 128), 128, 0, st>>>((int)n, C, slice_ptr, deg, col, fid);
    k_diag_scale<<<noalloc_blocks(n_pad, 256), 256, 0, st>>>((int)n, (int)n_pad, diag, sd, isd, dg,
                                                              nullptr, flags, nullptr);
    k_values<<<noalloc_blocks(n_pad, 256), 256, 0, st>>>((int)n_pad, C, slice_ptr, slice_w, col,
                                                         fid, upper, lower, nullptr, sd, val64,
                                                         val32);
    CK(cudaGetLastError());

    const void *kern = (const void *)k_pcg64<4, Batch<4>::pcg>;   // pcg_solve's kernel for C = 128
    // the launch shape of a default handle: at most one block per
    // kDefaultMinSlices slices, metadata sized for the resulting share
    const int64_t cap = std::max<int64_t>(1, n_slices / kDefaultMinSlices);
    size_t smem = 0;
    meta_smem_bytes(n_slices, (int)std::min<int64_t>(sms, cap), &smem);
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNoallocBlock, smem));
    if (per_sm < 1)
        return LDU_ERR_UNSUPPORTED;
    const int grid =
        (int)std::min<int64_t>({(int64_t)per_sm * sms, (int64_t)sms * 32, kMaxGrid, cap});

    SolveParams P;
    P.A.n = (int)n;
    P.A.n_pad = (int)n_pad;
    P.A.n_slices = (int)n_slices;
    P.A.C = C;
    P.A.slice_ptr = slice_ptr;
    P.A.slice_w = slice_w;
    P.A.col = col;
    P.A.col16 = nullptr;
    P.A.val64 = val64;
    P.A.val32 = val32;
    P.A.sd = sd;
    P.A.isd = isd;
    P.A.dg = dg;
    P.A.meta_smem = smem > 0;
    P.A.meta_cap = (int)(smem / sizeof(int2));
    P.A.stage_w = 0;
    P.A.stages = 0;
    P.sync.count = bar_count;
    P.sync.err = bar_err;
    P.sync.timeout_ns = 10ull * 1000000000ull;
    P.slots = slots;
    P.tasks = nullptr;
    P.out = out;
    P.b = b;
    P.x = x;
    for (int k = 0; k < 10; ++k)
        P.v64[k] = k < 5 ? (double *)(base + kOffVec + (size_t)k * align256(sizeof(double) * kMaxRows))
                         : nullptr;
    for (int k = 0; k < 10; ++k)
        P.v32[k] = nullptr;
    P.tol = tol;
    P.maxit = maxit;
    P.rr_period = 0;
    P.tau = 0.0;
    P.restart = 0;
    P.deflate = 0;
    P.fault_inject = 0;
    void *args[] = {&P};
    CK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kNoallocBlock), args, smem, st));
    SolveOut h{};
    int h_err = 0, h_flags = 0;
    CK(cudaMemcpyAsync(&h, out, sizeof(SolveOut), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h_err, bar_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
#undef CK
    if (h_err == kDevTimeout)
        return LDU_ERR_BARRIER_TIMEOUT;
    if (h_flags & (kFlagBadDiag | kFlagNonFinite))
        return LDU_ERR_NOT_SPD;
    int status;
    switch (h.status) {
    case kDevOk: status = LDU_OK; break;
    case kDevNotConverged: status = LDU_NOT_CONVERGED; break;
    case kDevNotSpd: status = LDU_ERR_NOT_SPD; break;
    default: status = LDU_ERR_CUDA; break;
    }
    if (iters)
        *iters = h.iters;
    if (relres)
        *relres = h.relres;
    return status;
}
