// setup.cu -- handle creation: validation of the LDU addressing, repack into
// sliced ELL with symmetric diagonal scaling, value refresh, the standalone
// matrix-vector product and the adjoint face gradient.
//
// Repack (done on the device, every step a plain kernel):
//   1. validate faces, count each row's off-diagonals (degree)
//   2. slice width = widest row of the slice; slot offsets by prefix sum
//   3. scatter every face into both of its rows (atomic cursor per row)
//   4. sort each row's slots by (column, face) so the layout does not depend
//      on the order the atomics ran in
//   5. values: Ahat = a / (sqrt(d_row) sqrt(d_col)), in double and float
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ldupcg_impl.cuh"

using namespace ldu;

namespace ldu {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LDU_OK : (e == cudaErrorMemoryAllocation ? LDU_ERR_OOM : LDU_ERR_CUDA); }

SellView view_of(const ldu_matrix *A) {
    SellView v;
    v.n = (int)A->n;
    v.n_pad = (int)A->n_pad;
    v.n_slices = (int)A->n_slices;
    v.C = A->C;
    v.slice_ptr = A->slice_ptr;
    v.slice_w = A->slice_w;
    v.col = A->col;
    v.col16 = A->col16;
    v.val64 = A->val64;
    v.val32 = A->val32;
    v.sd = A->sd;
    v.isd = A->isd;
    v.dg = A->dg;
    v.meta_smem = 0;   // set by the launcher once the shared memory is sized
    v.meta_cap = 0;
    v.stage_w = 0;
    v.stages = 0;
    return v;
}

// Largest grid of a single-system launch: one block per min_slices slices.
int grid_cap(const ldu_matrix *A) {
    if (A->min_slices <= 0 || A->batch)
        return 1 << 30;
    return (int)std::max<int64_t>(1, std::min<int64_t>(A->n_slices / A->min_slices, 1 << 30));
}

// Shared memory for the per-block slice metadata: enough for the largest
// block share when the grid has at least `blocks` blocks; 0 (global reads)
// above kMetaSmemMax, so that with the kernels' static shared memory a
// block stays within the default 48 KB.
int meta_smem_bytes(int64_t n_slices, int blocks, size_t *bytes) {
    const int64_t per_block = (n_slices + blocks - 1) / blocks;
    const int64_t b = per_block * (int64_t)sizeof(int2);
    *bytes = b <= kMetaSmemMax ? (size_t)b : 0;
    return LDU_OK;
}

// Grid for a given dynamic shared-memory size (raising the kernel's limit
// above the default 48 KB when needed).
int grid_for_smem(const ldu_matrix *A, const void *kernel, int block, size_t smem, int *grid) {
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (per_sm < 1)
        return LDU_ERR_UNSUPPORTED;
    if (A->blocks_per_sm > 0)
        per_sm = std::min(per_sm, A->blocks_per_sm);
    *grid = std::min(per_sm * A->num_sms, A->max_grid);
    *grid = std::min(*grid, grid_cap(A));
    return LDU_OK;
}

int launch_persistent(const void *kernel, int grid, int block, void **args, size_t smem,
                      cudaStream_t s) {
    cudaError_t e = cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(block), args, smem, s);
    return cuda_status(e);
}

}  // namespace ldu

#include "setup_kernels.cuh"

namespace {

int blocks_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

template <typename T>
cudaError_t dev_alloc(T **p, int64_t count, int64_t *bytes) {
    *p = nullptr;
    size_t sz = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = cudaMalloc((void **)p, sz);
    if (e == cudaSuccess)
        *bytes += (int64_t)sz;
    return e;
}

}  // namespace

namespace ldu {
void free_batch(ldu_matrix *A);   // solve_batched.cu
}

namespace {

void free_handle(ldu_matrix *A) {
    if (!A)
        return;
    ldu::free_batch(A);
    void *ptrs[] = {A->slice_ptr, A->slice_w, A->col, A->col16, A->fid, A->owner, A->neighbour,
                    A->val64, A->sd, A->isd, A->dg, A->sdf, A->val32, A->slots, A->bar_count,
                    A->bar_err, A->out_dev, A->flags_dev, A->row_cell, A->rhs};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    for (double *p : A->v64)
        if (p)
            cudaFree(p);
    for (float *p : A->v32)
        if (p)
            cudaFree(p);
    if (A->out_host)
        cudaFreeHost(A->out_host);
    std::free(A);
}

int values_from_arrays(ldu_matrix *A, const double *diag, const double *up, const double *lo,
                       cudaStream_t st) {
    const int T = 256;
    k_diag_scale<<<blocks_for(A->n_pad, T), T, 0, st>>>((int)A->n, (int)A->n_pad, diag, A->sd,
                                                        A->isd, A->dg, A->sdf, A->flags_dev,
                                                        A->row_cell);
    k_values<<<blocks_for(A->n_pad, T), T, 0, st>>>((int)A->n_pad, A->C, A->slice_ptr, A->slice_w,
                                                    A->col, A->fid, up, lo, nullptr, A->sd,
                                                    A->val64, A->val32);
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

const char *ldu_status_string(int s) {
    switch (s) {
    case LDU_OK: return "ok";
    case LDU_NOT_CONVERGED: return "not converged (iteration cap)";
    case LDU_ERR_BAD_ARG: return "bad argument";
    case LDU_ERR_BAD_ADDRESSING: return "bad LDU addressing (index out of range or owner >= neighbour)";
    case LDU_ERR_NOT_SPD: return "matrix not symmetric positive definite (non-positive diagonal or CG breakdown)";
    case LDU_ERR_CUDA: return "CUDA runtime error";
    case LDU_ERR_BARRIER_TIMEOUT: return "grid barrier timed out";
    case LDU_ERR_OOM: return "out of device memory";
    case LDU_ERR_UNSUPPORTED: return "size not supported by the layout";
    default: return "unknown status";
    }
}

int ldu_create(int64_t n, int64_t nf, const int32_t *owner, const int32_t *neighbour,
               const double *diag, const double *upper, const double *lower, const ldu_opts *opt,
               ldu_stream_t stream, ldu_matrix **out) {
    if (!out)
        return LDU_ERR_BAD_ARG;
    *out = nullptr;
    if (n < 0 || nf < 0 || (n > 0 && !diag) || (nf > 0 && (!owner || !neighbour || !upper || !lower)))
        return LDU_ERR_BAD_ARG;
    int C = 128, bt = 256, bps = 0, stg = 0, msl = kDefaultMinSlices;
    if (opt) {
        if (opt->slice_rows)
            C = opt->slice_rows;
        if (opt->block_threads)
            bt = opt->block_threads;
        bps = opt->blocks_per_sm;
        stg = opt->staging;
        if (opt->min_slices)
            msl = opt->min_slices;
    }
    if ((C != 32 && C != 64 && C != 128) || (bt != 128 && bt != 256) || bps < 0 ||
        (stg != 0 && stg != -1) || msl < -1)
        return LDU_ERR_BAD_ARG;
    if (n >= (int64_t)1 << 31 || nf >= (int64_t)1 << 30)
        return LDU_ERR_UNSUPPORTED;

    cudaStream_t st = (cudaStream_t)stream;
    ldu_matrix *A = (ldu_matrix *)std::calloc(1, sizeof(ldu_matrix));
    if (!A)
        return LDU_ERR_OOM;
    int rc = LDU_OK;
    int *deg = nullptr, *cursor = nullptr;
    int64_t b = 0;
    cudaError_t e;
#define CK(call)                        \
    do {                                \
        e = (call);                     \
        if (e != cudaSuccess) {         \
            rc = cuda_status(e);        \
            goto fail;                  \
        }                               \
    } while (0)

    CK(cudaGetDevice(&A->device));
    CK(cudaDeviceGetAttribute(&A->num_sms, cudaDevAttrMultiProcessorCount, A->device));
    A->n = n;
    A->n_cells = n;
    A->nf = nf;
    A->C = C;
    A->block_threads = bt;
    A->blocks_per_sm = bps;
    A->staging = stg;
    A->min_slices = msl;
    A->n_slices = (n + C - 1) / C;
    A->n_pad = A->n_slices * C;
    A->max_grid = A->num_sms * 32;

    CK(dev_alloc(&A->flags_dev, 4, &b));
    CK(cudaMemsetAsync(A->flags_dev, 0, 4 * sizeof(int), st));
    CK(dev_alloc(&deg, std::max<int64_t>(n, 1), &b));
    CK(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)std::max<int64_t>(n, 1), st));
    if (nf > 0)
        k_validate_count<<<blocks_for(nf, 256), 256, 0, st>>>(nf, (int)n, owner, neighbour, deg,
                                                               A->flags_dev);
    if (n > 0 || nf > 0)
        k_validate_values<<<blocks_for(std::max(n, nf), 256), 256, 0, st>>>(
            n, nf, diag, upper, lower, A->flags_dev);
    CK(cudaGetLastError());
    {
        int flags = 0;
        CK(cudaMemcpyAsync(&flags, A->flags_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (flags & (kFlagBadIndex | kFlagBadOrder)) {
            rc = LDU_ERR_BAD_ADDRESSING;
            goto fail;
        }
        if (flags & (kFlagBadDiag | kFlagNonFinite)) {
            rc = LDU_ERR_NOT_SPD;
            goto fail;
        }
    }
    // slice widths and slot offsets
    CK(dev_alloc(&A->slice_w, std::max<int64_t>(A->n_slices, 1), &b));
    CK(dev_alloc(&A->slice_ptr, A->n_slices + 1, &b));
    if (A->n_slices > 0)
        k_slice_width<<<blocks_for(A->n_slices, 128), 128, 0, st>>>((int)n, (int)A->n_slices, C,
                                                                     deg, A->slice_w);
    CK(cudaGetLastError());
    {
        std::vector<int> w((size_t)A->n_slices), ptr((size_t)A->n_slices + 1);
        if (A->n_slices > 0)
            CK(cudaMemcpyAsync(w.data(), A->slice_w, sizeof(int) * w.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        int64_t acc = 0;
        int maxw = 0;
        for (int64_t s = 0; s < A->n_slices; ++s) {
            ptr[(size_t)s] = (int)acc;
            acc += (int64_t)w[(size_t)s] * C;
            maxw = std::max(maxw, w[(size_t)s]);
            if (acc >= ((int64_t)1 << 31) - C) {
                rc = LDU_ERR_UNSUPPORTED;
                goto fail;
            }
        }
        ptr[(size_t)A->n_slices] = (int)acc;
        A->nnz_pad = acc;
        A->max_w = maxw;
        CK(cudaMemcpyAsync(A->slice_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));   // host vector goes out of scope
    }
    CK(dev_alloc(&A->col, A->nnz_pad, &b));
    CK(dev_alloc(&A->fid, A->nnz_pad, &b));
    CK(dev_alloc(&A->val64, A->nnz_pad, &b));
    CK(dev_alloc(&A->val32, A->nnz_pad, &b));
    CK(dev_alloc(&A->sd, A->n_pad, &b));
    CK(dev_alloc(&A->isd, A->n_pad, &b));
    CK(dev_alloc(&A->dg, A->n_pad, &b));
    CK(dev_alloc(&A->sdf, A->n_pad, &b));
    CK(dev_alloc(&A->owner, nf, &b));
    CK(dev_alloc(&A->neighbour, nf, &b));
    CK(dev_alloc(&cursor, std::max<int64_t>(n, 1), &b));
    CK(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)std::max<int64_t>(n, 1), st));
    if (nf > 0) {
        CK(cudaMemcpyAsync(A->owner, owner, sizeof(int32_t) * (size_t)nf, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(A->neighbour, neighbour, sizeof(int32_t) * (size_t)nf, cudaMemcpyDeviceToDevice, st));
    }
    if (A->n_pad > 0)
        k_fill_pad<<<blocks_for(A->n_pad, 256), 256, 0, st>>>((int)A->n_pad, C, A->slice_ptr,
                                                               A->slice_w, A->col, A->fid);
    if (nf > 0)
        k_scatter_faces<<<blocks_for(nf, 256), 256, 0, st>>>(nf, C, owner, neighbour, A->slice_ptr,
                                                              cursor, A->col, A->fid);
    if (n > 0)
        k_sort_rows<<<blocks_for(n, 128), 128, 0, st>>>((int)n, C, A->slice_ptr, deg, A->col, A->fid);
    CK(cudaGetLastError());
    if (stg == 0 && A->nnz_pad > 0) {
        // 16-bit column offsets for the staged sweeps, kept only if all fit
        CK(dev_alloc(&A->col16, A->nnz_pad, &b));
        k_col16<<<blocks_for(A->n_pad, 256), 256, 0, st>>>((int)A->n_pad, C, A->slice_ptr,
                                                            A->slice_w, A->col, A->col16,
                                                            A->flags_dev + 3);
        CK(cudaGetLastError());
        int overflow = 0;
        CK(cudaMemcpyAsync(&overflow, A->flags_dev + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (overflow) {
            cudaFree(A->col16);
            A->col16 = nullptr;
            b -= (int64_t)sizeof(short) * A->nnz_pad;
        }
    }
    if (A->n_pad > 0) {
        rc = values_from_arrays(A, diag, upper, lower, st);
        if (rc != LDU_OK)
            goto fail;
    }
    // work vectors and solver state
    for (int k = 0; k < 10; ++k) {
        CK(dev_alloc(&A->v64[k], A->n_pad, &b));
        CK(cudaMemsetAsync(A->v64[k], 0, sizeof(double) * (size_t)std::max<int64_t>(A->n_pad, 1), st));
    }
    for (int k = 0; k < 10; ++k) {
        CK(dev_alloc(&A->v32[k], A->n_pad, &b));
        CK(cudaMemsetAsync(A->v32[k], 0, sizeof(float) * (size_t)std::max<int64_t>(A->n_pad, 1), st));
    }
    CK(dev_alloc(&A->slots, (int64_t)2 * A->max_grid * kNumDots, &b));
    CK(dev_alloc(&A->bar_count, 64, &b));
    CK(dev_alloc(&A->bar_err, 64, &b));
    CK(dev_alloc(&A->out_dev, 1, &b));
    CK(cudaMallocHost((void **)&A->out_host, sizeof(SolveOut)));
    std::memset(A->out_host, 0, sizeof(SolveOut));
    CK(cudaStreamSynchronize(st));
    cudaFree(deg);
    cudaFree(cursor);
    deg = cursor = nullptr;
    b -= (int64_t)sizeof(int) * 2 * std::max<int64_t>(n, 1);
    A->device_bytes = b;
    A->last.status = LDU_OK;
    *out = A;
    return LDU_OK;
fail:
    cudaStreamSynchronize(st);
    if (deg)
        cudaFree(deg);
    if (cursor)
        cudaFree(cursor);
    free_handle(A);
    return rc;
#undef CK
}

void ldu_destroy(ldu_matrix *A) {
    if (!A)
        return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != A->device)
        cudaSetDevice(A->device);
    cudaDeviceSynchronize();
    free_handle(A);
    if (cur >= 0 && cur != A->device)
        cudaSetDevice(cur);
}

int ldu_update_values(ldu_matrix *A, const double *diag, const double *upper, const double *lower,
                      ldu_stream_t stream) {
    if (!A || (A->n > 0 && !diag) || (A->nf > 0 && (!upper || !lower)))
        return LDU_ERR_BAD_ARG;
    if (A->n_pad == 0)
        return LDU_OK;
    return values_from_arrays(A, diag, upper, lower, (cudaStream_t)stream);
}

int ldu_set_face_coeffs(ldu_matrix *A, const double *coef, const double *diag_extra,
                        ldu_stream_t stream) {
    if (!A || (A->nf > 0 && !coef) || (A->n > 0 && !diag_extra))
        return LDU_ERR_BAD_ARG;
    if (A->n_pad == 0)
        return LDU_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int T = 256;
    k_diag_from_coef<<<blocks_for(A->n_pad, T), T, 0, st>>>(
        (int)A->n, (int)A->n_pad, A->C, A->slice_ptr, A->slice_w, A->fid, coef, diag_extra, A->sd,
        A->isd, A->dg, A->sdf, A->flags_dev, A->row_cell);
    k_values<<<blocks_for(A->n_pad, T), T, 0, st>>>((int)A->n_pad, A->C, A->slice_ptr, A->slice_w,
                                                    A->col, A->fid, nullptr, nullptr, coef, A->sd,
                                                    A->val64, A->val32);
    return cuda_status(cudaGetLastError());
}

int ldu_spmv(const ldu_matrix *A, int precision, const void *x, void *y, ldu_stream_t stream) {
    if (!A || (A->n > 0 && (!x || !y)))
        return LDU_ERR_BAD_ARG;
    if (A->row_cell)
        return LDU_ERR_UNSUPPORTED;   // batched handles: solves and gradients only
    if (A->n == 0)
        return LDU_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int T = 256;
    if (precision == LDU_FP64) {
        // two passes through a work vector: one FP64 operation per stored entry
        double *u = A->v64[9];
        k_spmv_prescale<double><<<blocks_for(A->n, T), T, 0, st>>>((int)A->n, A->sd,
                                                                   (const double *)x, u);
        k_spmv<double, true><<<blocks_for(A->n, T), T, 0, st>>>((int)A->n, A->C, A->slice_ptr,
                                                                A->slice_w, A->col, A->val64, A->sd,
                                                                u, (double *)y);
    } else if (precision == LDU_FP32) {
        k_spmv<float, false><<<blocks_for(A->n, T), T, 0, st>>>((int)A->n, A->C, A->slice_ptr,
                                                                A->slice_w, A->col, A->val32, A->sdf,
                                                                (const float *)x, (float *)y);
    }
    else
        return LDU_ERR_BAD_ARG;
    return cuda_status(cudaGetLastError());
}

int ldu_face_grad(const ldu_matrix *A, const double *lambda, const double *x, double *dcoef,
                  ldu_stream_t stream) {
    if (!A || (A->nf > 0 && (!lambda || !x || !dcoef)))
        return LDU_ERR_BAD_ARG;
    if (A->nf == 0)
        return LDU_OK;
    k_face_grad<<<blocks_for(A->nf, 256), 256, 0, (cudaStream_t)stream>>>(A->nf, A->owner,
                                                                          A->neighbour, lambda, x,
                                                                          dcoef);
    return cuda_status(cudaGetLastError());
}

int ldu_value_grad(const ldu_matrix *A, const double *lambda, const double *x, double *dupper,
                   double *dlower, ldu_stream_t stream) {
    if (!A || (A->nf > 0 && (!lambda || !x || !dupper || !dlower)))
        return LDU_ERR_BAD_ARG;
    if (A->nf == 0)
        return LDU_OK;
    k_value_grad<<<blocks_for(A->nf, 256), 256, 0, (cudaStream_t)stream>>>(
        A->nf, A->owner, A->neighbour, lambda, x, dupper, dlower);
    return cuda_status(cudaGetLastError());
}

int ldu_harmonic_coeffs(const ldu_matrix *A, const double *k, const double *g,
                        const double *bfac, double *coef, double *diag_extra,
                        ldu_stream_t stream) {
    if (!A || (A->n_cells > 0 && (!k || !bfac || !diag_extra)) ||
        (A->nf > 0 && (!g || !coef)))
        return LDU_ERR_BAD_ARG;
    if (A->nf == 0 && A->n_cells == 0)
        return LDU_OK;
    k_harmonic_coeffs<<<blocks_for(std::max(A->nf, A->n_cells), 256), 256, 0,
                        (cudaStream_t)stream>>>(A->nf, A->n_cells, A->owner, A->neighbour, k, g,
                                                bfac, coef, diag_extra);
    return cuda_status(cudaGetLastError());
}

int ldu_harmonic_grad(const ldu_matrix *A, const double *k, const double *g, const double *bfac,
                      const double *dcoef, const double *ddiag_extra, double *dk,
                      ldu_stream_t stream) {
    if (!A || (A->n_cells > 0 && (!k || !bfac || !ddiag_extra || !dk)) ||
        (A->nf > 0 && (!g || !dcoef)))
        return LDU_ERR_BAD_ARG;
    if (A->n_pad == 0)
        return LDU_OK;
    k_harmonic_grad<<<blocks_for(A->n_pad, 256), 256, 0, (cudaStream_t)stream>>>(
        (int)A->n_pad, (int)A->n, A->C, A->slice_ptr, A->slice_w, A->col, A->fid, A->row_cell, k,
        g, bfac, dcoef, ddiag_extra, dk);
    return cuda_status(cudaGetLastError());
}

int ldu_diag_grad(const ldu_matrix *A, const double *lambda, const double *x, double *ddiag,
                  ldu_stream_t stream) {
    if (!A || (A->n_cells > 0 && (!lambda || !x || !ddiag)))
        return LDU_ERR_BAD_ARG;
    if (A->n_cells == 0)
        return LDU_OK;
    k_diag_grad<<<blocks_for(A->n_cells, 256), 256, 0, (cudaStream_t)stream>>>(A->n_cells, lambda,
                                                                             x, ddiag);
    return cuda_status(cudaGetLastError());
}

int ldu_last_stats(const ldu_matrix *A, ldu_solve_stats *stats) {
    if (!A || !stats)
        return LDU_ERR_BAD_ARG;
    *stats = A->last;
    return LDU_OK;
}

int ldu_get_info(const ldu_matrix *A, ldu_info *info) {
    if (!A || !info)
        return LDU_ERR_BAD_ARG;
    info->n = A->n;
    info->n_faces = A->nf;
    info->n_padded = A->n_pad;
    info->nnz_padded = A->nnz_pad;
    info->slice_rows = A->C;
    info->n_slices = A->n_slices;
    info->max_row_entries = A->max_w;
    info->device_bytes = A->device_bytes;
    info->col16 = A->col16 ? 1 : 0;
    return LDU_OK;
}

}  // extern "C"
