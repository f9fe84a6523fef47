// solve_batched.cu -- many independent systems solved in one persistent
// cooperative launch.
//
// Layout: the systems are concatenated into one block-diagonal handle, each
// system starting on a slice boundary (rows between systems are padding
// with unit diagonal and no faces), so a slice never straddles two systems.
//
// Schedule: the host splits the launch's blocks into teams.  A system with
// much work gets a team of several blocks (its own barrier counter and
// reduction slots), a small system a single block (barriers are then just
// __syncthreads).  Tasks are placed by longest-processing-time-first list
// scheduling on the blocks' estimated finish times; the tasks are numbered
// in the order they are placed and every block runs its tasks in increasing
// number.  That order rules out deadlock: the lowest-numbered unfinished task
// has every member either at it or done with all earlier tasks, so it always
// completes.  Each team runs the same solver bodies as the single-system
// kernels, scoped to its members.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "ldupcg_impl.cuh"
#include "solve_kernels.cuh"

using namespace ldu;

namespace {

struct SysDev {
    int row0, n, s_begin, s_count;
    long long b_off;
};

struct TaskDev {
    int sys, members, slot_off, pad;
};

struct BatchView {
    const SysDev *sys;
    const TaskDev *tasks;
    const int2 *list;        // (task, rank) entries, per block in increasing task order
    const int *list_begin;   // [grid + 1]
    unsigned *counters;      // 32 per task (one 128-byte line each)
};

__device__ __forceinline__ Scope task_scope(const SolveParams &P, const BatchView &B, int2 tr) {
    const TaskDev t = B.tasks[tr.x];
    const SysDev sy = B.sys[t.sys];
    Scope sc;
    sc.members = t.members;
    sc.rank = tr.y;
    sc.count = B.counters + (size_t)tr.x * 32;
    sc.slots = P.slots + t.slot_off;
    sc.range.begin = sy.s_begin + (int)(((long long)tr.y * sy.s_count) / t.members);
    sc.range.end = sy.s_begin + (int)(((long long)(tr.y + 1) * sy.s_count) / t.members);
    sc.row0 = sy.row0;
    sc.n = sy.n;
    sc.b_off = sy.b_off;
    sc.id = t.sys;
    return sc;
}

template <int R, int KB, bool DEFL, bool STG = false>
__global__ void __launch_bounds__(256, 2) k_mixed_batched(SolveParams P, BatchView B) {
    // one pipeline for all the block's systems: its mbarriers are set up once
    SlicePipe pipe;
    if constexpr (STG)
        pipe = pipe_open(P.A, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x & 31);
    for (int e = B.list_begin[blockIdx.x]; e < B.list_begin[blockIdx.x + 1]; ++e)
        if (!mixed_body<R, KB, DEFL, STG, StagedBatch<R, 2>::ks>(P, task_scope(P, B, B.list[e]),
                                                                  &pipe))
            return;
}

template <int R, int KB>
__global__ void __launch_bounds__(256, 2) k_pcg64_batched(SolveParams P, BatchView B) {
    for (int e = B.list_begin[blockIdx.x]; e < B.list_begin[blockIdx.x + 1]; ++e)
        if (!pcg64_body<R, KB>(P, task_scope(P, B, B.list[e])))
            return;
}

// combined addressing: local face indices + the system's first row; checks
// each face stays inside its system
__global__ void k_batch_faces(int64_t nf, int nsys, const int64_t *f_off, const int64_t *row0,
                              const int64_t *n, const int32_t *own, const int32_t *nbr,
                              int32_t *own_c, int32_t *nbr_c, int *flags) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsys - 1;   // last system with f_off <= f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (f_off[mid] <= f)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int o = own[f], nb = nbr[f];
        if (o < 0 || nb < 0 || o >= n[lo] || nb >= n[lo])
            atomicOr(flags, kFlagBadIndex);
        else if (o >= nb)
            atomicOr(flags, kFlagBadOrder);
        own_c[f] = (int32_t)(o + row0[lo]);
        nbr_c[f] = (int32_t)(nb + row0[lo]);
    }
}

// after the repack: the handle keeps face addressing and a row map in the
// caller's cell numbering (system offset + local index), for the value
// setters and the gradients
__global__ void k_batch_remap(int64_t nf, int nsys, const int64_t *f_off, const int64_t *b_off,
                              const int32_t *own, const int32_t *nbr, int32_t *own_h,
                              int32_t *nbr_h) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (f_off[mid] <= f)
                lo = mid;
            else
                hi = mid - 1;
        }
        own_h[f] = (int32_t)(own[f] + b_off[lo]);
        nbr_h[f] = (int32_t)(nbr[f] + b_off[lo]);
    }
}

__global__ void k_batch_rowmap(int64_t rows, int nsys, const int64_t *row0, const int64_t *n,
                               const int64_t *b_off, int *row_cell) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row0[mid] <= r)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t i = r - row0[lo];
        row_cell[r] = i < n[lo] ? (int)(b_off[lo] + i) : -1;
    }
}

__global__ void k_batch_diag(int64_t rows, int nsys, const int64_t *row0, const int64_t *n,
                             const int64_t *b_off, const double *diag, double *diag_c) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row0[mid] <= r)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t i = r - row0[lo];
        diag_c[r] = i < n[lo] ? diag[b_off[lo] + i] : 1.0;
    }
}

int blocks_of(int64_t work, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 1 << 20));
}

template <int R>
struct BatchKernels {
    static const void *mixed(bool defl) {
        return defl ? (const void *)k_mixed_batched<R, Batch<R>::mixed, true>
                    : (const void *)k_mixed_batched<R, Batch<R>::mixed, false>;
    }
    static const void *mixed_staged() {
        return (const void *)k_mixed_batched<R, Batch<R>::mixed, false, true>;
    }
    static const void *pcg() { return (const void *)k_pcg64_batched<R, Batch<R>::pcg>; }
};

const void *batch_kernel(int C, int precision, bool defl) {
    if (precision == LDU_FP64)
        return C == 32 ? BatchKernels<1>::pcg() : (C == 64 ? BatchKernels<2>::pcg() : BatchKernels<4>::pcg());
    return C == 32 ? BatchKernels<1>::mixed(defl)
                   : (C == 64 ? BatchKernels<2>::mixed(defl) : BatchKernels<4>::mixed(defl));
}

// the mixed kernel whose float sweeps stage the matrix in shared memory
const void *batch_kernel_staged(int C) {
    return C == 32 ? BatchKernels<1>::mixed_staged()
                   : (C == 64 ? BatchKernels<2>::mixed_staged() : BatchKernels<4>::mixed_staged());
}

// dynamic shared memory of the staged kernel for meta_bytes of slice metadata
size_t batch_staged_smem(const ldu_matrix *A, size_t meta_bytes) {
    return staged_smem_bytes((int)(meta_bytes / sizeof(int2)), A->block_threads / 32, A->max_w,
                             A->C, A->col16 ? 2 : 4, 2);
}

}  // namespace

struct ldu_batch {
    int nsys;
    std::vector<int64_t> n, nf, row0, b_off, s_begin, s_count;
    SysDev *sys_dev;
    TaskDev *tasks_dev;
    int2 *list_dev;
    int *list_begin_dev;
    unsigned *counters_dev;
    double *slots_dev;
    SolveOut *out_dev;
    SolveOut *out_host;   // pinned
    int ntasks;
    int grid;
    size_t smem;
    bool staged;      // the mixed solve may use the staged kernel
    int max_team_used;
    batch_opts opts;
};

namespace ldu {

void free_batch(ldu_matrix *A) {
    if (!A || !A->batch)
        return;
    ldu_batch *B = A->batch;
    void *ptrs[] = {B->sys_dev, B->tasks_dev, B->list_dev, B->list_begin_dev, B->counters_dev,
                    B->slots_dev, B->out_dev};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (B->out_host)
        cudaFreeHost(B->out_host);
    delete B;
    A->batch = nullptr;
}

}  // namespace ldu

namespace {

// Longest-processing-time-first list schedule of the systems on G blocks.
// Work of a system: cells x estimated iterations (proportional to the cube
// root of the cell count, as for a 3-D Laplacian); a team of m blocks takes
// work/m plus a per-iteration barrier cost.
int build_schedule(ldu_matrix *A, ldu_batch *Bt, const batch_opts &o, cudaStream_t st) {
    const int G = Bt->grid;
    const int nsys = Bt->nsys;
    const int max_team = std::max(1, std::min(o.max_team > 0 ? o.max_team : 32, G));
    const double scale = o.team_work_scale > 0.0 ? o.team_work_scale : 1.0;
    std::vector<double> iters(nsys), work(nsys);
    double total = 0.0;
    for (int k = 0; k < nsys; ++k) {
        iters[k] = std::max(8.0, 8.0 * std::cbrt((double)std::max<int64_t>(Bt->n[k], 1)));
        work[k] = iters[k] * (double)std::max<int64_t>(Bt->n[k], 1);
        total += work[k];
    }
    // per-iteration cost of a barrier, in cell-iterations of one block
    const double lat1 = 2000.0, latm = 5000.0;
    const double per_block = total / G * scale;
    std::vector<int> members(nsys);
    for (int k = 0; k < nsys; ++k) {
        int m = (int)std::ceil(work[k] / per_block);
        m = std::max(1, std::min({m, max_team, (int)std::max<int64_t>(Bt->s_count[k], 1)}));
        members[k] = m;
    }
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int k) {
        return work[k] / members[k] + iters[k] * (members[k] > 1 ? latm : lat1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<double> load(G, 0.0);
    std::vector<std::vector<int2>> lists(G);
    std::vector<TaskDev> tasks;
    int slot_off = 0;
    size_t max_share = 0;
    std::vector<int> idx(G);
    for (int k : order) {
        const int m = members[k];
        std::iota(idx.begin(), idx.end(), 0);
        std::partial_sort(idx.begin(), idx.begin() + m, idx.end(),
                          [&](int a, int b) { return load[a] < load[b] || (load[a] == load[b] && a < b); });
        std::sort(idx.begin(), idx.begin() + m);
        double start = 0.0;
        for (int j = 0; j < m; ++j)
            start = std::max(start, load[idx[j]]);
        const double end = start + cost(k);
        const int t = (int)tasks.size();
        tasks.push_back(TaskDev{k, m, slot_off, 0});
        slot_off += 2 * m * kNumDots;
        for (int j = 0; j < m; ++j) {
            load[idx[j]] = end;
            lists[idx[j]].push_back(make_int2(t, j));
        }
        const int64_t share = (Bt->s_count[k] + m - 1) / m;
        max_share = std::max(max_share, (size_t)share);
    }
    std::vector<int> begin(G + 1, 0);
    std::vector<int2> flat;
    for (int g = 0; g < G; ++g) {
        begin[g] = (int)flat.size();
        flat.insert(flat.end(), lists[g].begin(), lists[g].end());
    }
    begin[G] = (int)flat.size();
    // device tables
    void *ptrs[] = {Bt->tasks_dev, Bt->list_dev, Bt->list_begin_dev, Bt->counters_dev, Bt->slots_dev};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    Bt->tasks_dev = nullptr;
    Bt->list_dev = nullptr;
    Bt->list_begin_dev = nullptr;
    Bt->counters_dev = nullptr;
    Bt->slots_dev = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc((void **)&Bt->tasks_dev, sizeof(TaskDev) * tasks.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&Bt->list_dev, sizeof(int2) * std::max<size_t>(flat.size(), 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&Bt->list_begin_dev, sizeof(int) * begin.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&Bt->counters_dev, sizeof(unsigned) * 32 * tasks.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&Bt->slots_dev, sizeof(double) * std::max(slot_off, 1))) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(Bt->tasks_dev, tasks.data(), sizeof(TaskDev) * tasks.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(Bt->list_dev, flat.data(), sizeof(int2) * flat.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(Bt->list_begin_dev, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_status(e);
    Bt->ntasks = (int)tasks.size();
    Bt->smem = max_share * sizeof(int2) <= (size_t)kMetaSmemMax ? max_share * sizeof(int2) : 0;
    Bt->max_team_used = *std::max_element(members.begin(), members.end());
    Bt->opts = o;
    (void)A;
    return LDU_OK;
}

}  // namespace

extern "C" {

int ldu_create_batched(int nsys, const int64_t *n, const int64_t *nFaces, const int32_t *owner,
                       const int32_t *neighbour, const double *diag, const double *upper,
                       const double *lower, const ldu_opts *opt, ldu_stream_t stream,
                       ldu_matrix **out) {
    if (!out || nsys <= 0 || !n || !nFaces)
        return LDU_ERR_BAD_ARG;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    int C = opt && opt->slice_rows ? opt->slice_rows : 128;
    if (C != 32 && C != 64 && C != 128)
        return LDU_ERR_BAD_ARG;
    ldu_batch *Bt = new ldu_batch();
    Bt->nsys = nsys;
    int64_t rows = 0, faces = 0, cells = 0;
    std::vector<int64_t> f_off(nsys);
    for (int k = 0; k < nsys; ++k) {
        if (n[k] < 0 || nFaces[k] < 0) {
            delete Bt;
            return LDU_ERR_BAD_ARG;
        }
        Bt->n.push_back(n[k]);
        Bt->nf.push_back(nFaces[k]);
        Bt->row0.push_back(rows);
        Bt->b_off.push_back(cells);
        Bt->s_begin.push_back(rows / C);
        const int64_t sl = (n[k] + C - 1) / C;
        Bt->s_count.push_back(sl);
        f_off[k] = faces;
        rows += sl * C;
        faces += nFaces[k];
        cells += n[k];
    }
    if (cells > 0 && !diag) {
        delete Bt;
        return LDU_ERR_BAD_ARG;
    }
    if (faces > 0 && (!owner || !neighbour || !upper || !lower)) {
        delete Bt;
        return LDU_ERR_BAD_ARG;
    }
    if (rows >= ((int64_t)1 << 31) || faces >= ((int64_t)1 << 30)) {
        delete Bt;
        return LDU_ERR_UNSUPPORTED;
    }
    int rc = LDU_OK;
    int32_t *own_c = nullptr, *nbr_c = nullptr;
    double *diag_c = nullptr;
    int64_t *tab = nullptr;
    int *flags = nullptr;
    ldu_matrix *A = nullptr;
    cudaError_t e;
#define CKB(call)                       \
    do {                                \
        if ((e = (call)) != cudaSuccess) { \
            rc = cuda_status(e);        \
            goto fail;                  \
        }                               \
    } while (0)
    CKB(cudaMalloc((void **)&own_c, sizeof(int32_t) * std::max<int64_t>(faces, 1)));
    CKB(cudaMalloc((void **)&nbr_c, sizeof(int32_t) * std::max<int64_t>(faces, 1)));
    CKB(cudaMalloc((void **)&diag_c, sizeof(double) * std::max<int64_t>(rows, 1)));
    CKB(cudaMalloc((void **)&tab, sizeof(int64_t) * 4 * nsys));
    CKB(cudaMalloc((void **)&flags, sizeof(int)));
    {
        std::vector<int64_t> h(4 * (size_t)nsys);
        for (int k = 0; k < nsys; ++k) {
            h[k] = f_off[k];
            h[nsys + k] = Bt->row0[k];
            h[2 * nsys + k] = Bt->n[k];
            h[3 * nsys + k] = Bt->b_off[k];
        }
        CKB(cudaMemcpyAsync(tab, h.data(), sizeof(int64_t) * h.size(), cudaMemcpyHostToDevice, st));
        CKB(cudaMemsetAsync(flags, 0, sizeof(int), st));
        if (faces > 0)
            k_batch_faces<<<blocks_of(faces, 256), 256, 0, st>>>(faces, nsys, tab, tab + nsys,
                                                                  tab + 2 * nsys, owner, neighbour,
                                                                  own_c, nbr_c, flags);
        k_batch_diag<<<blocks_of(rows, 256), 256, 0, st>>>(rows, nsys, tab + nsys, tab + 2 * nsys,
                                                          tab + 3 * nsys, diag, diag_c);
        CKB(cudaGetLastError());
        int hf = 0;
        CKB(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        CKB(cudaStreamSynchronize(st));
        if (hf) {
            rc = LDU_ERR_BAD_ADDRESSING;
            goto fail;
        }
    }
    rc = ldu_create(rows, faces, own_c, nbr_c, diag_c, upper, lower, opt, stream, &A);
    if (rc != LDU_OK)
        goto fail;
    // caller numbering for the setters and gradients
    CKB(cudaMalloc((void **)&A->row_cell, sizeof(int) * std::max<int64_t>(rows, 1)));
    if (faces > 0)
        k_batch_remap<<<blocks_of(faces, 256), 256, 0, st>>>(faces, nsys, tab, tab + 3 * nsys, owner,
                                                              neighbour, A->owner, A->neighbour);
    k_batch_rowmap<<<blocks_of(rows, 256), 256, 0, st>>>(rows, nsys, tab + nsys, tab + 2 * nsys,
                                                        tab + 3 * nsys, A->row_cell);
    CKB(cudaGetLastError());
    CKB(cudaStreamSynchronize(st));
    A->n_cells = cells;
    {
        std::vector<SysDev> sys(nsys);
        for (int k = 0; k < nsys; ++k)
            sys[k] = SysDev{(int)Bt->row0[k], (int)Bt->n[k], (int)Bt->s_begin[k],
                            (int)Bt->s_count[k], (long long)Bt->b_off[k]};
        CKB(cudaMalloc((void **)&Bt->sys_dev, sizeof(SysDev) * nsys));
        CKB(cudaMemcpyAsync(Bt->sys_dev, sys.data(), sizeof(SysDev) * nsys, cudaMemcpyHostToDevice, st));
        CKB(cudaMalloc((void **)&Bt->out_dev, sizeof(SolveOut) * nsys));
        CKB(cudaMallocHost((void **)&Bt->out_host, sizeof(SolveOut) * nsys));
        CKB(cudaStreamSynchronize(st));
    }
    {
        // the launch grid: the smallest co-resident count over the batched kernels
        int per_sm = 1 << 30;
        for (int prec : {LDU_FP64, LDU_MIXED})
            for (int d = 0; d < 2; ++d) {
                int ps = 0;
                CKB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, batch_kernel(C, prec, d),
                                                                  A->block_threads, kMetaSmemMax));
                per_sm = std::min(per_sm, ps);
            }
        if (A->blocks_per_sm > 0)
            per_sm = std::min(per_sm, A->blocks_per_sm);
        if (per_sm < 1) {
            rc = LDU_ERR_UNSUPPORTED;
            goto fail;
        }
        Bt->grid = per_sm * A->num_sms;
        // staged float sweeps, when the staged kernel keeps the same number of
        // blocks per SM co-resident with its largest shared memory
        Bt->staged = false;
        if (A->staging == 0 && A->max_w > 0) {
            const void *ks = batch_kernel_staged(C);
            const size_t sm = batch_staged_smem(A, kMetaSmemMax);
            int ps = 0;
            if (sm <= (size_t)228 * 1024 / (size_t)per_sm - 5 * 1024 &&
                cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
                    cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, ks, A->block_threads, sm) ==
                    cudaSuccess &&
                ps >= per_sm)
                Bt->staged = true;
            cudaGetLastError();   // a refused attribute or query only turns staging off
        }
    }
    A->batch = Bt;
    {
        batch_opts o{};
        rc = build_schedule(A, Bt, o, st);
        if (rc != LDU_OK)
            goto fail;
    }
    cudaFree(own_c);
    cudaFree(nbr_c);
    cudaFree(diag_c);
    cudaFree(tab);
    cudaFree(flags);
    *out = A;
    return LDU_OK;
fail:
    cudaStreamSynchronize(st);
    if (own_c)
        cudaFree(own_c);
    if (nbr_c)
        cudaFree(nbr_c);
    if (diag_c)
        cudaFree(diag_c);
    if (tab)
        cudaFree(tab);
    if (flags)
        cudaFree(flags);
    {
        // decide ownership before the handle goes away: once attached, the
        // batch tables are freed with the handle
        const bool attached = A && Bt && A->batch == Bt;
        if (A)
            ldu_destroy(A);
        if (Bt && !attached) {
            if (Bt->sys_dev)
                cudaFree(Bt->sys_dev);
            if (Bt->out_dev)
                cudaFree(Bt->out_dev);
            if (Bt->out_host)
                cudaFreeHost(Bt->out_host);
            delete Bt;
        }
    }
    return rc;
#undef CKB
}

int ldu_batch_schedule(ldu_matrix *A, const batch_opts *opts, ldu_stream_t stream) {
    if (!A || !A->batch)
        return LDU_ERR_BAD_ARG;
    batch_opts o{};
    if (opts)
        o = *opts;
    if (o.max_team < 0 || o.team_work_scale < 0.0)
        return LDU_ERR_BAD_ARG;
    return build_schedule(A, A->batch, o, (cudaStream_t)stream);
}

int ldu_batch_info(const ldu_matrix *A, int *nsys, int *grid_blocks, int *ntasks, int *max_team) {
    if (!A || !A->batch)
        return LDU_ERR_BAD_ARG;
    if (nsys)
        *nsys = A->batch->nsys;
    if (grid_blocks)
        *grid_blocks = A->batch->grid;
    if (ntasks)
        *ntasks = A->batch->ntasks;
    if (max_team)
        *max_team = A->batch->max_team_used;
    return LDU_OK;
}

int pcg_solve_batched_async(const ldu_matrix *Ac, const double *b, double *x, double tol, int maxit,
                            int precision, const pcg_opts *o, ldu_stream_t stream) {
    ldu_matrix *A = const_cast<ldu_matrix *>(Ac);
    if (!A || !A->batch || maxit < 0 || !(tol >= 0.0) || (A->n > 0 && (!b || !x)))
        return LDU_ERR_BAD_ARG;
    if (precision != LDU_FP64 && precision != LDU_MIXED)
        return LDU_ERR_BAD_ARG;
    ldu_batch *Bt = A->batch;
    pcg_opts opt{};
    if (o)
        opt = *o;
    if (opt.rr_period < 0 || opt.tau < 0.0 || opt.barrier_timeout_s < 0.0 ||
        (opt.deflate != 0 && opt.deflate != 1))
        return LDU_ERR_BAD_ARG;
    if (precision == LDU_MIXED && opt.rr_period == 0 && opt.tau == 0.0)
        opt.rr_period = 12;   // small systems: a plain period of 12
    cudaStream_t st = (cudaStream_t)stream;
    const bool defl = precision == LDU_MIXED && opt.deflate;
    const bool stg = precision == LDU_MIXED && !defl && Bt->staged;
    const void *kern = stg ? batch_kernel_staged(A->C) : batch_kernel(A->C, precision, defl);
    const size_t smem = stg ? batch_staged_smem(A, Bt->smem) : Bt->smem;
    SolveParams P;
    P.A = view_of(A);
    P.A.meta_smem = Bt->smem > 0;
    P.A.meta_cap = (int)(Bt->smem / sizeof(int2));
    P.A.stage_w = stg ? A->max_w : 0;
    P.A.stages = stg ? 2 : 0;
    P.sync.count = A->bar_count;
    P.sync.err = A->bar_err;
    const double tmo = opt.barrier_timeout_s > 0.0 ? opt.barrier_timeout_s : 10.0;
    P.sync.timeout_ns = (unsigned long long)(tmo * 1e9);
    P.slots = Bt->slots_dev;
    P.tasks = nullptr;
    P.out = Bt->out_dev;
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
    P.deflate = precision == LDU_MIXED ? opt.deflate : 0;
    P.fault_inject = 0;
    BatchView B;
    B.sys = Bt->sys_dev;
    B.tasks = Bt->tasks_dev;
    B.list = Bt->list_dev;
    B.list_begin = Bt->list_begin_dev;
    B.counters = Bt->counters_dev;
    cudaError_t e;
    if ((e = cudaMemsetAsync(Bt->counters_dev, 0, sizeof(unsigned) * 32 * Bt->ntasks, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(A->bar_err, 0, sizeof(int) * 64, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(Bt->out_dev, 0xff, sizeof(SolveOut) * Bt->nsys, st)) != cudaSuccess)
        return cuda_status(e);
    void *args[] = {&P, &B};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Bt->grid);
    cfg.blockDim = dim3(A->block_threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, kern, args);
    A->last.staged = stg ? 1 : 0;
    A->last.grid_blocks = Bt->grid;
    A->last.block_threads = A->block_threads;
    return cuda_status(e);
}

int ldu_batch_results(const ldu_matrix *A, int *iters, double *relres, int *status,
                      ldu_stream_t stream) {
    if (!A || !A->batch)
        return LDU_ERR_BAD_ARG;
    ldu_batch *Bt = A->batch;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    int err = 0;
    if ((e = cudaMemcpyAsync(Bt->out_host, Bt->out_dev, sizeof(SolveOut) * Bt->nsys, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&err, A->bar_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_status(e);
    if (err == kDevTimeout)
        return LDU_ERR_BARRIER_TIMEOUT;
    if (err != 0)
        return LDU_ERR_CUDA;
    int worst = LDU_OK;
    for (int k = 0; k < Bt->nsys; ++k) {
        const SolveOut &o = Bt->out_host[k];
        int s;
        switch (o.status) {
        case kDevOk: s = LDU_OK; break;
        case kDevNotConverged: s = LDU_NOT_CONVERGED; break;
        case kDevNotSpd: s = LDU_ERR_NOT_SPD; break;
        default: s = LDU_ERR_CUDA; break;
        }
        if (status)
            status[k] = s;
        if (iters)
            iters[k] = o.iters;
        if (relres)
            relres[k] = o.relres;
        if (s < 0 && (worst >= 0 || s < worst))
            worst = s;
        else if (s == LDU_NOT_CONVERGED && worst == LDU_OK)
            worst = s;
    }
    return worst;
}

int pcg_solve_batched(const ldu_matrix *A, const double *b, double *x, double tol, int maxit,
                      int precision, const pcg_opts *opts, int *iters, double *relres, int *status,
                      ldu_stream_t stream) {
    int rc = pcg_solve_batched_async(A, b, x, tol, maxit, precision, opts, stream);
    if (rc != LDU_OK)
        return rc;
    return ldu_batch_results(A, iters, relres, status, stream);
}

}  // extern "C"
