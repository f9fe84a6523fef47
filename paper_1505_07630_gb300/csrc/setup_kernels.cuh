// setup_kernels.cuh -- device kernels of the repack (validation, slice
// widths, slot fill, face scatter, per-row sort, scaling, values), the
// standalone SpMV and the face gradient.  Included by the .cu files that
// launch them; each gets its own copy (anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include "ldupcg_impl.cuh"

namespace {

using namespace ldu;

__global__ void k_validate_count(int64_t nf, int n, const int32_t *__restrict__ own,
                                 const int32_t *__restrict__ nbr, int *deg, int *flags) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int o = own[f], nb = nbr[f];
        if (o < 0 || nb < 0 || o >= n || nb >= n) {
            atomicOr(flags, kFlagBadIndex);
            continue;
        }
        if (o >= nb) {
            atomicOr(flags, kFlagBadOrder);
            continue;
        }
        atomicAdd(deg + o, 1);
        atomicAdd(deg + nb, 1);
    }
}

__global__ void k_validate_values(int64_t n, int64_t nf, const double *diag, const double *up,
                                  const double *lo, int *flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = diag[i];
        if (!isfinite(d))
            atomicOr(flags, kFlagNonFinite);
        else if (!(d > 0.0))
            atomicOr(flags, kFlagBadDiag);
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += stride)
        if (!isfinite(up[f]) || !isfinite(lo[f]))
            atomicOr(flags, kFlagNonFinite);
}

// one thread per slice: width = max degree of its rows
__global__ void k_slice_width(int n, int n_slices, int C, const int *deg, int *slice_w) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices)
        return;
    int w = 0;
    for (int i = 0; i < C; ++i) {
        const int r = s * C + i;
        if (r < n)
            w = max(w, deg[r]);
    }
    slice_w[s] = w;
}

// padding everywhere first: col = own row, fid = pad
__global__ void k_fill_pad(int n_pad, int C, const int *slice_ptr, const int *slice_w, int *col,
                           uint32_t *fid) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    const int s = r / C, i = r - s * C;
    const int w = slice_w[s];
    for (int k = 0; k < w; ++k) {
        const int at = slice_ptr[s] + k * C + i;
        col[at] = r;
        fid[at] = kPadFid;
    }
}

__global__ void k_scatter_faces(int64_t nf, int C, const int32_t *__restrict__ own,
                                const int32_t *__restrict__ nbr, const int *slice_ptr, int *cursor,
                                int *col, uint32_t *fid) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int o = own[f], nb = nbr[f];
        int k = atomicAdd(cursor + o, 1);
        int at = slice_ptr[o / C] + k * C + (o % C);
        col[at] = nb;
        fid[at] = (uint32_t)f;
        k = atomicAdd(cursor + nb, 1);
        at = slice_ptr[nb / C] + k * C + (nb % C);
        col[at] = o;
        fid[at] = (uint32_t)f | kLowerBit;
    }
}

// insertion sort of each row's real slots by (column, face id)
__global__ void k_sort_rows(int n, int C, const int *slice_ptr, const int *deg, int *col,
                            uint32_t *fid) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const int s = r / C, i = r - s * C;
    const int base = slice_ptr[s] + i;
    const int d = deg[r];
    for (int a = 1; a < d; ++a) {
        const int ca = col[base + a * C];
        const uint32_t fa = fid[base + a * C];
        int b = a - 1;
        while (b >= 0) {
            const int cb = col[base + b * C];
            const uint32_t fb = fid[base + b * C];
            if (cb < ca || (cb == ca && (fb & ~kLowerBit) <= (fa & ~kLowerBit)))
                break;
            col[base + (b + 1) * C] = cb;
            fid[base + (b + 1) * C] = fb;
            --b;
        }
        col[base + (b + 1) * C] = ca;
        fid[base + (b + 1) * C] = fa;
    }
}

// 16-bit offsets (column minus row) of every stored slot of row r; raises
// kFlagOverflow when one does not fit, and the handle then keeps int32
// columns only.
__global__ void k_col16(int n_pad, int C, const int *slice_ptr, const int *slice_w, const int *col,
                        short *col16, int *flag) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    const int s = r / C, i = r - s * C;
    const int base = slice_ptr[s] + i, w = slice_w[s];
    bool fits = true;
    for (int k = 0; k < w; ++k) {
        const int d = col[base + k * C] - r;
        const bool ok = d >= -32768 && d <= 32767;
        fits = fits && ok;
        col16[base + k * C] = ok ? (short)d : (short)0;
    }
    if (!fits)
        atomicOr(flag, kFlagOverflow);
}

// diagonal scaling factors; padded rows get sd = isd = 1, dg = 0.  With a
// row map (batched handles) diag is in the caller's cell order and rows
// between systems (map -1) keep a unit diagonal.
__global__ void k_diag_scale(int n, int n_pad, const double *diag, double *sd, double *isd,
                             double *dg, float *sdf, int *flags, const int *row_cell) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    if (r < n) {
        const int c = row_cell ? row_cell[r] : r;
        const double d = c >= 0 ? diag[c] : 1.0;
        if (!(d > 0.0) || !isfinite(d))
            atomicOr(flags, kFlagBadDiag);
        const double q = sqrt(d);
        sd[r] = q;
        isd[r] = 1.0 / q;
        dg[r] = d;
        if (sdf)
            sdf[r] = (float)q;
    } else {
        sd[r] = 1.0;
        isd[r] = 1.0;
        dg[r] = 0.0;
        if (sdf)
            sdf[r] = 1.0f;
    }
}

// diag[r] = extra[r] + sum of coef over the row's faces, in slot order
// (extra in the caller's cell order when a row map is given)
__global__ void k_diag_from_coef(int n, int n_pad, int C, const int *slice_ptr, const int *slice_w,
                                 const uint32_t *fid, const double *coef, const double *extra,
                                 double *sd, double *isd, double *dg, float *sdf, int *flags,
                                 const int *row_cell) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    if (r >= n) {
        sd[r] = 1.0;
        isd[r] = 1.0;
        dg[r] = 0.0;
        sdf[r] = 1.0f;
        return;
    }
    const int s = r / C, i = r - s * C;
    const int w = slice_w[s];
    const int c = row_cell ? row_cell[r] : r;
    double d = c >= 0 ? extra[c] : 1.0;
    for (int k = 0; k < w; ++k) {
        const uint32_t f = fid[slice_ptr[s] + k * C + i];
        if (f != kPadFid)
            d += coef[f & ~kLowerBit];
    }
    if (!(d > 0.0) || !isfinite(d))
        atomicOr(flags, kFlagBadDiag);
    const double q = sqrt(d);
    sd[r] = q;
    isd[r] = 1.0 / q;
    dg[r] = d;
    sdf[r] = (float)q;
}

// scaled off-diagonal values of every slot.  coef != nullptr: a = -coef[f];
// else a = upper[f] (owner row) or lower[f] (neighbour row).
__global__ void k_values(int n_pad, int C, const int *slice_ptr, const int *slice_w, const int *col,
                         const uint32_t *fid, const double *up, const double *lo,
                         const double *coef, const double *sd, double *v64, float *v32) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    const int s = r / C, i = r - s * C;
    const int w = slice_w[s];
    const double sr = sd[r];
    for (int k = 0; k < w; ++k) {
        const int at = slice_ptr[s] + k * C + i;
        const uint32_t f = fid[at];
        double v = 0.0;
        if (f != kPadFid) {
            const uint32_t face = f & ~kLowerBit;
            const double a = coef ? -coef[face] : ((f & kLowerBit) ? lo[face] : up[face]);
            v = a / (sr * sd[col[at]]);
        }
        v64[at] = v;
        v32[at] = (float)v;
    }
}

// y = A x = D^1/2 (I + Ahat_off) D^1/2 x, one thread per row.  scale holds the
// factors sd in the product's type: the float copy for the float product, so
// that no entry converts a double (conversions run on this GPU's slow FP64
// pipe, which they otherwise saturate).  PRESCALED: x already holds u = sd x
// (k_spmv_prescale), which leaves one FP64 operation per stored entry in the
// double product instead of two; the products and their order are the same
// either way.  Every column stored for a row below n is below n (a padding
// slot points at its own row, with value 0), so the loop needs no bounds
// test.  Caller buffers hold exactly n entries.
template <typename T, bool PRESCALED>
__global__ void k_spmv(int n, int C, const int *slice_ptr, const int *slice_w, const int *col,
                       const T *val, const T *scale, const T *__restrict__ x, T *__restrict__ y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const int s = r / C, i = r - s * C;
    const int w = slice_w[s];
    const T sr = scale[r];
    T acc = PRESCALED ? x[r] : sr * x[r];
    for (int k = 0; k < w; ++k) {
        const int at = slice_ptr[s] + k * C + i;
        const int c = col[at];
        acc = fma(val[at], PRESCALED ? x[c] : scale[c] * x[c], acc);
    }
    y[r] = sr * acc;
}

// u = sd x, the input of the prescaled product
template <typename T>
__global__ void k_spmv_prescale(int n, const T *__restrict__ scale, const T *__restrict__ x,
                                T *__restrict__ u) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n)
        u[r] = scale[r] * x[r];
}

// dL/d(diag_extra)_i = -lambda_i x_i (the diagonal enters A as +e_i e_i^T)
__global__ void k_diag_grad(int64_t n, const double *__restrict__ lam,
                            const double *__restrict__ x, double *__restrict__ g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        g[i] = -lam[i] * x[i];
}

// cell diffusivity -> face coefficients (harmonic mean) and wall terms;
// owner/neighbour and k in the caller's cell numbering
__global__ void k_harmonic_coeffs(int64_t nf, int64_t n, const int32_t *__restrict__ own,
                                  const int32_t *__restrict__ nbr, const double *__restrict__ k,
                                  const double *__restrict__ g, const double *__restrict__ bfac,
                                  double *__restrict__ coef, double *__restrict__ extra) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += stride) {
        const double ko = k[own[f]], kn = k[nbr[f]];
        coef[f] = g[f] * (2.0 * ko * kn / (ko + kn));
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        extra[i] = k[i] * bfac[i];
}

// dL/dk of the cell of row r: its wall term plus, over the faces of its
// stored slots in slot order, dL/dc_f g_f dk_f/dk_P with
// dk_f/dk_P = 2 k_N^2 / (k_P + k_N)^2.  One thread per row, no atomics.
// row_cell (batched handles) maps rows to caller cells, -1 between systems;
// without it rows below n are cells.
__global__ void k_harmonic_grad(int n_pad, int n, int C, const int *slice_ptr, const int *slice_w,
                                const int *col, const uint32_t *fid, const int *row_cell,
                                const double *__restrict__ k, const double *__restrict__ g,
                                const double *__restrict__ bfac, const double *__restrict__ dcoef,
                                const double *__restrict__ dextra, double *__restrict__ dk) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad)
        return;
    const int cell = row_cell ? row_cell[r] : (r < n ? r : -1);
    if (cell < 0)
        return;
    const int s = r / C, i = r - s * C;
    const int base = slice_ptr[s] + i, w = slice_w[s];
    const double kp = k[cell];
    double acc = dextra[cell] * bfac[cell];
    for (int q = 0; q < w; ++q) {
        const int at = base + q * C;
        const uint32_t f = fid[at];
        if (f == kPadFid)
            continue;
        const uint32_t face = f & ~kLowerBit;
        const int nrow = col[at];
        const double kn = k[row_cell ? row_cell[nrow] : nrow];
        const double sum = kp + kn;
        acc += dcoef[face] * g[face] * (2.0 * kn * kn / (sum * sum));
    }
    dk[cell] = acc;
}

__global__ void k_face_grad(int64_t nf, const int32_t *__restrict__ own,
                            const int32_t *__restrict__ nbr, const double *__restrict__ lam,
                            const double *__restrict__ x, double *__restrict__ g) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int o = own[f], nb = nbr[f];
        g[f] = -(lam[o] - lam[nb]) * (x[o] - x[nb]);
    }
}

// dL/dupper_f = -lambda_o x_n, dL/dlower_f = -lambda_n x_o (dL/dA_ij = -lambda_i x_j)
__global__ void k_value_grad(int64_t nf, const int32_t *__restrict__ own,
                             const int32_t *__restrict__ nbr, const double *__restrict__ lam,
                             const double *__restrict__ x, double *__restrict__ gup,
                             double *__restrict__ glo) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int o = own[f], nb = nbr[f];
        gup[f] = -lam[o] * x[nb];
        glo[f] = -lam[nb] * x[o];
    }
}

}  // namespace
