"""Python binding of libldupcg: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/ldupcg.h) and does nothing but check tensor placement, pass device
pointers and the current torch CUDA stream, and turn status codes into
exceptions.  All arithmetic of the solve runs in the library's kernels; if
the library is missing the import of this module succeeds but every call
raises, so there is never a silent fallback.
"""
import ctypes
import os

import torch

from . import build as _build

OK, NOT_CONVERGED = 0, 1
ERR_BAD_ARG, ERR_BAD_ADDRESSING, ERR_NOT_SPD = -1, -2, -3
ERR_CUDA, ERR_BARRIER_TIMEOUT, ERR_OOM, ERR_UNSUPPORTED = -4, -5, -6, -7
FP64, FP32, MIXED = 0, 1, 2
_PREC = {"fp64": FP64, "fp32": FP32, "mixed": MIXED, FP64: FP64, FP32: FP32, MIXED: MIXED}


class LduError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class LduOpts(ctypes.Structure):
    _fields_ = [("slice_rows", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("staging", ctypes.c_int),
                ("min_slices", ctypes.c_int)]


class PcgOpts(ctypes.Structure):
    _fields_ = [("rr_period", ctypes.c_int), ("tau", ctypes.c_double), ("restart", ctypes.c_int),
                ("barrier_timeout_s", ctypes.c_double), ("fault_inject", ctypes.c_int),
                ("deflate", ctypes.c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("max_team", ctypes.c_int), ("team_work_scale", ctypes.c_double)]


class AmgOpts(ctypes.Structure):
    _fields_ = [("max_coarse", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("lanes_per_row", ctypes.c_int)]


class LduSolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("replacements", ctypes.c_int), ("relres", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("grid_blocks", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("staged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LduInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_padded", ctypes.c_int64),
                ("nnz_padded", ctypes.c_int64), ("slice_rows", ctypes.c_int),
                ("n_slices", ctypes.c_int64), ("max_row_entries", ctypes.c_int),
                ("device_bytes", ctypes.c_int64), ("col16", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_vp = ctypes.c_void_p


def library_path():
    return _build.LIB


def lib():
    """Load libldupcg.so (built in-tree by build.py); raise if it is absent."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        pi, pd = ctypes.POINTER(i), ctypes.POINTER(d)
        L.ldu_create.argtypes = [i64, i64, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(LduOpts), _vp,
                                 ctypes.POINTER(_vp)]
        L.ldu_update_values.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.ldu_set_face_coeffs.argtypes = [_vp, _vp, _vp, _vp]
        L.ldu_spmv.argtypes = [_vp, i, _vp, _vp, _vp]
        L.pcg_solve.argtypes = [_vp, _vp, _vp, d, i, pi, pd, _vp]
        L.pipecg_solve.argtypes = [_vp, _vp, _vp, d, i, i, ctypes.POINTER(PcgOpts), pi, pd, _vp]
        L.ldu_face_grad.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.ldu_diag_grad.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.ldu_diag_grad.restype = i
        L.ldu_value_grad.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.ldu_value_grad.restype = i
        L.ldu_heat_steps.argtypes = [_vp, _vp, _vp, i, d, i, i, ctypes.POINTER(PcgOpts), pi, pd,
                                     _vp]
        L.ldu_heat_steps.restype = i
        L.ldu_piso_pressure.argtypes = [_vp, _vp, _vp, _vp, d, i, i, ctypes.POINTER(PcgOpts), pi,
                                        pd, _vp]
        L.ldu_piso_pressure.restype = i
        L.ldu_harmonic_coeffs.argtypes = [_vp] * 7
        L.ldu_harmonic_coeffs.restype = i
        L.ldu_harmonic_grad.argtypes = [_vp] * 8
        L.ldu_harmonic_grad.restype = i
        L.ldu_last_stats.argtypes = [_vp, ctypes.POINTER(LduSolveStats)]
        L.ldu_get_info.argtypes = [_vp, ctypes.POINTER(LduInfo)]
        L.ldu_destroy.argtypes = [_vp]
        L.ldu_destroy.restype = None
        L.pcg_solve_ldu_noalloc.argtypes = [i64, i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, d, i,
                                            pi, pd, _vp]
        L.pcg_solve_ldu_noalloc.restype = i
        L.ldu_create_batched.argtypes = [i, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                         ctypes.POINTER(LduOpts), _vp, ctypes.POINTER(_vp)]
        L.ldu_create_batched.restype = i
        L.ldu_batch_schedule.argtypes = [_vp, ctypes.POINTER(BatchOpts), _vp]
        L.ldu_batch_schedule.restype = i
        L.ldu_batch_info.argtypes = [_vp, pi, pi, pi, pi]
        L.ldu_batch_info.restype = i
        L.pcg_solve_batched_async.argtypes = [_vp, _vp, _vp, d, i, i, ctypes.POINTER(PcgOpts), _vp]
        L.pcg_solve_batched_async.restype = i
        L.ldu_batch_results.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.ldu_batch_results.restype = i
        L.pcg_solve_batched.argtypes = [_vp, _vp, _vp, d, i, i, ctypes.POINTER(PcgOpts), _vp, _vp,
                                        _vp, _vp]
        L.pcg_solve_batched.restype = i
        L.ldu_amg_create.argtypes = [i64, i64, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(AmgOpts),
                                     _vp, ctypes.POINTER(_vp)]
        L.ldu_amg_create.restype = i
        L.ldu_amg_destroy.argtypes = [_vp]
        L.ldu_amg_destroy.restype = None
        L.ldu_amg_info.argtypes = [_vp, pi, _vp, _vp, i]
        L.ldu_amg_info.restype = i
        L.ldu_amg_aggregates.argtypes = [_vp, i, _vp]
        L.ldu_amg_aggregates.restype = i
        L.ldu_amg_vcycle.argtypes = [_vp, i, _vp, _vp, _vp]
        L.ldu_amg_vcycle.restype = i
        L.amg_pcg_solve.argtypes = [_vp, _vp, _vp, d, i, i, pi, pd, _vp]
        L.amg_pcg_solve.restype = i
        L.amg_pipecg_solve.argtypes = [_vp, _vp, _vp, d, i, pi, pd, _vp]
        L.amg_pipecg_solve.restype = i
        L.ldu_status_string.argtypes = [i]
        L.ldu_status_string.restype = ctypes.c_char_p
        for name in ("ldu_create", "ldu_update_values", "ldu_set_face_coeffs", "ldu_spmv",
                     "pcg_solve", "pipecg_solve", "ldu_face_grad", "ldu_last_stats",
                     "ldu_get_info"):
            getattr(L, name).restype = i
        _LIB = L
    return _LIB


def status_string(status):
    try:
        return lib().ldu_status_string(int(status)).decode()
    except RuntimeError:
        return "library not loaded"


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _dev(t, dtype, n, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {n} elements")
    return _vp(t.data_ptr())


def _check(status, what, allow_not_converged=True):
    if status == OK or (status == NOT_CONVERGED and allow_not_converged):
        return status
    raise LduError(status, what)


class LduMatrix:
    """A device-resident handle of one LDU matrix (owner of its allocations)."""

    def __init__(self, handle, n, nfaces, device):
        self._h = handle
        self.n = n
        self.nfaces = nfaces
        self.device = device

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("LduMatrix was destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().ldu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        out = LduInfo()
        _check(lib().ldu_get_info(self.handle, ctypes.byref(out)), "ldu_get_info")
        return out.as_dict()

    def stats(self):
        out = LduSolveStats()
        _check(lib().ldu_last_stats(self.handle, ctypes.byref(out)), "ldu_last_stats")
        return out.as_dict()


def ldu_create(n, owner, neighbour, diag, upper, lower, slice_rows=0, block_threads=0,
               blocks_per_sm=0, staging=0, min_slices=0, stream=None):
    """Create a handle from device tensors (int32 owner/neighbour, float64 values)."""
    nf = owner.numel()
    args = [ctypes.c_int64(n), ctypes.c_int64(nf),
            _dev(owner, torch.int32, nf, "owner"), _dev(neighbour, torch.int32, nf, "neighbour"),
            _dev(diag, torch.float64, n, "diag"), _dev(upper, torch.float64, nf, "upper"),
            _dev(lower, torch.float64, nf, "lower")]
    opts = LduOpts(slice_rows, block_threads, blocks_per_sm, staging, min_slices)
    h = _vp()
    st = lib().ldu_create(*args, ctypes.byref(opts), _stream(stream), ctypes.byref(h))
    _check(st, "ldu_create", allow_not_converged=False)
    return LduMatrix(h, n, nf, diag.device)


def ldu_update_values(A, diag, upper, lower, stream=None):
    st = lib().ldu_update_values(A.handle, _dev(diag, torch.float64, A.n, "diag"),
                                 _dev(upper, torch.float64, A.nfaces, "upper"),
                                 _dev(lower, torch.float64, A.nfaces, "lower"), _stream(stream))
    _check(st, "ldu_update_values", allow_not_converged=False)


def ldu_set_face_coeffs(A, coef, diag_extra, stream=None):
    st = lib().ldu_set_face_coeffs(A.handle, _dev(coef, torch.float64, A.nfaces, "coef"),
                                   _dev(diag_extra, torch.float64, A.n, "diag_extra"),
                                   _stream(stream))
    _check(st, "ldu_set_face_coeffs", allow_not_converged=False)


def ldu_spmv(A, x, y=None, precision="fp64", stream=None):
    p = _PREC[precision]
    dt = torch.float64 if p == FP64 else torch.float32
    if y is None:
        y = torch.empty(A.n, dtype=dt, device=x.device)
    st = lib().ldu_spmv(A.handle, p, _dev(x, dt, A.n, "x"), _dev(y, dt, A.n, "y"), _stream(stream))
    _check(st, "ldu_spmv", allow_not_converged=False)
    return y


def pcg_solve(A, b, x=None, tol=1e-8, maxit=20000, stream=None, check=True):
    """Jacobi-PCG; x (in: initial guess, out: solution) is allocated if None.
    Returns (x, status, iters, relres)."""
    if x is None:
        x = torch.zeros(A.n, dtype=torch.float64, device=b.device)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().pcg_solve(A.handle, _dev(b, torch.float64, A.n, "b"),
                         _dev(x, torch.float64, A.n, "x"), float(tol), int(maxit),
                         ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(st, "pcg_solve")
    return x, st, it.value, rr.value


def pipecg_solve(A, b, x=None, tol=1e-8, maxit=20000, precision="fp64", rr_period=0, tau=0.0,
                 restart=False, deflate=False, barrier_timeout_s=0.0, fault_inject=0, stream=None,
                 check=True):
    """Pipelined Jacobi-PCG (precision 'fp64' or 'mixed').
    Returns (x, status, iters, relres)."""
    if x is None:
        x = torch.zeros(A.n, dtype=torch.float64, device=b.device)
    opts = PcgOpts(int(rr_period), float(tau), int(bool(restart)), float(barrier_timeout_s),
                   int(fault_inject), int(bool(deflate)))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().pipecg_solve(A.handle, _dev(b, torch.float64, A.n, "b"),
                            _dev(x, torch.float64, A.n, "x"), float(tol), int(maxit),
                            _PREC[precision], ctypes.byref(opts), ctypes.byref(it),
                            ctypes.byref(rr), _stream(stream))
    if check:
        _check(st, "pipecg_solve")
    return x, st, it.value, rr.value


def ldu_face_grad(A, lam, x, out=None, stream=None):
    if out is None:
        out = torch.empty(A.nfaces, dtype=torch.float64, device=x.device)
    st = lib().ldu_face_grad(A.handle, _dev(lam, torch.float64, A.n, "lambda"),
                             _dev(x, torch.float64, A.n, "x"),
                             _dev(out, torch.float64, A.nfaces, "dcoef"), _stream(stream))
    _check(st, "ldu_face_grad", allow_not_converged=False)
    return out


def pcg_solve_ldu_noalloc(n, owner, neighbour, diag, upper, lower, b, x, tol=1e-8, maxit=20000,
                          stream=None, check=True):
    """Jacobi-PCG straight from device LDU arrays, using only the library's
    fixed device scratch (no allocation; n <= 32768).  Returns
    (x, status, iters, relres)."""
    nf = owner.numel()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().pcg_solve_ldu_noalloc(
        ctypes.c_int64(n), ctypes.c_int64(nf), _dev(owner, torch.int32, nf, "owner"),
        _dev(neighbour, torch.int32, nf, "neighbour"), _dev(diag, torch.float64, n, "diag"),
        _dev(upper, torch.float64, nf, "upper"), _dev(lower, torch.float64, nf, "lower"),
        _dev(b, torch.float64, n, "b"), _dev(x, torch.float64, n, "x"), float(tol), int(maxit),
        ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(st, "pcg_solve_ldu_noalloc")
    return x, st, it.value, rr.value


def ldu_diag_grad(A, lam, x, out=None, stream=None):
    """dL/d(diag_extra) = -lambda * x in the library's kernel."""
    if out is None:
        out = torch.empty(A.n, dtype=torch.float64, device=x.device)
    st = lib().ldu_diag_grad(A.handle, _dev(lam, torch.float64, A.n, "lambda"),
                             _dev(x, torch.float64, A.n, "x"),
                             _dev(out, torch.float64, A.n, "ddiag"), _stream(stream))
    _check(st, "ldu_diag_grad", allow_not_converged=False)
    return out


def ldu_value_grad(A, lam, x, dupper=None, dlower=None, stream=None):
    """(dL/dupper, dL/dlower) = (-lambda_o x_n, -lambda_n x_o) per face."""
    if dupper is None:
        dupper = torch.empty(A.nfaces, dtype=torch.float64, device=x.device)
    if dlower is None:
        dlower = torch.empty(A.nfaces, dtype=torch.float64, device=x.device)
    st = lib().ldu_value_grad(A.handle, _dev(lam, torch.float64, A.n, "lam"),
                              _dev(x, torch.float64, A.n, "x"),
                              _dev(dupper, torch.float64, A.nfaces, "dupper"),
                              _dev(dlower, torch.float64, A.nfaces, "dlower"), _stream(stream))
    _check(st, "ldu_value_grad", allow_not_converged=False)
    return dupper, dlower


def ldu_heat_steps(A, mass, T, nsteps, tol=1e-8, maxit=20000, precision="mixed", stream=None,
                   check=True, **opts):
    """nsteps backward-Euler heat steps (M + A) T^(n+1) = M T^n on a handle
    that holds M + A, in place on T, each step warm-started from the last.
    precision: 'fp64' (Jacobi-PCG) or 'mixed'.  Returns
    (T, status, iterations over all steps, last true relative residual)."""
    o = _pcg_opts(**opts)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().ldu_heat_steps(A.handle, _dev(mass, torch.float64, A.n, "mass"),
                              _dev(T, torch.float64, A.n, "T"), int(nsteps), float(tol),
                              int(maxit), _PREC["fp64" if precision == "fp64" else "mixed"],
                              ctypes.byref(o), ctypes.byref(it), ctypes.byref(rr),
                              _stream(stream))
    if check:
        _check(st, "ldu_heat_steps")
    return T, st, it.value, rr.value


def ldu_piso_pressure(A, coef, phi, p, tol=1e-8, maxit=20000, precision="mixed", rr_period=0,
                      tau=0.0, deflate=False, stream=None, check=True):
    """Pressure stage of a PISO step: b = -div(phi), solve A p = b from p,
    phi -= coef (p_N - p_P).  phi and p are updated in place; returns
    (status, iters, relres)."""
    prec = {"fp64": FP64, "mixed": MIXED}[precision]
    opts = PcgOpts(rr_period=rr_period, tau=tau, deflate=int(bool(deflate)))
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().ldu_piso_pressure(A.handle, _dev(coef, torch.float64, A.nfaces, "coef"),
                                 _dev(phi, torch.float64, A.nfaces, "phi"),
                                 _dev(p, torch.float64, A.n, "p"), float(tol), int(maxit), prec,
                                 ctypes.byref(opts), ctypes.byref(it), ctypes.byref(rr),
                                 _stream(stream))
    if check:
        _check(st, "ldu_piso_pressure")
    return st, it.value, rr.value


def ldu_harmonic_coeffs(A, k, g, bfac, coef=None, extra=None, stream=None):
    """(coef, diag_extra) of the FVM Laplacian for cell diffusivities k:
    coef_f = g_f 2 k_o k_n / (k_o + k_n), diag_extra_P = k_P bfac_P."""
    if coef is None:
        coef = torch.empty(A.nfaces, dtype=torch.float64, device=k.device)
    if extra is None:
        extra = torch.empty(A.n, dtype=torch.float64, device=k.device)
    st = lib().ldu_harmonic_coeffs(A.handle, _dev(k, torch.float64, A.n, "k"),
                                   _dev(g, torch.float64, A.nfaces, "g"),
                                   _dev(bfac, torch.float64, A.n, "bfac"),
                                   _dev(coef, torch.float64, A.nfaces, "coef"),
                                   _dev(extra, torch.float64, A.n, "diag_extra"), _stream(stream))
    _check(st, "ldu_harmonic_coeffs", allow_not_converged=False)
    return coef, extra


def ldu_harmonic_grad(A, k, g, bfac, dcoef, dextra, out=None, stream=None):
    """dL/dk from dL/dcoef and dL/d(diag_extra) (chain rule of
    ldu_harmonic_coeffs), one fixed-order sum per cell."""
    if out is None:
        out = torch.empty(A.n, dtype=torch.float64, device=k.device)
    st = lib().ldu_harmonic_grad(A.handle, _dev(k, torch.float64, A.n, "k"),
                                 _dev(g, torch.float64, A.nfaces, "g"),
                                 _dev(bfac, torch.float64, A.n, "bfac"),
                                 _dev(dcoef, torch.float64, A.nfaces, "dcoef"),
                                 _dev(dextra, torch.float64, A.n, "ddiag_extra"),
                                 _dev(out, torch.float64, A.n, "dk"), _stream(stream))
    _check(st, "ldu_harmonic_grad", allow_not_converged=False)
    return out


def ldu_destroy(A):
    A.close()


def from_system(sys_, device="cuda", **opts):
    """Upload an ldu_cases.LduSystem and create its handle (inputs only)."""
    t = lambda a, dt: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()  # noqa: E731
    A = ldu_create(sys_.n, t(sys_.owner, torch.int32), t(sys_.neighbour, torch.int32),
                   t(sys_.diag, torch.float64), t(sys_.upper, torch.float64),
                   t(sys_.lower, torch.float64), **opts)
    return A


# ---- aggregation-AMG preconditioned CG ---------------------------------------

class LduAmg:
    """A device-resident AMG hierarchy (owner of its allocations)."""

    def __init__(self, handle, n, device):
        self._h = handle
        self.n = n
        self.device = device

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("LduAmg was destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().ldu_amg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """{'levels': L, 'rows': [...], 'nnz': [...]} of every level."""
        import numpy as np
        cap = 80
        rows = np.zeros(cap, dtype=np.int64)
        nnz = np.zeros(cap, dtype=np.int64)
        lv = ctypes.c_int()
        _check(lib().ldu_amg_info(self.handle, ctypes.byref(lv), _vp(rows.ctypes.data),
                                  _vp(nnz.ctypes.data), cap), "ldu_amg_info")
        L = lv.value
        return {"levels": L, "rows": rows[:L].tolist(), "nnz": nnz[:L].tolist()}


def ldu_amg_create(n, owner, neighbour, diag, upper, lower, max_coarse=0, max_levels=0,
                   lanes_per_row=0, stream=None):
    """Build the AMG hierarchy of an LDU matrix given as device tensors."""
    nf = owner.numel()
    args = [ctypes.c_int64(n), ctypes.c_int64(nf),
            _dev(owner, torch.int32, nf, "owner"), _dev(neighbour, torch.int32, nf, "neighbour"),
            _dev(diag, torch.float64, n, "diag"), _dev(upper, torch.float64, nf, "upper"),
            _dev(lower, torch.float64, nf, "lower")]
    aopts = AmgOpts(max_coarse, max_levels, lanes_per_row)
    h = _vp()
    st = lib().ldu_amg_create(*args, ctypes.byref(aopts), _stream(stream), ctypes.byref(h))
    _check(st, "ldu_amg_create", allow_not_converged=False)
    return LduAmg(h, n, diag.device)


def ldu_amg_destroy(M):
    M.close()


def ldu_amg_info(M):
    return M.info()


def ldu_amg_aggregates(M, level=0):
    """Aggregate number of every row of a level (host int32 numpy array)."""
    import numpy as np
    rows = M.info()["rows"]
    if not 0 <= level < len(rows) - 1:
        raise ValueError(f"level {level} has no prolongator")
    out = np.zeros(rows[level], dtype=np.int32)
    _check(lib().ldu_amg_aggregates(M.handle, int(level), _vp(out.ctypes.data)),
           "ldu_amg_aggregates", allow_not_converged=False)
    return out


def ldu_amg_vcycle(M, b, x=None, stream=None):
    """x = V(b), one V(1,1) cycle from zero, in b's precision (float64 or float32)."""
    if b.dtype not in (torch.float64, torch.float32):
        raise ValueError("b must be float64 or float32")
    if x is None:
        x = torch.empty_like(b)
    prec = FP64 if b.dtype == torch.float64 else FP32
    st = lib().ldu_amg_vcycle(M.handle, prec, _dev(b, b.dtype, M.n, "b"),
                              _dev(x, b.dtype, M.n, "x"), _stream(stream))
    _check(st, "ldu_amg_vcycle", allow_not_converged=False)
    return x


def amg_pcg_solve(M, b, x=None, tol=1e-8, maxit=500, precision="fp64", stream=None, check=True):
    """AMG-preconditioned CG (precision "fp64" or "mixed"); returns
    (x, iters, relres, status)."""
    if x is None:
        x = torch.zeros_like(b)
    prec = {"fp64": FP64, "mixed": MIXED}[precision]
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().amg_pcg_solve(M.handle, _dev(b, torch.float64, M.n, "b"),
                             _dev(x, torch.float64, M.n, "x"), float(tol), int(maxit), prec,
                             ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(st, "amg_pcg_solve")
    return x, it.value, rr.value, st


def amg_pipecg_solve(M, b, x=None, tol=1e-8, maxit=500, stream=None, check=True):
    """Pipelined AMG-preconditioned CG (FP64 cycle); returns (x, iters, relres, status)."""
    if x is None:
        x = torch.zeros_like(b)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().amg_pipecg_solve(M.handle, _dev(b, torch.float64, M.n, "b"),
                                _dev(x, torch.float64, M.n, "x"), float(tol), int(maxit),
                                ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(st, "amg_pipecg_solve")
    return x, it.value, rr.value, st


def amg_from_system(sys_, device="cuda", **opts):
    """Upload an ldu_cases.LduSystem and build its AMG hierarchy."""
    t = lambda a, dt: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()  # noqa: E731
    return ldu_amg_create(sys_.n, t(sys_.owner, torch.int32), t(sys_.neighbour, torch.int32),
                          t(sys_.diag, torch.float64), t(sys_.upper, torch.float64),
                          t(sys_.lower, torch.float64), **opts)


# ---- batches ----------------------------------------------------------------

def ldu_create_batched(sizes, face_counts, owner, neighbour, diag, upper, lower, slice_rows=0,
                       block_threads=0, blocks_per_sm=0, staging=0, min_slices=0,
                       stream=None):
    """Batched handle from concatenated device arrays (face indices local to
    their system).  sizes / face_counts: per-system cells and faces."""
    import numpy as np
    nsys = len(sizes)
    n_h = np.ascontiguousarray(sizes, dtype=np.int64)
    f_h = np.ascontiguousarray(face_counts, dtype=np.int64)
    n_tot, f_tot = int(n_h.sum()), int(f_h.sum())
    opts = LduOpts(slice_rows, block_threads, blocks_per_sm, staging, min_slices)
    h = _vp()
    st = lib().ldu_create_batched(
        nsys, _vp(n_h.ctypes.data), _vp(f_h.ctypes.data), _dev(owner, torch.int32, f_tot, "owner"),
        _dev(neighbour, torch.int32, f_tot, "neighbour"), _dev(diag, torch.float64, n_tot, "diag"),
        _dev(upper, torch.float64, f_tot, "upper"), _dev(lower, torch.float64, f_tot, "lower"),
        ctypes.byref(opts), _stream(stream), ctypes.byref(h))
    _check(st, "ldu_create_batched", allow_not_converged=False)
    A = LduMatrix(h, n_tot, f_tot, diag.device)
    A.nsys = nsys
    A.sizes = n_h.copy()
    return A


def from_systems(systems, device="cuda", **opts):
    """Upload a list of ldu_cases.LduSystem and create one batched handle."""
    import numpy as np
    cat = lambda name, dt: torch.as_tensor(  # noqa: E731
        np.concatenate([getattr(s_, name) for s_ in systems])).to(device=device, dtype=dt)
    return ldu_create_batched([s_.n for s_ in systems], [s_.nfaces for s_ in systems],
                              cat("owner", torch.int32), cat("neighbour", torch.int32),
                              cat("diag", torch.float64), cat("upper", torch.float64),
                              cat("lower", torch.float64), **opts)


def ldu_batch_schedule(A, max_team=0, team_work_scale=0.0, stream=None):
    o = BatchOpts(int(max_team), float(team_work_scale))
    _check(lib().ldu_batch_schedule(A.handle, ctypes.byref(o), _stream(stream)),
           "ldu_batch_schedule", allow_not_converged=False)


def ldu_batch_info(A):
    v = [ctypes.c_int(0) for _ in range(4)]
    _check(lib().ldu_batch_info(A.handle, *[ctypes.byref(t) for t in v]), "ldu_batch_info")
    return dict(zip(("nsys", "grid_blocks", "ntasks", "max_team"), (t.value for t in v)))


def _pcg_opts(rr_period=0, tau=0.0, restart=False, deflate=False, barrier_timeout_s=0.0):
    return PcgOpts(int(rr_period), float(tau), int(bool(restart)), float(barrier_timeout_s), 0,
                   int(bool(deflate)))


def pcg_solve_batched_async(A, b, x, tol=1e-8, maxit=20000, precision="mixed", stream=None,
                            **opts):
    """Queue the batched solve (no synchronisation; graph-capturable)."""
    o = _pcg_opts(**opts)
    st = lib().pcg_solve_batched_async(A.handle, _dev(b, torch.float64, A.n, "b"),
                                       _dev(x, torch.float64, A.n, "x"), float(tol), int(maxit),
                                       _PREC[precision], ctypes.byref(o), _stream(stream))
    _check(st, "pcg_solve_batched_async", allow_not_converged=False)


def ldu_batch_results(A, stream=None):
    """(worst status, iters[nsys], relres[nsys], status[nsys]) of the last batched solve."""
    import numpy as np
    it = np.zeros(A.nsys, dtype=np.int32)
    rr = np.zeros(A.nsys, dtype=np.float64)
    stv = np.zeros(A.nsys, dtype=np.int32)
    worst = lib().ldu_batch_results(A.handle, _vp(it.ctypes.data), _vp(rr.ctypes.data),
                                    _vp(stv.ctypes.data), _stream(stream))
    return worst, it, rr, stv


def pcg_solve_batched(A, b, x=None, tol=1e-8, maxit=20000, precision="mixed", stream=None,
                      check=True, **opts):
    """Solve every system of a batched handle.  Returns
    (x, worst status, iters[nsys], relres[nsys], status[nsys])."""
    if x is None:
        x = torch.zeros(A.n, dtype=torch.float64, device=b.device)
    pcg_solve_batched_async(A, b, x, tol, maxit, precision, stream, **opts)
    worst, it, rr, stv = ldu_batch_results(A, stream)
    if check:
        _check(worst, "pcg_solve_batched")
    return x, worst, it, rr, stv
