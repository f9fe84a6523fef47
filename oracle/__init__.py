"""The oracle: plain FP64 CPU reference of the LDU Jacobi / pipelined PCG path.

TEST INFRASTRUCTURE ONLY -- imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path; the two meet only in the seeded inputs of `ldu_cases`.

Routines (C source in ldu_oracle.c, each citing what it restates):
  spmv, pcg, pipecg, mixed_pipecg, face_grad, value_grad, harmonic_coeffs, harmonic_grad,
  lu_solve, true_relres
plus two plain numpy helpers, `dense` (the LDU matrix written out densely)
and `matrix_from_coef` (the FVM matrix of a set of face coefficients).
"""
import ctypes

import numpy as np

from . import build_oracle

OK, NOT_CONVERGED, BAD_ARG, NOT_SPD, OOM = 0, 1, -1, -3, -6

_lib = None
_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle.build())
        L = _lib
        i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        pint = ctypes.POINTER(c_int)
        mat = [i64, i64, _i32, _i32, _d, _d, _d]
        L.or_spmv.argtypes = mat + [_d, _d]
        L.or_spmv.restype = None
        L.or_true_relres.argtypes = mat + [_d, _d]
        L.or_true_relres.restype = c_double
        L.or_pcg.argtypes = mat + [_d, _d, c_double, c_int, c_int, pint, _d, _d]
        L.or_pcg.restype = c_int
        L.or_pipecg.argtypes = mat + [_d, _d, c_double, c_int, c_int, pint, _d, _d]
        L.or_pipecg.restype = c_int
        L.or_mixed_pipecg.argtypes = mat + [_d, _d, c_double, c_int, c_double, c_int, c_int,
                                            c_int, pint, pint, _d]
        L.or_mixed_pipecg.restype = c_int
        L.or_face_grad.argtypes = [i64, _i32, _i32, _d, _d, _d]
        L.or_face_grad.restype = None
        L.or_value_grad.argtypes = [i64, i64, _i32, _i32, _d, _d, _d, _d, _d]
        L.or_value_grad.restype = None
        L.or_harmonic_coeffs.argtypes = [i64, i64, _i32, _i32, _d, _d, _d, _d, _d]
        L.or_harmonic_coeffs.restype = None
        L.or_harmonic_grad.argtypes = [i64, i64, _i32, _i32, _d, _d, _d, _d, _d, _d]
        L.or_harmonic_grad.restype = None
        L.or_lu_solve.argtypes = [i64, _d, _d]
        L.or_lu_solve.restype = c_int
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _mat(s, diag=None, upper=None, lower=None):
    ow = np.ascontiguousarray(s.owner, dtype=np.int32)
    nb = np.ascontiguousarray(s.neighbour, dtype=np.int32)
    dg = _f64(s.diag if diag is None else diag)
    up = _f64(s.upper if upper is None else upper)
    lo = _f64(s.lower if lower is None else lower)
    keep = (ow, nb, dg, up, lo)
    args = [ctypes.c_int64(s.n), ctypes.c_int64(ow.shape[0]), _p(ow, _i32), _p(nb, _i32),
            _p(dg), _p(up), _p(lo)]
    return args, keep


def spmv(s, x, **vals):
    """y = A x with A the system's LDU matrix (face loop, FP64)."""
    args, keep = _mat(s, **vals)
    x = _f64(x)
    y = np.empty(s.n)
    lib().or_spmv(*args, _p(x), _p(y))
    return y


def true_relres(s, x, b=None):
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = _f64(x)
    return float(lib().or_true_relres(*args, _p(b), _p(x)))


class Result:
    def __init__(self, x, status, iters, relres, hist=None, **kw):
        self.x, self.status, self.iters, self.relres, self.hist = x, status, iters, relres, hist
        self.__dict__.update(kw)

    def __repr__(self):
        return f"Result(status={self.status}, iters={self.iters}, relres={self.relres:.3e})"


def pcg(s, b=None, x0=None, tol=1e-8, maxit=20000, jacobi=True, history=False):
    """Jacobi-preconditioned CG (jacobi=False: plain CG)."""
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = np.zeros(s.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan) if history else None
    st = lib().or_pcg(*args, _p(b), _p(x), tol, maxit, int(bool(jacobi)), ctypes.byref(it),
                      ctypes.byref(rr), _p(hist) if history else None)
    return Result(x, st, it.value, rr.value, hist)


def pipecg(s, b=None, x0=None, tol=1e-8, maxit=20000, rr_period=0, history=False):
    """Pipelined Jacobi-PCG with residual replacement."""
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = np.zeros(s.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan) if history else None
    st = lib().or_pipecg(*args, _p(b), _p(x), tol, maxit, rr_period, ctypes.byref(it),
                         ctypes.byref(rr), _p(hist) if history else None)
    return Result(x, st, it.value, rr.value, hist)


def mixed_pipecg(s, b=None, x0=None, tol=1e-8, period=12, tau=0.0, restart=False,
                 maxit=20000, deflate=False):
    """FP32 pipelined Jacobi-PCG with FP64 residual replacement every `period`
    iterations (and when gamma dropped by tau^2, or convergence is predicted);
    restart=True turns the replacements into classic defect-correction restarts."""
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = np.zeros(s.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    nrep = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().or_mixed_pipecg(*args, _p(b), _p(x), tol, period, tau, int(bool(restart)),
                               int(bool(deflate)), maxit,
                               ctypes.byref(it), ctypes.byref(nrep), ctypes.byref(rr))
    return Result(x, st, it.value, rr.value, replacements=nrep.value)


def face_grad(owner, neighbour, lam, x):
    """dL/dc_f = -(lambda_o - lambda_n)(x_o - x_n) per internal face."""
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    nb = np.ascontiguousarray(neighbour, dtype=np.int32)
    lam = _f64(lam)
    x = _f64(x)
    g = np.empty(ow.shape[0])
    lib().or_face_grad(ctypes.c_int64(ow.shape[0]), _p(ow, _i32), _p(nb, _i32), _p(lam), _p(x),
                       _p(g))
    return g


def value_grad(owner, neighbour, lam, x):
    """(ddiag, dupper, dlower): dL/dA_ij = -lambda_i x_j for every stored LDU value."""
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    nb = np.ascontiguousarray(neighbour, dtype=np.int32)
    lam = _f64(lam)
    x = _f64(x)
    dd = np.empty(x.shape[0])
    du = np.empty(ow.shape[0])
    dl = np.empty(ow.shape[0])
    lib().or_value_grad(ctypes.c_int64(x.shape[0]), ctypes.c_int64(ow.shape[0]), _p(ow, _i32),
                        _p(nb, _i32), _p(lam), _p(x), _p(dd), _p(du), _p(dl))
    return dd, du, dl


def harmonic_coeffs(owner, neighbour, k, g, bfac):
    """(coef, extra): c_f = g_f 2 k_o k_n / (k_o + k_n), extra_P = k_P bfac_P."""
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    nb = np.ascontiguousarray(neighbour, dtype=np.int32)
    k, g, bfac = _f64(k), _f64(g), _f64(bfac)
    coef = np.empty(ow.shape[0])
    extra = np.empty(k.shape[0])
    lib().or_harmonic_coeffs(ctypes.c_int64(k.shape[0]), ctypes.c_int64(ow.shape[0]),
                             _p(ow, _i32), _p(nb, _i32), _p(k), _p(g), _p(bfac), _p(coef),
                             _p(extra))
    return coef, extra


def harmonic_grad(owner, neighbour, k, g, bfac, dcoef, dextra):
    """dL/dk per cell from dL/dcoef and dL/dextra (chain rule of harmonic_coeffs)."""
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    nb = np.ascontiguousarray(neighbour, dtype=np.int32)
    k, g, bfac, dcoef, dextra = _f64(k), _f64(g), _f64(bfac), _f64(dcoef), _f64(dextra)
    dk = np.empty(k.shape[0])
    lib().or_harmonic_grad(ctypes.c_int64(k.shape[0]), ctypes.c_int64(ow.shape[0]),
                           _p(ow, _i32), _p(nb, _i32), _p(k), _p(g), _p(bfac), _p(dcoef),
                           _p(dextra), _p(dk))
    return dk


def lu_solve(A, b):
    """Dense partial-pivot LU solve (own code; tiny systems)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    st = lib().or_lu_solve(ctypes.c_int64(A.shape[0]), _p(A), _p(x))
    if st != OK:
        raise np.linalg.LinAlgError("singular matrix in oracle LU")
    return x


def dense(s, diag=None, upper=None, lower=None):
    """The LDU matrix written out as a dense array (tiny systems)."""
    A = np.zeros((s.n, s.n))
    A[np.arange(s.n), np.arange(s.n)] = s.diag if diag is None else diag
    A[s.owner, s.neighbour] = s.upper if upper is None else upper
    A[s.neighbour, s.owner] = s.lower if lower is None else lower
    return A


def matrix_from_coef(s, coef):
    """(diag, upper, lower) of the positive FVM matrix with face coefficients
    coef and the system's fixed boundary part diag_extra."""
    diag = np.array(s.diag_extra, dtype=np.float64, copy=True)
    np.add.at(diag, s.owner, coef)
    np.add.at(diag, s.neighbour, coef)
    return diag, -np.asarray(coef, float), -np.asarray(coef, float)
