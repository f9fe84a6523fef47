"""The oracle: plain FP64 CPU reference of the LDU Jacobi / pipelined PCG path.

TEST INFRASTRUCTURE ONLY -- imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path; the two meet only in the seeded inputs of `ldu_cases`.

Routines (C source in ldu_oracle.c, each citing what it restates):
  spmv, pcg, pipecg, mixed_pipecg, face_grad, value_grad, harmonic_coeffs, harmonic_grad,
  lu_solve, true_relres
plus `lanczos_cond` (the condition number estimate of M^-1 A from CG's own
coefficients), and two plain numpy helpers, `dense` (the LDU matrix written
out densely) and `matrix_from_coef` (the FVM matrix of a set of face
coefficients).  `pcg(..., omp=True)` runs the same Jacobi-PCG from the
OpenMP build of the source on every host core (`threads()` says how many).
"""
import ctypes
import os

import numpy as np

from . import build_oracle

OK, NOT_CONVERGED, BAD_ARG, NOT_SPD, OOM = 0, 1, -1, -3, -6

_libs = {}
_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)


def lib(omp=False):
    if omp not in _libs:
        L = ctypes.CDLL(build_oracle.build(omp=omp))
        _libs[omp] = L
        i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        pint = ctypes.POINTER(c_int)
        mat = [i64, i64, _i32, _i32, _d, _d, _d]
        L.or_spmv.argtypes = mat + [_d, _d]
        L.or_spmv.restype = None
        L.or_true_relres.argtypes = mat + [_d, _d]
        L.or_true_relres.restype = c_double
        L.or_pcg.argtypes = mat + [_d, _d, c_double, c_int, c_int, pint, _d, _d, _d]
        L.or_pcg.restype = c_int
        L.or_pipecg.argtypes = mat + [_d, _d, c_double, c_int, c_int, pint, _d, _d]
        L.or_pipecg.restype = c_int
        L.or_mixed_pipecg.argtypes = mat + [_d, _d, c_double, c_int, c_double, c_int, c_int,
                                            c_int, pint, pint, _d]
        L.or_mixed_pipecg.restype = c_int
        L.or_mixed_pipecg_ex.argtypes = L.or_mixed_pipecg.argtypes + [c_int, _d, c_int, pint]
        L.or_mixed_pipecg_ex.restype = c_int
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
        L.or_threads.argtypes = []
        L.or_threads.restype = c_int
        L.or_set_threads.argtypes = [c_int]
        L.or_set_threads.restype = None
        if omp and "OMP_NUM_THREADS" not in os.environ:
            L.or_set_threads(host_cores())
    return _libs[omp]


def host_cores():
    """CPUs this process may really use: the affinity mask, capped by a
    cgroup CPU quota (a container can see more CPUs than its quota lets it
    run at once, and OpenMP threads beyond the quota only wait on each
    other)."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    quota = None
    try:
        with open("/sys/fs/cgroup/cpu.max") as f:
            q, period = f.read().split()[:2]
            if q != "max":
                quota = int(q) / int(period)
    except (OSError, ValueError):
        try:
            with open("/sys/fs/cgroup/cpu/cpu.cfs_quota_us") as f:
                q = int(f.read())
            with open("/sys/fs/cgroup/cpu/cpu.cfs_period_us") as f:
                period = int(f.read())
            if q > 0:
                quota = q / period
        except (OSError, ValueError):
            pass
    if quota is not None:
        n = min(n, max(1, int(quota)))
    return max(1, int(n or 1))


def threads(omp=False):
    """Host threads the Jacobi-PCG of that build uses (1 for the plain build)."""
    return int(lib(omp).or_threads())


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


def pcg(s, b=None, x0=None, tol=1e-8, maxit=20000, jacobi=True, history=False, coeffs=False,
        omp=False):
    """Jacobi-preconditioned CG (jacobi=False: plain CG).  coeffs=True also
    returns CG's alpha_k and beta_k (Result.alpha, Result.beta; beta_k = 0
    where the search restarted).  omp=True: the OpenMP build (all host cores)."""
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = np.zeros(s.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan) if history else None
    ab = np.zeros(2 * max(maxit, 1)) if coeffs else None
    st = lib(omp).or_pcg(*args, _p(b), _p(x), tol, maxit, int(bool(jacobi)), ctypes.byref(it),
                         ctypes.byref(rr), _p(hist) if history else None,
                         _p(ab) if coeffs else None)
    kw = {}
    if coeffs:
        kw = dict(alpha=ab[0:2 * it.value:2].copy(), beta=ab[1:2 * it.value:2].copy())
    return Result(x, st, it.value, rr.value, hist, **kw)


def lanczos_cond(s, b=None, tol=1e-10, maxit=20000, jacobi=True, omp=False):
    """(kappa, lambda_min, lambda_max): extreme eigenvalue estimates of M^-1 A
    (M = diag(A); jacobi=False: of A) from the Lanczos tridiagonal matrix that
    CG builds implicitly (Saad, Iterative Methods, Sec. 6.7.3); see
    cond_from_coeffs."""
    r = pcg(s, b=b, tol=tol, maxit=maxit, jacobi=jacobi, coeffs=True, omp=omp)
    return cond_from_coeffs(r.alpha, r.beta)


def cond_from_coeffs(alpha, beta):
    """(kappa, lambda_min, lambda_max) from CG's alpha_k and beta_k: the
    Lanczos tridiagonal matrix
        T[k, k]     = 1/alpha_k + beta_(k-1)/alpha_(k-1)   (beta_(-1) = 0)
        T[k, k + 1] = sqrt(beta_k) / alpha_k
    has Ritz values that approach the extreme eigenvalues of M^-1 A from
    inside as CG proceeds.  Only the steps before the first restart
    (beta_k = 0) are used: a restart begins a new Lanczos sequence."""
    from scipy.linalg import eigh_tridiagonal
    a, bt = np.asarray(alpha, float), np.asarray(beta, float)
    k = len(a)
    cut = np.flatnonzero(bt[:k - 1] == 0.0)
    if cut.size:
        k = int(cut[0]) + 1
    a, bt = a[:k], bt[:k]
    diag = 1.0 / a
    diag[1:] += bt[:k - 1] / a[:k - 1]
    off = np.sqrt(bt[:k - 1]) / a[:k - 1]
    ev = eigh_tridiagonal(diag, off, eigvals_only=True)
    return float(ev[-1] / ev[0]), float(ev[0]), float(ev[-1])


def reference_solution(s, b=None, tol=4e-15, maxit=None, omp=True):
    """The tight FP64 reference x* = A^-1 b: Jacobi-PCG run to relative
    residual `tol` (4e-15: about where FP64 rounding of b - A x stops the
    true residual on these meshes, near 1e-15) or until it stagnates at the
    iteration cap.  Returns (x*, its true relres, kappa estimate of M^-1 A
    from the same run's Lanczos coefficients)."""
    maxit = maxit or max(20 * int(round(s.n ** (1.0 / 3.0))) + 200, 400)
    r = pcg(s, b=b, tol=tol, maxit=maxit, coeffs=True, omp=omp)
    if r.status not in (OK, NOT_CONVERGED):
        raise RuntimeError(f"reference solve failed: {r}")
    return r.x, r.relres, cond_from_coeffs(r.alpha, r.beta)[0]


def accuracy_tol(kappa, target=1e-8, floor=1e-13):
    """Residual tolerance whose solutions have relative error <= target:
    ||x - x*|| / ||x*|| <= kappa ||b - A x|| / ||b||, so target / kappa,
    floored at 1e-13 (below it FP64 rounding of b - A x decides)."""
    return max(target / kappa, floor)


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
                 maxit=20000, deflate=False, sigma1=False, trace=False):
    """FP32 pipelined Jacobi-PCG with FP64 residual replacement every `period`
    iterations (and when gamma dropped by tau^2, or convergence is predicted);
    restart=True turns the replacements into classic defect-correction restarts.
    sigma1=True keeps the float unit at 1 (no power-of-two rescaling).
    trace=True also returns Result.trace, one row per event (see TRACE_*)."""
    args, keep = _mat(s)
    b = _f64(s.b if b is None else b)
    x = np.zeros(s.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    nrep = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    cap = 3 * maxit + 8 if trace else 0
    tr = np.zeros((cap, 6)) if trace else None
    ntr = ctypes.c_int(0)
    st = lib().or_mixed_pipecg_ex(*args, _p(b), _p(x), tol, period, tau, int(bool(restart)),
                                  int(bool(deflate)), maxit,
                                  ctypes.byref(it), ctypes.byref(nrep), ctypes.byref(rr),
                                  1 if sigma1 else 0, _p(tr) if trace else None, cap,
                                  ctypes.byref(ntr))
    kw = {"replacements": nrep.value}
    if trace:
        kw["trace"] = tr[:ntr.value].copy()
    return Result(x, st, it.value, rr.value, **kw)


# columns of mixed_pipecg's trace rows
TRACE_IT, TRACE_EVENT = 0, 1
TRACE_STEP_AP, TRACE_STEP_GRATIO, TRACE_STEP_DENOM = 2, 3, 4
TRACE_REP_PREDICTED, TRACE_REP_RELRES, TRACE_REP_WR, TRACE_REP_TRIGGER = 2, 3, 4, 5
TRIG_FORCED, TRIG_PERIOD, TRIG_TAU, TRIG_PREDICTED, TRIG_CAP = 1, 2, 4, 8, 16


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
