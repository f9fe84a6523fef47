"""Differentiable solve: x = A(c)^-1 b as a torch.autograd.Function.

A is the finite-volume matrix of face coefficients c (upper = lower = -c_f,
each c_f added to both adjacent diagonals) plus a fixed boundary part of the
diagonal (see ldu_set_face_coeffs).  For a loss L(x), with A symmetric, the
adjoint lambda solves A lambda = dL/dx with the same kernels as the forward
solve, and
    dL/db = lambda
    dL/dc_f = -(lambda_o - lambda_n)(x_o - x_n)      (ldu_face_grad)
    dL/d(diag_extra)_i = -lambda_i x_i               (ldu_diag_grad)
The handle may be a batched handle: b, x, c and diag_extra are then the
systems' arrays concatenated, and both solves are one batched launch.

ldu_solve_values is the same solve differentiable in the stored LDU values
themselves (diag, upper, lower; the forward values must be symmetric, as CG
needs), with dL/dA_ij = -lambda_i x_j: dL/ddiag_i = -lambda_i x_i
(ldu_diag_grad), dL/dupper_f = -lambda_o x_n, dL/dlower_f = -lambda_n x_o
(ldu_value_grad) -- the derivative also in non-symmetric directions.

harmonic_coeffs maps cell diffusivities k to (c, diag_extra) through the
harmonic-mean faces of the FVM Laplacian (ldu_harmonic_coeffs), with
    dL/dk_P = dL/d(diag_extra)_P bfac_P
              + sum over the faces f of P of dL/dc_f g_f 2 k_N^2 / (k_P + k_N)^2
in the library's kernel (ldu_harmonic_grad); composed with ldu_solve it
gives the gradient of a loss with respect to every cell's diffusivity.
"""
import torch

from . import ldupcg


def _solve(A, b, x, cfg):
    if getattr(A, "nsys", None) is not None:
        prec = "fp64" if cfg["precision"] in ("fp64", "pcg") else "mixed"
        ldupcg.pcg_solve_batched(A, b, x, tol=cfg["tol"], maxit=cfg["maxit"], precision=prec,
                                 check=cfg["check"], **cfg["kw"])
    elif cfg["precision"] in ("fp64", "pcg"):
        ldupcg.pcg_solve(A, b, x, tol=cfg["tol"], maxit=cfg["maxit"], check=cfg["check"])
    elif cfg["precision"] == "pipe":
        ldupcg.pipecg_solve(A, b, x, tol=cfg["tol"], maxit=cfg["maxit"], precision="fp64",
                            check=cfg["check"], **cfg["kw"])
    else:
        ldupcg.pipecg_solve(A, b, x, tol=cfg["tol"], maxit=cfg["maxit"], precision="mixed",
                            check=cfg["check"], **cfg["kw"])


class LduSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, diag_extra, b, A, cfg):
        coef = coef.detach().contiguous()
        diag_extra = diag_extra.detach().contiguous()
        ldupcg.ldu_set_face_coeffs(A, coef, diag_extra)
        x = torch.zeros_like(b)
        if cfg.get("x0") is not None:
            x.copy_(cfg["x0"])
        _solve(A, b.detach().contiguous(), x, cfg)
        ctx.save_for_backward(coef, diag_extra, x)
        ctx.A = A
        ctx.cfg = cfg
        return x

    @staticmethod
    def backward(ctx, gx):
        coef, diag_extra, x = ctx.saved_tensors
        A = ctx.A
        # the handle may have been re-valued by another forward since
        ldupcg.ldu_set_face_coeffs(A, coef, diag_extra)
        lam = torch.zeros_like(x)
        _solve(A, gx.detach().contiguous(), lam, ctx.cfg)
        g_coef = ldupcg.ldu_face_grad(A, lam, x) if ctx.needs_input_grad[0] else None
        g_extra = ldupcg.ldu_diag_grad(A, lam, x) if ctx.needs_input_grad[1] else None
        g_b = lam if ctx.needs_input_grad[2] else None
        return g_coef, g_extra, g_b, None, None


def ldu_solve(A, coef, diag_extra, b, precision="fp64", tol=1e-12, maxit=100000, x0=None,
              check=True, **kw):
    """x = A(coef, diag_extra)^-1 b, differentiable in coef, diag_extra and b.
    precision: 'fp64' (Jacobi-PCG), 'pipe' (FP64 pipelined) or 'mixed'."""
    cfg = dict(precision=precision, tol=tol, maxit=maxit, x0=x0, check=check, kw=kw)
    return LduSolve.apply(coef, diag_extra, b, A, cfg)


class LduSolveValues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, diag, upper, lower, b, A, cfg):
        diag = diag.detach().contiguous()
        upper = upper.detach().contiguous()
        lower = lower.detach().contiguous()
        if not torch.equal(upper, lower):
            raise ValueError("ldu_solve_values: CG needs symmetric values (upper == lower)")
        ldupcg.ldu_update_values(A, diag, upper, lower)
        x = torch.zeros_like(b)
        if cfg.get("x0") is not None:
            x.copy_(cfg["x0"])
        _solve(A, b.detach().contiguous(), x, cfg)
        ctx.save_for_backward(diag, upper, lower, x)
        ctx.A = A
        ctx.cfg = cfg
        return x

    @staticmethod
    def backward(ctx, gx):
        diag, upper, lower, x = ctx.saved_tensors
        A = ctx.A
        ldupcg.ldu_update_values(A, diag, upper, lower)
        lam = torch.zeros_like(x)
        _solve(A, gx.detach().contiguous(), lam, ctx.cfg)   # A^T = A
        g_diag = ldupcg.ldu_diag_grad(A, lam, x) if ctx.needs_input_grad[0] else None
        g_up = g_lo = None
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            g_up, g_lo = ldupcg.ldu_value_grad(A, lam, x)
        g_b = lam if ctx.needs_input_grad[3] else None
        return (g_diag, g_up if ctx.needs_input_grad[1] else None,
                g_lo if ctx.needs_input_grad[2] else None, g_b, None, None)


def ldu_solve_values(A, diag, upper, lower, b, precision="fp64", tol=1e-12, maxit=100000,
                     x0=None, check=True, **kw):
    """x = A^-1 b for the LDU values (diag, upper, lower), differentiable in
    all three and in b.  precision as ldu_solve."""
    cfg = dict(precision=precision, tol=tol, maxit=maxit, x0=x0, check=check, kw=kw)
    return LduSolveValues.apply(diag, upper, lower, b, A, cfg)


class HarmonicCoeffs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, g, bfac, A):
        k = k.detach().contiguous()
        g = g.detach().contiguous()
        bfac = bfac.detach().contiguous()
        coef, extra = ldupcg.ldu_harmonic_coeffs(A, k, g, bfac)
        ctx.save_for_backward(k, g, bfac)
        ctx.A = A
        return coef, extra

    @staticmethod
    def backward(ctx, g_coef, g_extra):
        k, g, bfac = ctx.saved_tensors
        if g_coef is None:
            g_coef = torch.zeros(ctx.A.nfaces, dtype=torch.float64, device=k.device)
        if g_extra is None:
            g_extra = torch.zeros_like(k)
        dk = ldupcg.ldu_harmonic_grad(ctx.A, k, g, bfac, g_coef.contiguous(),
                                      g_extra.contiguous())
        return dk, None, None, None


def harmonic_coeffs(A, k, g, bfac):
    """(coef, diag_extra) of cell diffusivities k, differentiable in k.
    g: geometric factor per internal face; bfac: Dirichlet-wall factor per cell."""
    return HarmonicCoeffs.apply(k, g, bfac, A)
