"""Oracle of the pressure stage of a PISO step (Sec. 2, icoFoam: the
pressure solution and the explicit correction that follows it), restated
plainly on the CPU.  TEST INFRASTRUCTURE ONLY (tests and the CPU baseline).

The momentum predictor leaves face fluxes phi* that are not divergence free.
The pressure stage, as this project reads it for an LDU system with face
coefficients c_f (the positive assembly: (A p)_P = sum over P's faces of
c_f (p_P - p_other), plus the reference-cell pin of the system):

  1. b = -div(phi*), the discrete divergence summing +phi_f over the faces a
     cell owns and -phi_f over the faces where it is the neighbour;
  2. solve A p = b with CG (the paper's pressure solver), starting from the
     previous pressure;
  3. correct the fluxes explicitly, phi_f = phi*_f - c_f (p_N - p_P), P the
     owner and N the neighbour of face f.

With these signs div(phi) = div(phi*) + A_L p (A_L the Laplacian without the
pin), which vanishes once A p = b, so the corrected fluxes are divergence
free to the solver's tolerance (the pinned cell's p is 0 because div sums to
zero over the cells).
"""
import numpy as np

from . import mixed_pipecg, pcg


def divergence(owner, neighbour, n, phi):
    """div_P = sum of phi over faces P owns - sum over faces where P is the neighbour."""
    div = np.zeros(n)
    for f in range(len(owner)):
        div[owner[f]] += phi[f]
        div[neighbour[f]] -= phi[f]
    return div


def divergence_fast(owner, neighbour, n, phi):
    """The same sum through numpy's unbuffered scatter (large systems)."""
    div = np.zeros(n)
    np.add.at(div, owner, phi)
    np.add.at(div, neighbour, -np.asarray(phi))
    return div


def flux_correct(owner, neighbour, coef, phi, p):
    """phi_f - c_f (p_N - p_P)."""
    return np.asarray(phi, float) - np.asarray(coef, float) * (p[neighbour] - p[owner])


class Result:
    def __init__(self, p, phi, iters, relres, status):
        self.p, self.phi, self.iters, self.relres, self.status = p, phi, iters, relres, status


def pressure_step(s, coef, phi, p0=None, tol=1e-8, maxit=20000, precision="fp64",
                  deflate=False):
    """One pressure stage on system s (its matrix is the pressure matrix of
    the face coefficients coef): returns the new pressure and fluxes."""
    div = (divergence if s.n <= 20000 else divergence_fast)(s.owner, s.neighbour, s.n, phi)
    b = -div
    if precision == "fp64":
        r = pcg(s, b=b, x0=p0, tol=tol, maxit=maxit)
    else:
        r = mixed_pipecg(s, b=b, x0=p0, tol=tol, maxit=maxit, period=16, tau=0.3,
                         deflate=deflate)
    phi_new = flux_correct(s.owner, s.neighbour, coef, phi, r.x)
    return Result(r.x, phi_new, r.iters, r.relres, r.status)
