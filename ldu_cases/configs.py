"""The five synthetic workloads, each parameterised by size so that the same
recipe also yields small cases.

1. laplacianFoam-style Poisson block: uniform s^3, unit diffusivity,
   Dirichlet 0 on the x-min/x-max walls, zero-gradient elsewhere,
   b ~ U[-1, 1].                                        (s = 32)
2. Same boundary conditions, per-cell diffusivity lognormal(0, 1) with
   harmonic-mean faces, cells randomly permuted then RCM-renumbered. (s = 128)
3. icoFoam-style pressure equation on a graded block (ratio 4 toward all
   walls), c_f = |S|/(|d| a_f) with a_P ~ U[0.5, 2], pure Neumann with cell 0
   pinned (diagonal doubled), b = divergence of a random face flux. (s = 256)
4. Many independent systems of the config-2 kind (no reordering) with cube
   sides drawn uniformly from [lo, hi].                  (512 systems, 8..48)
5. Differentiable case: s^3, a batch of lognormal diffusivity fields and a
   reference field for the target.                        (s = 64, batch 8)

Seeds select independent streams (see rng.TAGS); the same seed always gives
the same arrays on every machine.
"""
import numpy as np

from . import rng
from .mesh import (BoxGeometry, assemble, diffusion_coefficients, flux_divergence,
                   graded_widths, harmonic_factors, pressure_coefficients, uniform_widths)
from .reorder import random_order, rcm_order, renumber

X_WALLS = ((0, 0), (0, 1))
ALL_WALLS = tuple((a, s) for a in range(3) for s in range(2))


def poisson_box(nx, ny=None, nz=None, seed=0, sub=0, diffusivity="unit", sigma=1.0,
                dirichlet=X_WALLS, rhs="uniform", name="poisson"):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    geo = BoxGeometry(uniform_widths(nx), uniform_widths(ny), uniform_widths(nz))
    n = geo.n
    if diffusivity == "unit":
        k = np.ones(n)
    elif diffusivity == "lognormal":
        k = np.exp(sigma * rng.normal(rng.stream_base(seed, "diffusivity", sub), n))
    elif diffusivity == "ref_lognormal":
        k = np.exp(sigma * rng.normal(rng.stream_base(seed, "ref_diffusivity", sub), n))
    else:
        raise ValueError(diffusivity)
    coef, extra = diffusion_coefficients(geo, k, dirichlet)
    if isinstance(rhs, str) and rhs == "uniform":
        b = rng.uniform(rng.stream_base(seed, "rhs", sub), n, -1.0, 1.0)
    elif isinstance(rhs, str) and rhs == "zero":
        b = np.zeros(n)
    elif isinstance(rhs, str):
        raise ValueError(rhs)
    else:
        b = np.asarray(rhs, dtype=np.float64)
    s = assemble(geo, coef, extra, b, name=name,
                 meta=dict(seed=seed, sub=sub, diffusivity=diffusivity, dirichlet=dirichlet))
    s.meta["k_cell"] = k
    s.meta["g_face"], s.meta["bfac"] = harmonic_factors(geo, dirichlet)
    return s


def config1(s=32, seed=0):
    return poisson_box(s, seed=seed, name=f"poisson{s}^3-unit")


def config2(s=128, seed=0, reorder=True):
    sys_ = poisson_box(s, seed=seed, diffusivity="lognormal",
                       name=f"poisson{s}^3-lognormal-rcm")
    if reorder:
        sys_ = renumber(sys_, random_order(sys_.n, seed))
        sys_ = renumber(sys_, rcm_order(sys_))
    return sys_


def config3(s=256, seed=0, ratio=4.0):
    w = graded_widths(s, ratio)
    geo = BoxGeometry(w, w, w)
    aP = rng.uniform(rng.stream_base(seed, "aP"), geo.n, 0.5, 2.0)
    coef = pressure_coefficients(geo, aP)
    phi = rng.uniform(rng.stream_base(seed, "flux"), geo.owner.shape[0], -1.0, 1.0)
    b = flux_divergence(geo, phi)
    extra = np.zeros(geo.n)
    sys_ = assemble(geo, coef, extra, b, name=f"pressure{s}^3-graded",
                    meta=dict(seed=seed, ratio=ratio))
    # reference cell: double the pinned cell's diagonal (setReference-style)
    sys_.diag_extra = sys_.diag_extra.copy()
    sys_.diag_extra[0] += sys_.diag[0]
    sys_.diag = sys_.diag.copy()
    sys_.diag[0] *= 2.0
    sys_.meta["widths"] = w
    return sys_


def config4_sides(nsys=512, lo=8, hi=48, seed=0):
    return rng.integers(rng.stream_base(seed, "sides"), nsys, lo, hi)


def config4(nsys=512, lo=8, hi=48, seed=0):
    sides = config4_sides(nsys, lo, hi, seed)
    return [poisson_box(int(sd), seed=seed, sub=i, diffusivity="lognormal",
                        name=f"batch{i}-{int(sd)}^3") for i, sd in enumerate(sides)]


def config5(s=64, batch=8, seed=0):
    """Returns (systems, reference systems): member i has its own lognormal
    diffusivity and RHS; its target comes from the reference field."""
    systems = [poisson_box(s, seed=seed, sub=i, diffusivity="lognormal",
                           name=f"grad{s}^3-{i}") for i in range(batch)]
    refs = [poisson_box(s, seed=seed, sub=i, diffusivity="ref_lognormal",
                        rhs=systems[i].b, name=f"gradref{s}^3-{i}") for i in range(batch)]
    return systems, refs
