"""Differentiable solve: autograd gradients of L = 0.5 ||x(c, b) - x_t||^2
against the oracle's adjoint gradient and against central finite
differences of the loss.

Tolerances: gradients from the oracle's dense LU adjoint within 1e-8
(relative, tight solves); full-size members within 1e-6 of the oracle's
PCG adjoint; finite differences (h = 1e-6, loss difference formed as
0.5 sum (x+ - x-)(x+ + x- - 2 x_t) to avoid cancellation) within relative
1e-5, floor 1e-5 * max |grad|."""
import numpy as np
import pytest

import ldu_cases as lc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1505_07630_gb300 as p
    return p


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "pipe", "mixed"])
def test_gradients_match_oracle_adjoint(pkg, oracle_mod, precision):
    s = lc.poisson_box(6, 5, 4, diffusivity="lognormal", seed=3)
    A = pkg.from_system(s)
    xt = np.random.default_rng(0).uniform(-1, 1, s.n)
    coef = dev(s.coef).requires_grad_(True)
    extra = dev(s.diag_extra).requires_grad_(True)
    b = dev(s.b).requires_grad_(True)
    x = pkg.ldu_solve(A, coef, extra, b, precision=precision, tol=1e-13)
    loss = 0.5 * ((x - dev(xt)) ** 2).sum()
    loss.backward()
    d, u, lo = oracle_mod.matrix_from_coef(s, s.coef)
    M = oracle_mod.dense(s, d, u, lo)
    x_o = oracle_mod.lu_solve(M, s.b)
    lam = oracle_mod.lu_solve(M.T, x_o - xt)
    g_c = oracle_mod.face_grad(s.owner, s.neighbour, lam, x_o)
    for got, ref in ((coef.grad, g_c), (extra.grad, -lam * x_o), (b.grad, lam)):
        got = got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), precision
    A.close()


def test_finite_differences_small(pkg):
    s = lc.poisson_box(5, 4, 6, diffusivity="lognormal", seed=8)
    A = pkg.from_system(s)
    xt = dev(np.random.default_rng(1).uniform(-1, 1, s.n))
    coef = dev(s.coef).requires_grad_(True)
    b = dev(s.b).requires_grad_(True)
    extra = dev(s.diag_extra)
    x = pkg.ldu_solve(A, coef, extra, b, tol=1e-14)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    h = 1e-6
    rng = np.random.default_rng(2)

    def dloss(c, bb):
        with torch.no_grad():
            xp = pkg.ldu_solve(A, c[0], extra, bb[0], tol=1e-14, x0=x, check=False)
            xm = pkg.ldu_solve(A, c[1], extra, bb[1], tol=1e-14, x0=x, check=False)
            return float(0.5 * ((xp - xm) * (xp + xm - 2 * xt)).sum()) / (2 * h)

    gc = coef.grad.cpu().numpy()
    for f in rng.choice(s.nfaces, 10, replace=False):
        cp, cm = coef.detach().clone(), coef.detach().clone()
        cp[f] += h
        cm[f] -= h
        fd = dloss((cp, cm), (b.detach(), b.detach()))
        assert abs(fd - gc[f]) <= 1e-5 * max(abs(gc[f]), np.abs(gc).max()), (f, fd, gc[f])
    gb = b.grad.cpu().numpy()
    for i in rng.choice(s.n, 10, replace=False):
        bp, bm = b.detach().clone(), b.detach().clone()
        bp[i] += h
        bm[i] -= h
        fd = dloss((coef.detach(), coef.detach()), (bp, bm))
        assert abs(fd - gb[i]) <= 1e-5 * max(abs(gb[i]), np.abs(gb).max()), (i, fd, gb[i])
    A.close()


def test_config5_batch_of_8(pkg, oracle_mod):
    """64^3 mesh, batch of 8 lognormal fields, targets from a reference field
    (oracle solves), one batched handle for forward and adjoint; oracle
    adjoint on two members; finite differences on 20 faces and 20 RHS
    entries of the whole batch."""
    systems, refs = lc.config5()
    A = pkg.from_systems(systems)
    xt_np = [oracle_mod.pcg(r, tol=1e-10).x for r in refs]
    xt = dev(np.concatenate(xt_np))
    coef = dev(np.concatenate([s.coef for s in systems])).requires_grad_(True)
    extra = dev(np.concatenate([s.diag_extra for s in systems]))
    b = dev(np.concatenate([s.b for s in systems])).requires_grad_(True)
    x = pkg.ldu_solve(A, coef, extra, b, tol=1e-13)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    gc = coef.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()
    n, F = systems[0].n, systems[0].nfaces
    for m in (0, 5):
        s = systems[m]
        xo = oracle_mod.pcg(s, tol=1e-13).x
        lam = oracle_mod.pcg(s, b=xo - xt_np[m], tol=1e-13).x
        ref_c = oracle_mod.face_grad(s.owner, s.neighbour, lam, xo)
        got_c = gc[m * F:(m + 1) * F]
        assert np.linalg.norm(got_c - ref_c) <= 1e-6 * np.linalg.norm(ref_c), m
        got_b = gb[m * n:(m + 1) * n]
        assert np.linalg.norm(got_b - lam) <= 1e-6 * np.linalg.norm(lam), m
    h = 1e-6
    rng = np.random.default_rng(5)

    def dloss(c, bb):
        with torch.no_grad():
            xp = pkg.ldu_solve(A, c[0], extra, bb[0], tol=1e-14, x0=x, check=False)
            xm = pkg.ldu_solve(A, c[1], extra, bb[1], tol=1e-14, x0=x, check=False)
            return float(0.5 * ((xp - xm) * (xp + xm - 2 * xt)).sum()) / (2 * h)

    for f in rng.choice(coef.numel(), 20, replace=False):
        cp, cm = coef.detach().clone(), coef.detach().clone()
        cp[f] += h
        cm[f] -= h
        fd = dloss((cp, cm), (b.detach(), b.detach()))
        assert abs(fd - gc[f]) <= 1e-5 * max(abs(gc[f]), np.abs(gc).max()), (f, fd, gc[f])
    for i in rng.choice(b.numel(), 20, replace=False):
        bp, bm = b.detach().clone(), b.detach().clone()
        bp[i] += h
        bm[i] -= h
        fd = dloss((coef.detach(), coef.detach()), (bp, bm))
        assert abs(fd - gb[i]) <= 1e-5 * max(abs(gb[i]), np.abs(gb).max()), (i, fd, gb[i])
    A.close()


# ---- gradient with respect to cell diffusivities (harmonic-mean faces) -----

def harmonic_inputs(systems):
    cat = lambda key: dev(np.concatenate([s.meta[key] for s in systems]))  # noqa: E731
    return cat("k_cell"), cat("g_face"), cat("bfac")


@pytest.mark.parametrize("batched", [False, True])
def test_harmonic_kernels_match_oracle(pkg, oracle_mod, batched):
    systems = [lc.poisson_box(7, 5, 6, diffusivity="lognormal", seed=21),
               lc.poisson_box(4, 9, 3, diffusivity="lognormal", seed=22, sub=1)]
    if not batched:
        systems = systems[:1]
    A = pkg.from_systems(systems) if batched else pkg.from_system(systems[0])
    k, g, bfac = harmonic_inputs(systems)
    coef, extra = pkg.ldu_harmonic_coeffs(A, k, g, bfac)
    rng = np.random.default_rng(4)
    dcoef_np = rng.standard_normal(coef.numel())
    dextra_np = rng.standard_normal(extra.numel())
    dk = pkg.ldu_harmonic_grad(A, k, g, bfac, dev(dcoef_np), dev(dextra_np))
    dk2 = pkg.ldu_harmonic_grad(A, k, g, bfac, dev(dcoef_np), dev(dextra_np))
    assert torch.equal(dk, dk2)                     # fixed summation order
    fo = co = 0
    for s in systems:
        c_ref, e_ref = oracle_mod.harmonic_coeffs(s.owner, s.neighbour, s.meta["k_cell"],
                                                  s.meta["g_face"], s.meta["bfac"])
        F, n = s.nfaces, s.n
        assert np.allclose(coef[fo:fo + F].cpu().numpy(), c_ref, rtol=1e-15, atol=0)
        assert np.allclose(extra[co:co + n].cpu().numpy(), e_ref, rtol=1e-15, atol=0)
        dk_ref = oracle_mod.harmonic_grad(s.owner, s.neighbour, s.meta["k_cell"],
                                          s.meta["g_face"], s.meta["bfac"],
                                          dcoef_np[fo:fo + F], dextra_np[co:co + n])
        got = dk[co:co + n].cpu().numpy()
        assert np.max(np.abs(got - dk_ref)) <= 1e-13 * np.max(np.abs(dk_ref))
        fo += F
        co += n
    A.close()


def test_cell_diffusivity_gradient_end_to_end(pkg, oracle_mod):
    """dL/dk of L = 0.5 ||x(k) - x_t||^2 through harmonic_coeffs and ldu_solve
    against the oracle's dense-LU adjoint and chain rule."""
    s = lc.poisson_box(6, 5, 4, diffusivity="lognormal", seed=23)
    A = pkg.from_system(s)
    k = dev(s.meta["k_cell"]).requires_grad_(True)
    g, bfac = dev(s.meta["g_face"]), dev(s.meta["bfac"])
    xt = np.random.default_rng(6).uniform(-1, 1, s.n)
    for precision in ("fp64", "mixed"):
        k.grad = None
        coef, extra = pkg.harmonic_coeffs(A, k, g, bfac)
        x = pkg.ldu_solve(A, coef, extra, dev(s.b), precision=precision, tol=1e-13)
        (0.5 * ((x - dev(xt)) ** 2).sum()).backward()
        M = oracle_mod.dense(s)
        xo = oracle_mod.lu_solve(M, s.b)
        lam = oracle_mod.lu_solve(M.T, xo - xt)
        dcoef = oracle_mod.face_grad(s.owner, s.neighbour, lam, xo)
        ref = oracle_mod.harmonic_grad(s.owner, s.neighbour, s.meta["k_cell"], s.meta["g_face"],
                                       s.meta["bfac"], dcoef, -lam * xo)
        got = k.grad.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), precision
    A.close()


def test_cell_diffusivity_gradient_finite_differences(pkg):
    """12^3 box: dL/dk on 10 random cells (walls included) against central
    differences of the GPU loss, relative step 1e-6."""
    s = lc.poisson_box(12, diffusivity="lognormal", seed=24)
    A = pkg.from_system(s)
    k0 = dev(s.meta["k_cell"])
    g, bfac = dev(s.meta["g_face"]), dev(s.meta["bfac"])
    xt = dev(np.random.default_rng(7).uniform(-1, 1, s.n))
    b = dev(s.b)
    k = k0.clone().requires_grad_(True)
    coef, extra = pkg.harmonic_coeffs(A, k, g, bfac)
    x = pkg.ldu_solve(A, coef, extra, b, tol=1e-14)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    gk = k.grad.cpu().numpy()

    def solve(kk):
        with torch.no_grad():
            c, e = pkg.ldu_harmonic_coeffs(A, kk, g, bfac)
            return pkg.ldu_solve(A, c, e, b, tol=1e-14, x0=x, check=False)

    rng = np.random.default_rng(8)
    wall = np.flatnonzero(s.meta["bfac"] > 0)
    cells = np.concatenate([rng.choice(s.n, 7, replace=False), rng.choice(wall, 3, replace=False)])
    for i in cells:
        h = 1e-6 * float(k0[i])
        kp, km = k0.clone(), k0.clone()
        kp[i] += h
        km[i] -= h
        xp, xm = solve(kp), solve(km)
        fd = float(0.5 * ((xp - xm) * (xp + xm - 2 * xt)).sum()) / (2 * h)
        assert abs(fd - gk[i]) <= 1e-5 * max(abs(gk[i]), np.abs(gk).max()), (i, fd, gk[i])
    A.close()


def test_value_grad_kernel_is_bit_exact(pkg, oracle_mod):
    s = lc.poisson_box(9, 7, 5, diffusivity="lognormal", seed=12)
    A = pkg.from_system(s)
    rng = np.random.default_rng(4)
    lam, x = rng.standard_normal(s.n), rng.standard_normal(s.n)
    gu, gl = pkg.ldu_value_grad(A, dev(lam), dev(x))
    _, ou, ol = oracle_mod.value_grad(s.owner, s.neighbour, lam, x)
    assert np.array_equal(gu.cpu().numpy(), ou) and np.array_equal(gl.cpu().numpy(), ol)
    A.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_value_gradients_match_oracle_adjoint(pkg, oracle_mod, precision):
    """ldu_solve_values: gradients with respect to diag, upper, lower (each
    entry independent, so including non-symmetric directions) and b, against
    the oracle's dense adjoint; the oracle's value gradient is itself pinned
    by non-symmetric finite differences."""
    s = lc.poisson_box(6, 5, 4, diffusivity="lognormal", seed=3)
    A = pkg.from_system(s)
    xt = np.random.default_rng(0).uniform(-1, 1, s.n)
    diag = dev(s.diag).requires_grad_(True)
    up = dev(s.upper).requires_grad_(True)
    lo = dev(s.lower).requires_grad_(True)
    b = dev(s.b).requires_grad_(True)
    x = pkg.ldu_solve_values(A, diag, up, lo, b, precision=precision, tol=1e-13)
    (0.5 * ((x - dev(xt)) ** 2).sum()).backward()
    M = oracle_mod.dense(s)
    x_o = oracle_mod.lu_solve(M, s.b)
    lam = oracle_mod.lu_solve(M.T, x_o - xt)
    gd, gu, gl = oracle_mod.value_grad(s.owner, s.neighbour, lam, x_o)
    for got, ref in ((diag.grad, gd), (up.grad, gu), (lo.grad, gl), (b.grad, lam)):
        got = got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), precision
    # the face-coefficient chain: c_f enters as upper = lower = -c_f and +c_f on both diagonals
    gc = oracle_mod.face_grad(s.owner, s.neighbour, lam, x_o)
    g = (-up.grad - lo.grad + diag.grad[torch.as_tensor(s.owner, device="cuda").long()]
         + diag.grad[torch.as_tensor(s.neighbour, device="cuda").long()]).cpu().numpy()
    assert np.linalg.norm(g - gc) <= 1e-8 * np.linalg.norm(gc)
    A.close()


def test_value_solve_refuses_nonsymmetric_values(pkg):
    s = lc.poisson_box(4, 4, 4, diffusivity="lognormal", seed=5)
    A = pkg.from_system(s)
    lo = dev(s.lower)
    lo[3] *= 1.01
    with pytest.raises(ValueError):
        pkg.ldu_solve_values(A, dev(s.diag), dev(s.upper), lo, dev(s.b))
    A.close()
