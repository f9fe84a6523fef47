"""Pins of the oracle against what the mathematics and the paper fix.

Each pin is chosen so that a plausible slip in the oracle (a dropped face
term, upper and lower swapped, a wrong sign in alpha or beta, a transposed
axis, a missing restart) fails at least one of them:
  * closed-form eigenpairs of the uniform-grid operator on non-cubic grids;
  * plain CG: one step on an eigenvector, K steps on K eigenvectors;
  * a non-symmetric LDU matrix against brute force on a dense copy;
  * the solution of a dense LU solve (own code, itself checked against LAPACK);
  * pipelined PCG iterate-equivalent to PCG (Sec. 4.1: it reorders CG);
  * relabelling invariance; breakdown / cap / zero-rhs behaviour;
  * the adjoint face gradient against central finite differences;
  * Table 2 iteration magnitudes (soft).
"""
import json
import os

import numpy as np
import pytest

import ldu_cases as lc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- closed forms -----------------------------------------------------------

def eigpair(shape, m):
    """Eigenpair of the unit-diffusivity operator with Dirichlet x-walls and
    zero-gradient y/z walls on a uniform grid of the unit box.  Per axis the
    cell-centred 1-D operators are tridiag(-1, 2, -1) with end diagonals 3
    (Dirichlet at the wall face) or 1 (zero gradient); their eigenpairs are
    4 sin^2(m pi / 2N) with sin / cos (m pi (j + 1/2) / N).  The 3-D operator
    is sum_a (|S_a| / h_a) T_a, so eigenvalues add and eigenvectors multiply."""
    nx, ny, nz = shape
    mx, my, mz = m
    h = [1.0 / nx, 1.0 / ny, 1.0 / nz]
    cx = h[1] * h[2] / h[0]
    cy = h[0] * h[2] / h[1]
    cz = h[0] * h[1] / h[2]
    lam = (cx * 4 * np.sin(mx * np.pi / (2 * nx)) ** 2
           + cy * 4 * np.sin(my * np.pi / (2 * ny)) ** 2
           + cz * 4 * np.sin(mz * np.pi / (2 * nz)) ** 2)
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    vx = np.sin(mx * np.pi * (i + 0.5) / nx)
    vy = np.cos(my * np.pi * (j + 0.5) / ny)
    vz = np.cos(mz * np.pi * (k + 0.5) / nz)
    v = (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).ravel()
    return lam, v


SHAPES = [(5, 6, 7), (8, 8, 8), (7, 3, 4)]
MODES = [(1, 0, 0), (2, 1, 3), (5, 2, 0), (3, 2, 1)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", MODES)
def test_spmv_eigenvector(oracle_mod, shape, mode):
    mode = tuple(min(mi, si - (1 if a else 0)) for a, (mi, si) in enumerate(zip(mode, shape)))
    s = lc.poisson_box(*shape)
    lam, v = eigpair(shape, mode)
    y = oracle_mod.spmv(s, v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13 * max(lam, 1.0) * np.max(np.abs(v))


@pytest.mark.parametrize("shape", SHAPES)
def test_pcg_solves_eigen_rhs(oracle_mod, shape):
    lam, v = eigpair(shape, (2, 1, 1))
    s = lc.poisson_box(*shape)
    r = oracle_mod.pcg(s, b=lam * v, tol=1e-13)
    assert r.status == 0
    assert np.max(np.abs(r.x - v)) <= 1e-11


def test_plain_cg_one_step_on_eigenvector(oracle_mod):
    shape = (6, 5, 4)
    lam, v = eigpair(shape, (3, 2, 1))
    s = lc.poisson_box(*shape)
    r = oracle_mod.pcg(s, b=v, tol=1e-12, jacobi=False)
    assert r.status == 0 and r.iters == 1
    assert np.max(np.abs(r.x - v / lam)) <= 1e-12 * np.max(np.abs(v / lam))


def test_plain_cg_finite_termination(oracle_mod):
    shape = (6, 5, 4)
    s = lc.poisson_box(*shape)
    modes = [(1, 0, 0), (3, 2, 1), (6, 4, 3)]
    pairs = [eigpair(shape, m) for m in modes]
    lams = [p[0] for p in pairs]
    assert len(set(np.round(lams, 12))) == 3
    b = sum(v for _, v in pairs)
    x_exact = sum(v / lam for lam, v in pairs)
    r = oracle_mod.pcg(s, b=b, tol=1e-11, jacobi=False, history=True)
    assert r.status == 0 and r.iters == 3
    assert r.hist[2] > 1e-6                       # not converged one step early
    assert np.max(np.abs(r.x - x_exact)) <= 1e-10 * np.max(np.abs(x_exact))


def test_spmv_nonsymmetric_brute_force(oracle_mod):
    s = lc.poisson_box(4, 3, 5, diffusivity="lognormal")
    g = np.random.default_rng(1)
    up = g.uniform(-2, -0.1, s.nfaces)
    lo = g.uniform(-2, -0.1, s.nfaces)
    dg = g.uniform(5, 9, s.n)
    x = g.uniform(-1, 1, s.n)
    y = oracle_mod.spmv(s, x, diag=dg, upper=up, lower=lo)
    A = np.zeros((s.n, s.n))
    for f in range(s.nfaces):
        A[s.owner[f], s.neighbour[f]] += up[f]
        A[s.neighbour[f], s.owner[f]] += lo[f]
    for i in range(s.n):
        A[i, i] += dg[i]
    assert np.max(np.abs(y - A @ x)) <= 1e-13 * np.max(np.abs(A) @ np.abs(x))


# ---- against a direct solve ----------------------------------------------------

TINY = [
    lambda: lc.poisson_box(4, 5, 6, diffusivity="lognormal", seed=3),
    lambda: lc.config2(s=6, seed=1),
    lambda: lc.config3(s=6, seed=2),
]


def test_lu_matches_lapack(oracle_mod):
    s = TINY[0]()
    A = oracle_mod.dense(s)
    x = oracle_mod.lu_solve(A, s.b)
    ref = np.linalg.solve(A, s.b)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("make", TINY)
def test_pcg_matches_lu(oracle_mod, make):
    s = make()
    x_lu = oracle_mod.lu_solve(oracle_mod.dense(s), s.b)
    r = oracle_mod.pcg(s, tol=1e-14, maxit=10 * s.n)
    assert r.status == 0 and r.relres <= 1e-14
    assert np.linalg.norm(r.x - x_lu) <= 1e-11 * np.linalg.norm(x_lu)
    assert r.iters <= s.n                          # CG terminates within n steps


@pytest.mark.parametrize("make", TINY)
def test_pipecg_matches_lu(oracle_mod, make):
    s = make()
    x_lu = oracle_mod.lu_solve(oracle_mod.dense(s), s.b)
    r = oracle_mod.pipecg(s, tol=1e-13, maxit=10 * s.n)
    assert r.status == 0 and r.relres <= 1e-13
    assert np.linalg.norm(r.x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


@pytest.mark.parametrize("make", TINY)
@pytest.mark.parametrize("mode", [dict(period=16), dict(period=0, tau=1e-3, restart=True),
                                  dict(period=16, deflate=True)])
def test_mixed_reaches_fp64_accuracy(oracle_mod, make, mode):
    s = make()
    x_lu = oracle_mod.lu_solve(oracle_mod.dense(s), s.b)
    r = oracle_mod.mixed_pipecg(s, tol=1e-12, **mode)
    assert r.status == 0 and r.relres <= 1e-12
    assert r.replacements >= 3                     # FP32 alone cannot reach 1e-12
    assert np.linalg.norm(r.x - x_lu) <= 1e-9 * np.linalg.norm(x_lu)


def test_mixed_keeps_fp64_iteration_count(oracle_mod):
    """Replacing the residual without restarting keeps the convergence of the
    FP64 method; restarting (defect correction) loses it."""
    s = lc.config2(s=16)
    ref = oracle_mod.pcg(s, tol=1e-8)
    rel = oracle_mod.mixed_pipecg(s, tol=1e-8, period=16)
    rst = oracle_mod.mixed_pipecg(s, tol=1e-8, period=0, tau=1e-3, restart=True)
    assert rel.status == 0 and rst.status == 0
    assert rel.relres <= 1e-8 and rst.relres <= 1e-8
    assert rel.iters <= 1.1 * ref.iters + 2
    assert rst.iters > rel.iters


def test_deflation_removes_the_pressure_mode(oracle_mod):
    """On the pure-Neumann pressure case (one pinned cell) the constant vector
    is a near-null mode; deflating it must cut the iteration count and still
    give the FP64 solution."""
    s = lc.config3(s=16)
    plain = oracle_mod.mixed_pipecg(s, tol=1e-10, period=16)
    defl = oracle_mod.mixed_pipecg(s, tol=1e-10, period=16, deflate=True)
    assert plain.status == 0 and defl.status == 0 and defl.relres <= 1e-10
    assert defl.iters <= 0.7 * plain.iters
    xs = oracle_mod.pcg(s, tol=1e-13).x
    assert np.linalg.norm(defl.x - xs) <= 1e-6 * np.linalg.norm(xs)


# ---- pipelined == PCG, relabelling, edge cases -----------------------------------

@pytest.mark.parametrize("make", [lambda: lc.config1(s=16), lambda: lc.config2(s=14),
                                  lambda: lc.config3(s=12)])
def test_pipelined_iterate_equivalent(oracle_mod, make):
    s = make()
    a = oracle_mod.pcg(s, tol=1e-8)
    b = oracle_mod.pipecg(s, tol=1e-8)
    assert a.status == 0 and b.status == 0
    assert abs(a.iters - b.iters) <= 0.02 * a.iters + 2
    assert a.relres <= 1e-8 and b.relres <= 1e-8
    xs = oracle_mod.pcg(s, tol=1e-13).x
    for r in (a, b):
        assert np.linalg.norm(r.x - xs) <= 1e-4 * np.linalg.norm(xs)


def test_relabelling_invariance(oracle_mod):
    s0 = lc.config2(s=12, reorder=False)
    s1 = lc.config2(s=12, reorder=True)
    a = oracle_mod.pcg(s0, tol=1e-10)
    b = oracle_mod.pcg(s1, tol=1e-10)
    assert abs(a.iters - b.iters) <= 2
    xa = oracle_mod.pcg(s0, tol=1e-14).x
    xb = oracle_mod.pcg(s1, tol=1e-14).x
    assert np.max(np.abs(xb - xa[s1.cell_of])) <= 1e-11 * np.max(np.abs(xa))


def test_zero_rhs_and_warm_start(oracle_mod):
    s = lc.config1(s=6)
    for f in (oracle_mod.pcg, oracle_mod.pipecg, oracle_mod.mixed_pipecg):
        r = f(s, b=np.zeros(s.n), x0=np.ones(s.n))
        assert r.status == 0 and r.relres == 0.0 and np.all(r.x == 0)
    xs = oracle_mod.pcg(s, tol=1e-12).x
    for f in (oracle_mod.pcg, oracle_mod.pipecg):
        r = f(s, x0=xs, tol=1e-8)
        assert r.status == 0 and r.iters == 0


def test_iteration_cap_and_breakdown(oracle_mod):
    s = lc.config1(s=8)
    r = oracle_mod.pcg(s, maxit=5)
    assert r.status == 1 and r.iters == 5 and r.relres > 1e-8
    r = oracle_mod.pipecg(s, maxit=5)
    assert r.status == 1 and r.iters == 5
    import copy
    t = copy.copy(s)
    t.diag = -s.diag                                # -A: negative definite
    t.upper = -s.upper
    t.lower = -s.lower
    assert oracle_mod.pcg(t).status == -3
    assert oracle_mod.pipecg(t).status == -3
    t.upper = s.upper.copy()
    t.lower = s.lower.copy()
    t.diag = s.diag.copy()
    t.diag[: s.n // 2] *= -1.0                      # indefinite
    r = oracle_mod.pcg(t, maxit=500)
    assert r.status == -3


# ---- adjoint gradient -----------------------------------------------------------

def test_face_gradient_matches_finite_differences(oracle_mod):
    s = lc.poisson_box(3, 4, 5, diffusivity="lognormal", seed=7)
    g = np.random.default_rng(0)
    x_t = g.uniform(-1, 1, s.n)
    coef = s.coef.copy()

    def solve(c, b):
        d, u, lo = oracle_mod.matrix_from_coef(s, c)
        return oracle_mod.lu_solve(oracle_mod.dense(s, d, u, lo), b)

    def loss(c, b):
        x = solve(c, b)
        return 0.5 * np.sum((x - x_t) ** 2), x

    L0, x = loss(coef, s.b)
    d, u, lo = oracle_mod.matrix_from_coef(s, coef)
    assert np.allclose(d, s.diag, rtol=1e-14)
    lam = oracle_mod.lu_solve(oracle_mod.dense(s, d, u, lo).T, x - x_t)
    grad_c = oracle_mod.face_grad(s.owner, s.neighbour, lam, x)
    h = 1e-6
    fd_c = np.empty(s.nfaces)
    for f in range(s.nfaces):
        cp = coef.copy()
        cm = coef.copy()
        cp[f] += h
        cm[f] -= h
        xp = solve(cp, s.b)
        xm = solve(cm, s.b)
        fd_c[f] = 0.5 * np.sum((xp - xm) * (xp + xm - 2 * x_t)) / (2 * h)
    assert np.max(np.abs(fd_c - grad_c)) <= 1e-5 * np.max(np.abs(grad_c))
    fd_b = np.empty(s.n)
    for i in range(s.n):
        bp = s.b.copy()
        bm = s.b.copy()
        bp[i] += h
        bm[i] -= h
        xp = solve(coef, bp)
        xm = solve(coef, bm)
        fd_b[i] = 0.5 * np.sum((xp - xm) * (xp + xm - 2 * x_t)) / (2 * h)
    assert np.max(np.abs(fd_b - lam)) <= 1e-5 * np.max(np.abs(lam))


def test_harmonic_coeffs_match_the_assembly(oracle_mod):
    """The oracle's map from cell diffusivities to face coefficients and
    wall terms reproduces the generator's assembly of the same box."""
    s = lc.poisson_box(6, 5, 4, diffusivity="lognormal", seed=11)
    coef, extra = oracle_mod.harmonic_coeffs(s.owner, s.neighbour, s.meta["k_cell"],
                                             s.meta["g_face"], s.meta["bfac"])
    assert np.allclose(coef, s.coef, rtol=1e-15, atol=0)
    assert np.allclose(extra, s.diag_extra, rtol=1e-15, atol=0)
    assert np.all(extra[s.diag_extra == 0] == 0)


def test_cell_diffusivity_gradient_matches_finite_differences(oracle_mod):
    """dL/dk_P through the harmonic-mean faces and the Dirichlet wall terms
    (adjoint solve, face gradient, chain rule) against central differences
    of L(k) = 0.5 ||x(k) - x_t||^2 with x(k) from a dense LU solve."""
    s = lc.poisson_box(3, 4, 3, diffusivity="lognormal", seed=12)
    k0, gf, bfac = s.meta["k_cell"], s.meta["g_face"], s.meta["bfac"]
    x_t = np.random.default_rng(3).uniform(-1, 1, s.n)

    def solve(k):
        coef, extra = oracle_mod.harmonic_coeffs(s.owner, s.neighbour, k, gf, bfac)
        diag = extra.copy()
        np.add.at(diag, s.owner, coef)
        np.add.at(diag, s.neighbour, coef)
        M = oracle_mod.dense(s, diag, -coef, -coef)
        return M, oracle_mod.lu_solve(M, s.b)

    M, x = solve(k0)
    lam = oracle_mod.lu_solve(M.T, x - x_t)
    dcoef = oracle_mod.face_grad(s.owner, s.neighbour, lam, x)
    dk = oracle_mod.harmonic_grad(s.owner, s.neighbour, k0, gf, bfac, dcoef, -lam * x)
    fd = np.empty(s.n)
    for i in range(s.n):
        h = 1e-6 * k0[i]
        kp, km = k0.copy(), k0.copy()
        kp[i] += h
        km[i] -= h
        xp, xm = solve(kp)[1], solve(km)[1]
        fd[i] = 0.5 * np.sum((xp - xm) * (xp + xm - 2 * x_t)) / (2 * h)
    assert np.max(np.abs(fd - dk)) <= 1e-5 * np.max(np.abs(dk))
    # a wall cell's derivative includes its wall term: dropping it is visible
    wall = np.flatnonzero(bfac > 0)
    no_wall = oracle_mod.harmonic_grad(s.owner, s.neighbour, k0, gf, np.zeros(s.n), dcoef,
                                       -lam * x)
    assert np.max(np.abs(no_wall[wall] - fd[wall])) > 1e-3 * np.max(np.abs(dk))


# ---- Table 2 magnitudes (soft) ---------------------------------------------------

def test_table2_plain_cg_magnitude(oracle_mod):
    ref = json.load(open(os.path.join(GOLDEN, "table2_iterations.json")))
    its = {}
    for nside in (32, 64):
        s = lc.poisson_box(nside, dirichlet=lc.ALL_WALLS)
        r = oracle_mod.pcg(s, tol=1e-8, jacobi=False)
        assert r.status == 0
        its[nside] = r.iters
    paper64 = ref["GPU CG"]["64"]
    assert 0.5 * paper64 <= its[64] <= 2.0 * paper64
    # iterations grow like the cube side (sqrt of the condition number):
    # the paper's 128/64 ratio is 636/325 = 1.96
    ratio = its[64] / its[32]
    assert 1.6 <= ratio <= 2.4


def test_value_gradient_matches_nonsymmetric_finite_differences(oracle_mod):
    """dL/dA_ij = -lambda_i x_j for upper, lower and diagonal entries taken
    one at a time, so every perturbation but the diagonal's makes A
    non-symmetric: central differences through the oracle's dense LU of the
    perturbed matrix (lambda from A^T).  The sum over a face's four entries
    reproduces the face-coefficient gradient."""
    s = lc.poisson_box(3, 3, 4, diffusivity="lognormal", seed=9)
    g = np.random.default_rng(1)
    x_t = g.uniform(-1, 1, s.n)
    base = oracle_mod.dense(s)

    def loss(A):
        x = oracle_mod.lu_solve(A, s.b)
        return x

    x = loss(base)
    lam = oracle_mod.lu_solve(base.T, x - x_t)
    dd, du, dl = oracle_mod.value_grad(s.owner, s.neighbour, lam, x)
    h = 1e-6

    def fd(i, j):
        Ap = base.copy()
        Am = base.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        xp, xm = loss(Ap), loss(Am)
        return 0.5 * np.sum((xp - xm) * (xp + xm - 2 * x_t)) / (2 * h)

    scale = max(np.max(np.abs(du)), np.max(np.abs(dl)), np.max(np.abs(dd)))
    for f in range(0, s.nfaces, 3):
        o, n = int(s.owner[f]), int(s.neighbour[f])
        assert abs(fd(o, n) - du[f]) <= 1e-5 * scale
        assert abs(fd(n, o) - dl[f]) <= 1e-5 * scale
    for i in range(0, s.n, 4):
        assert abs(fd(i, i) - dd[i]) <= 1e-5 * scale
    # c_f enters as upper = lower = -c_f and +c_f on both diagonals
    gc = oracle_mod.face_grad(s.owner, s.neighbour, lam, x)
    assert np.allclose(-du - dl + dd[s.owner] + dd[s.neighbour], gc, rtol=1e-12, atol=1e-15)
