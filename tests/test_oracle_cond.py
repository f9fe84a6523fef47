"""Pins of the oracle's condition-number estimate and of its OpenMP build.

lanczos_cond reads the extreme eigenvalues of M^-1 A off the Lanczos
tridiagonal matrix that CG's alpha_k, beta_k define (Saad, Sec. 6.7.3); the
accuracy tests size their tolerance 1e-8 / kappa from it.  It is pinned to
the closed-form spectrum of the uniform-grid operator (plain CG, M = I) and
to a dense eigen-solve of the Jacobi-scaled matrix.  The OpenMP build of the
same source must give the plain build's Jacobi-PCG: bitwise with one thread
(each row adds its faces in the face loop's order), within rounding with
several.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import ldu_cases as lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def closed_form_extremes(shape):
    """Smallest and largest eigenvalue of the unit-diffusivity operator with
    Dirichlet x-walls and zero-gradient y/z walls: per axis 4 sin^2(m pi / 2N)
    weighted by |S_a|/h_a, m = 1..N along x and 0..N-1 along y and z."""
    nx, ny, nz = shape
    h = [1.0 / nx, 1.0 / ny, 1.0 / nz]
    cx, cy, cz = h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2]
    lo = cx * 4 * np.sin(np.pi / (2 * nx)) ** 2
    hi = (cx * 4 * np.sin(nx * np.pi / (2 * nx)) ** 2
          + cy * 4 * np.sin((ny - 1) * np.pi / (2 * ny)) ** 2
          + cz * 4 * np.sin((nz - 1) * np.pi / (2 * nz)) ** 2)
    return lo, hi


@pytest.mark.parametrize("shape", [(12, 10, 9), (16, 16, 16), (20, 6, 7)])
def test_lanczos_extremes_match_closed_form(oracle_mod, shape):
    s = lc.poisson_box(*shape)
    kappa, lmin, lmax = oracle_mod.lanczos_cond(s, tol=1e-12, jacobi=False)
    lo, hi = closed_form_extremes(shape)
    assert abs(lmin - lo) <= 1e-6 * lo, (lmin, lo)
    assert abs(lmax - hi) <= 1e-6 * hi, (lmax, hi)
    assert abs(kappa - hi / lo) <= 2e-6 * hi / lo


@pytest.mark.parametrize("make", [lambda: lc.poisson_box(7, 6, 5, diffusivity="lognormal", seed=3),
                                  lambda: lc.config2(s=8, seed=1),
                                  lambda: lc.config3(s=8, seed=2)])
def test_lanczos_jacobi_matches_dense_spectrum(oracle_mod, make):
    """Jacobi: the spectrum of M^-1 A is that of D^-1/2 A D^-1/2."""
    s = make()
    kappa, lmin, lmax = oracle_mod.lanczos_cond(s, tol=1e-13)
    A = oracle_mod.dense(s)
    d = 1.0 / np.sqrt(np.diag(A))
    ev = np.linalg.eigvalsh(d[:, None] * A * d[None, :])
    assert abs(lmin - ev[0]) <= 1e-6 * ev[0]
    assert abs(lmax - ev[-1]) <= 1e-6 * ev[-1]
    assert abs(kappa - ev[-1] / ev[0]) <= 3e-6 * ev[-1] / ev[0]


def test_lanczos_coefficients_are_cg_steps(oracle_mod):
    """alpha_k and beta_k are the step's own: one alpha per iteration, and the
    last beta is the ratio of successive (r, M^-1 r) CG would use next."""
    s = lc.config2(s=9)
    r = oracle_mod.pcg(s, tol=1e-10, coeffs=True)
    assert r.status == 0 and len(r.alpha) == r.iters and len(r.beta) == r.iters
    assert np.all(r.alpha > 0) and np.all(r.beta[:-1] > 0)
    plain = oracle_mod.pcg(s, tol=1e-10)
    assert np.array_equal(plain.x, r.x)            # recording changes nothing


def test_omp_build_matches_plain_build(oracle_mod):
    s = lc.config2(s=18)
    a = oracle_mod.pcg(s, tol=1e-10)
    b = oracle_mod.pcg(s, tol=1e-10, omp=True)
    assert oracle_mod.threads() == 1 and oracle_mod.threads(omp=True) >= 1
    assert a.status == b.status == 0
    assert abs(a.iters - b.iters) <= 1
    assert np.linalg.norm(a.x - b.x) <= 1e-9 * np.linalg.norm(a.x)


def test_omp_build_is_bitwise_the_plain_build_on_one_thread():
    """With one thread the OpenMP build's rows add their faces in the face
    loop's order and its sums run in index order: every operation of the
    solve is the plain build's, so the results agree bitwise, on faces in
    the generator's order and shuffled."""
    code = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
import ldu_cases as lc, oracle
s = lc.config2(s=11)
g = np.random.default_rng(5)
o = g.permutation(s.nfaces)
t = lc.LduSystem(n=s.n, owner=s.owner[o], neighbour=s.neighbour[o], diag=s.diag,
                 upper=s.upper[o], lower=s.lower[o], b=s.b, coef=s.coef[o],
                 diag_extra=s.diag_extra, shape=s.shape)
out = []
for sys_ in (s, t):
    a = oracle.pcg(sys_, tol=1e-11)
    b = oracle.pcg(sys_, tol=1e-11, omp=True)
    out.append([a.iters == b.iters, bool(np.array_equal(a.x, b.x)), a.relres == b.relres])
print(json.dumps({"threads": oracle.threads(omp=True), "same": out}))
""" % ROOT
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300, check=True)
    got = json.loads(res.stdout.strip().splitlines()[-1])
    assert got["threads"] == 1
    assert got["same"] == [[True, True, True], [True, True, True]]
