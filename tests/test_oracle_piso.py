"""Pins of the PISO pressure-stage oracle (oracle/piso.py) against what the
mathematics fixes: a two-cell case worked by hand, the divergence of a
circulating flux, divergence-free corrected fluxes, the pinned cell's zero
pressure, idempotence of the projection, and the correction's orthogonality
to divergence-free fields.  Any sign slip in the divergence, the right-hand
side or the correction leaves a non-zero divergence and fails."""
import numpy as np
import pytest

import ldu_cases as lc
from ldu_cases import configs, rng
from oracle import piso


def pressure_case(s=10, seed=3):
    sys_ = configs.config3(s=s, seed=seed)
    phi = rng.uniform(rng.stream_base(seed, "piso-flux"), sys_.owner.shape[0], -1.0, 1.0)
    return sys_, phi


def face_index(s):
    return {(int(o), int(n)): f for f, (o, n) in enumerate(zip(s.owner, s.neighbour))}


def circulation(s, nx, ny, i, j, k):
    """A unit flux circulating around the z-edge shared by cells (i,j),
    (i+1,j), (i+1,j+1), (i,j+1) of plane k: divergence free."""
    c = lambda a, b: a + nx * (b + ny * k)  # noqa: E731
    fi = face_index(s)
    psi = np.zeros(s.owner.shape[0])
    psi[fi[(c(i, j), c(i + 1, j))]] += 1.0          # (i,j) -> (i+1,j)
    psi[fi[(c(i + 1, j), c(i + 1, j + 1))]] += 1.0  # (i+1,j) -> (i+1,j+1)
    psi[fi[(c(i, j + 1), c(i + 1, j + 1))]] -= 1.0  # (i+1,j+1) -> (i,j+1)
    psi[fi[(c(i, j), c(i, j + 1))]] -= 1.0          # (i,j+1) -> (i,j)
    return psi


def test_two_cells_by_hand():
    """Cells 0 and 1, one face with coefficient c and flux phi*; cell 0 is
    pinned (diagonal doubled).  A = [[2c, -c], [-c, c]], b = -div = [-phi*, phi*]
    gives p = (0, phi*/c) and the only divergence-free flux, 0."""
    c, phi_s = 2.5, 0.7
    s = lc.LduSystem(n=2, owner=np.array([0], np.int32), neighbour=np.array([1], np.int32),
                     diag=np.array([2 * c, c]), upper=np.array([-c]), lower=np.array([-c]),
                     b=np.zeros(2), coef=np.array([c]), diag_extra=np.array([c, 0.0]),
                     shape=(2, 1, 1), cell_of=np.arange(2), name="two", meta={})
    r = piso.pressure_step(s, s.coef, np.array([phi_s]), tol=1e-14)
    assert r.p == pytest.approx([0.0, phi_s / c], abs=1e-14)
    assert abs(r.phi[0]) <= 1e-14


def test_divergence_definition_and_sum():
    s, phi = pressure_case(6)
    div = piso.divergence(s.owner, s.neighbour, s.n, phi)
    assert abs(div.sum()) <= 1e-12 * np.abs(phi).sum()
    assert np.allclose(div, piso.divergence_fast(s.owner, s.neighbour, s.n, phi), atol=1e-14)
    # one face: +phi at its owner, -phi at its neighbour, nothing elsewhere
    one = np.zeros_like(phi)
    one[5] = 2.0
    d1 = piso.divergence(s.owner, s.neighbour, s.n, one)
    assert d1[s.owner[5]] == 2.0 and d1[s.neighbour[5]] == -2.0 and np.count_nonzero(d1) == 2


def test_circulating_flux_is_left_alone():
    s, _ = pressure_case(6)
    psi = circulation(s, 6, 6, 2, 3, 4)
    assert np.all(piso.divergence(s.owner, s.neighbour, s.n, psi) == 0.0)
    r = piso.pressure_step(s, s.coef, psi, tol=1e-12)
    assert np.max(np.abs(r.p)) == 0.0 and np.array_equal(r.phi, psi) and r.iters == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_corrected_flux_is_divergence_free(precision):
    s, phi = pressure_case(10)
    tol = 1e-10
    r = piso.pressure_step(s, s.coef, phi, tol=tol, precision=precision, deflate=True)
    assert r.status == 0
    div0 = piso.divergence(s.owner, s.neighbour, s.n, phi)
    div1 = piso.divergence(s.owner, s.neighbour, s.n, r.phi)
    # div(phi) = A p - b - d_0 p_0 e_0: the residual, and p_0 = 0 up to rounding
    assert np.linalg.norm(div1) <= 2 * tol * np.linalg.norm(div0)
    assert abs(r.p[0]) <= 1e-9 * np.max(np.abs(r.p))


def test_projection_is_idempotent_and_orthogonal():
    s, phi = pressure_case(8)
    r1 = piso.pressure_step(s, s.coef, phi, tol=1e-12)
    r2 = piso.pressure_step(s, s.coef, r1.phi, tol=1e-12)
    assert np.max(np.abs(r2.phi - r1.phi)) <= 1e-9 * np.max(np.abs(r1.phi))
    # phi - phi* = -c (G p) is orthogonal, in the 1/c-weighted face product,
    # to every divergence-free flux (discrete integration by parts)
    psi = circulation(s, 8, 8, 1, 5, 2) + 0.5 * circulation(s, 8, 8, 4, 4, 6)
    d = r1.phi - phi
    assert abs(np.sum(d * psi / s.coef)) <= 1e-12 * np.sum(np.abs(d * psi / s.coef)) + 1e-15


def test_warm_start_from_previous_pressure():
    """Two successive steps with slowly varying phi*: the second, started from
    the first's pressure, needs fewer iterations than from zero and reaches
    the same pressure."""
    s, phi = pressure_case(10)
    dphi = rng.uniform(rng.stream_base(7, "piso-dflux"), phi.shape[0], -1.0, 1.0)
    r1 = piso.pressure_step(s, s.coef, phi, tol=1e-10)
    phi2 = phi + 1e-3 * dphi
    warm = piso.pressure_step(s, s.coef, phi2, p0=r1.p, tol=1e-10)
    cold = piso.pressure_step(s, s.coef, phi2, tol=1e-10)
    assert warm.iters < cold.iters
    assert np.max(np.abs(warm.p - cold.p)) <= 1e-6 * np.max(np.abs(cold.p))


def test_stage_is_the_weighted_projection():
    """The corrected flux is the closed-form projection of phi* onto the
    divergence-free fluxes in the 1/c-weighted face product,
    phi = (I - C D^T (D C D^T)^+ D) phi*, with D the face-to-cell divergence
    matrix and C = diag(c): computed densely here, independently of the
    stage's solve-and-correct steps."""
    s, phi = pressure_case(6)
    F, n = s.owner.shape[0], s.n
    D = np.zeros((n, F))
    D[s.owner, np.arange(F)] = 1.0
    D[s.neighbour, np.arange(F)] = -1.0
    C = np.diag(s.coef)
    L = D @ C @ D.T                      # the unpinned Laplacian (singular: constants)
    # L^+ (D phi) by least squares (D phi sums to zero, so it lies in L's range)
    proj = phi - C @ D.T @ np.linalg.lstsq(L, D @ phi, rcond=None)[0]
    r = piso.pressure_step(s, s.coef, phi, tol=1e-13)
    assert np.max(np.abs(r.phi - proj)) <= 1e-9 * np.max(np.abs(proj))
    assert np.max(np.abs(D @ proj)) <= 1e-10 * np.max(np.abs(D @ phi))
