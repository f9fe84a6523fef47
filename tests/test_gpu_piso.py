"""Pressure stage of a PISO step (Sec. 2, icoFoam) through the C ABI
against oracle/piso.py.

Bars: b = -div(phi) is formed on the device in each cell's neighbour order
(at most six terms), so the pressure agrees with the oracle's within the
solve's tolerance-derived bound (1e-6 relative at tol 1e-10: the error of a
solve to relative residual tol is at most cond * tol) and the corrected
fluxes within the same bound; the corrected fluxes' divergence, recomputed by
the oracle, is at most 2 tol times the predicted fluxes' divergence (it
equals the solve's residual); a divergence-free input leaves the pressure at
zero and the fluxes bitwise unchanged."""
import numpy as np
import pytest

from ldu_cases import configs, rng

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


@pytest.fixture(scope="module")
def piso():
    from oracle import piso as m
    return m


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def case(s, seed=3):
    sys_ = configs.config3(s=s, seed=seed)
    phi = rng.uniform(rng.stream_base(seed, "piso-flux"), sys_.owner.shape[0], -1.0, 1.0)
    return sys_, phi


@pytest.mark.parametrize("s,precision", [(10, "fp64"), (24, "fp64"), (24, "mixed")])
def test_pressure_stage_matches_oracle(pkg, piso, s, precision):
    sys_, phi = case(s)
    tol = 1e-10
    A = pkg.from_system(sys_)
    phi_d, p_d = dev(phi), torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    st, it, rr = pkg.ldu_piso_pressure(A, dev(sys_.coef), phi_d, p_d, tol=tol,
                                       precision=precision, deflate=precision == "mixed")
    assert st == 0 and rr <= tol
    ro = piso.pressure_step(sys_, sys_.coef, phi, tol=tol, precision=precision,
                            deflate=precision == "mixed")
    p, phin = p_d.cpu().numpy(), phi_d.cpu().numpy()
    assert np.max(np.abs(p - ro.p)) <= 1e-6 * np.max(np.abs(ro.p))
    assert np.max(np.abs(phin - ro.phi)) <= 1e-6 * np.max(np.abs(ro.phi)) + 1e-12
    div0 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phi)
    div1 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phin)
    assert np.linalg.norm(div1) <= 2 * tol * np.linalg.norm(div0)
    if precision == "fp64":
        assert abs(it - ro.iters) <= 0.02 * ro.iters + 2
    A.close()


def test_divergence_free_input_is_left_alone(pkg):
    sys_, _ = case(8)
    nx = ny = 8
    fi = {(int(o), int(n)): f for f, (o, n) in enumerate(zip(sys_.owner, sys_.neighbour))}
    c = lambda a, b, k: a + nx * (b + ny * k)  # noqa: E731
    psi = np.zeros(sys_.owner.shape[0])
    for (i, j, k, w) in ((2, 3, 4, 1.0), (5, 1, 1, -0.25)):
        psi[fi[(c(i, j, k), c(i + 1, j, k))]] += w
        psi[fi[(c(i + 1, j, k), c(i + 1, j + 1, k))]] += w
        psi[fi[(c(i, j + 1, k), c(i + 1, j + 1, k))]] -= w
        psi[fi[(c(i, j, k), c(i, j + 1, k))]] -= w
    A = pkg.from_system(sys_)
    phi_d, p_d = dev(psi), torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    st, it, rr = pkg.ldu_piso_pressure(A, dev(sys_.coef), phi_d, p_d, precision="fp64")
    assert st == 0 and it == 0
    assert float(p_d.abs().max()) == 0.0
    assert np.array_equal(phi_d.cpu().numpy(), psi)
    A.close()


def test_time_steps_warm_start(pkg, piso):
    """Five steps with slowly varying predicted fluxes on one handle: each
    starts from the previous pressure, needs fewer iterations than the first,
    and leaves divergence-free fluxes."""
    sys_, phi = case(24)
    dphi = rng.uniform(rng.stream_base(7, "piso-dflux"), phi.shape[0], -1.0, 1.0)
    A = pkg.from_system(sys_)
    coef = dev(sys_.coef)
    p_d = torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    its = []
    for k in range(5):
        phik = phi + 1e-3 * k * dphi
        phi_d = dev(phik)
        st, it, rr = pkg.ldu_piso_pressure(A, coef, phi_d, p_d, tol=1e-9, precision="mixed",
                                           deflate=True)
        assert st == 0
        its.append(it)
        div0 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phik)
        div1 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phi_d.cpu().numpy())
        assert np.linalg.norm(div1) <= 2e-9 * np.linalg.norm(div0)
    assert max(its[1:]) < its[0]
    A.close()


def test_full_size_128(pkg, piso):
    """The graded 128^3 pressure system (2.1 M cells, 6.2 M faces) by
    properties: divergence removed to the tolerance, pinned cell at zero."""
    sys_, phi = case(128)
    A = pkg.from_system(sys_)
    phi_d, p_d = dev(phi), torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    st, it, rr = pkg.ldu_piso_pressure(A, dev(sys_.coef), phi_d, p_d, tol=1e-8,
                                       precision="mixed", deflate=True)
    assert st == 0 and rr <= 1e-8
    div0 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phi)
    div1 = piso.divergence_fast(sys_.owner, sys_.neighbour, sys_.n, phi_d.cpu().numpy())
    assert np.linalg.norm(div1) <= 2e-8 * np.linalg.norm(div0)
    p = p_d.cpu().numpy()
    assert abs(p[0]) <= 1e-6 * np.max(np.abs(p))
    A.close()


def test_errors(pkg):
    sys_, phi = case(6)
    A = pkg.from_system(sys_)
    with pytest.raises(KeyError):
        pkg.ldu_piso_pressure(A, dev(sys_.coef), dev(phi), dev(np.zeros(sys_.n)),
                              precision="fp32")
    A.close()
    B = pkg.from_systems([sys_, sys_])
    nf2 = 2 * sys_.owner.shape[0]
    st, _, _ = pkg.ldu_piso_pressure(B, dev(np.ones(nf2)), dev(np.zeros(nf2)),
                                     dev(np.zeros(B.n)), precision="fp64", check=False)
    assert st == -7   # UNSUPPORTED: single-system handles only
    B.close()
