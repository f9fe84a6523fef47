"""Aggregation-AMG preconditioned CG (Sec. 5, Table 2's AMG-CG) through the
C ABI against oracle/amg.py.

Bars: the aggregates of every level and every level's row count are
bit-exact (integer work; strengths within a relative 1e-12 count as ties on
both sides, so rounding in the coarse matrices cannot flip a choice); one
V-cycle agrees with the oracle's within 1e-11 relative to max |x| (the
library applies A through its symmetrically scaled copy, whose entries
carry a few ulps, and the coarsest solve is a dense inverse instead of an
LU solve: both differences are rounding, amplified by at most the coarse
levels' condition numbers, a few hundred here); the PCG's iteration count
is within one of the oracle's and both meet the tolerance on the true
residual.

The mixed solve applies the same cycle in float (level matrices rounded
to float once, float vectors) inside the FP64 outer CG with the
Polak-Ribiere beta.  Its cycle agrees with the oracle's FP64 cycle within
2e-5 relative to max |x| (float rounding, about 6e-8 per operation,
amplified by the coarse levels' conditioning); the mixed PCG meets the
same FP64 tolerance on the true residual, within two iterations of the
oracle's count."""
import numpy as np
import pytest

import ldu_cases as lc
from ldu_cases import configs, reorder

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
def amg():
    from oracle import amg as m
    return m


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def rcm(s):
    return reorder.renumber(s, reorder.rcm_order(s))


CASES = {
    "unit24": lambda: lc.poisson_box(24),
    "lognormal_20x17x13": lambda: lc.poisson_box(20, 17, 13, diffusivity="lognormal", seed=3),
    "lognormal_rcm24": lambda: rcm(lc.poisson_box(24, diffusivity="lognormal", seed=1)),
    "graded32": lambda: configs.config1(32),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_hierarchy_and_aggregates_match_oracle(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    info = M.info()
    assert info["levels"] == len(levels) + 1
    assert info["rows"] == [L[0].shape[0] for L in levels] + [coarse.shape[0]]
    for lev, (Al, _, _) in enumerate(levels):
        agg_o, _ = amg.aggregate(Al)
        assert np.array_equal(pkg.ldu_amg_aggregates(M, lev), agg_o), lev
    M.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_vcycle_matches_oracle(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    rng = np.random.default_rng(7)
    for b in (np.asarray(s.b, dtype=np.float64), rng.uniform(-1, 1, s.n)):
        x = pkg.ldu_amg_vcycle(M, dev(b)).cpu().numpy()
        xo = amg.vcycle(levels, coarse, b)
        assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
    M.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_float_vcycle_matches_oracle(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    rng = np.random.default_rng(8)
    for b in (np.asarray(s.b, dtype=np.float64), rng.uniform(-1, 1, s.n)):
        b32 = torch.as_tensor(b.astype(np.float32), device="cuda")
        x = pkg.ldu_amg_vcycle(M, b32).cpu().numpy().astype(np.float64)
        xo = amg.vcycle(levels, coarse, b.astype(np.float32).astype(np.float64))
        err = np.max(np.abs(x - xo)) / np.max(np.abs(xo))
        assert err <= 2e-5, err
    M.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_amg_pcg_meets_fp64_tolerance(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    r = amg.amg_pcg(s, tol=1e-8, maxit=200)
    x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-8, maxit=200, precision="mixed")
    assert st == 0 and relres <= 1e-8
    assert abs(it - r.iters) <= 2, (it, r.iters)
    A = amg.csr_of(s)
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) <= 1.0001e-8 * np.linalg.norm(s.b)
    M.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_amg_pcg_matches_oracle(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    r = amg.amg_pcg(s, tol=1e-8, maxit=200)
    x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-8, maxit=200)
    assert st == 0
    assert abs(it - r.iters) <= 1, (it, r.iters)
    assert relres <= 1e-8 and r.relres <= 1e-8
    # the true residual, recomputed from the returned x
    A = amg.csr_of(s)
    xs = x.cpu().numpy()
    assert np.linalg.norm(s.b - A @ xs) <= 1.0001e-8 * np.linalg.norm(s.b)
    assert abs(relres - np.linalg.norm(s.b - A @ xs) / np.linalg.norm(s.b)) <= 1e-3 * relres + 1e-15
    M.close()


def test_amg_pcg_nonzero_initial_guess(pkg, amg):
    s = lc.poisson_box(16, 14, 12, diffusivity="lognormal", seed=9)
    M = pkg.amg_from_system(s)
    x0 = np.random.default_rng(3).uniform(-1, 1, s.n)
    x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), x=dev(x0), tol=1e-9, maxit=200)
    assert st == 0 and relres <= 1e-9 and it > 0
    A = amg.csr_of(s)
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) <= 1.0001e-9 * np.linalg.norm(s.b)


def test_small_system_is_the_coarsest_level(pkg, amg):
    """n <= max_coarse: no prolongator, the V-cycle is the exact inverse and
    PCG converges in one iteration (the float inverse of the mixed solve
    gains about 1e-6 a step, so a few)."""
    s = lc.poisson_box(7, 6, 5, diffusivity="lognormal", seed=2)
    M = pkg.amg_from_system(s)
    assert M.info() == {"levels": 1, "rows": [s.n], "nnz": [s.n + 2 * len(s.owner)]}
    b = np.asarray(s.b, dtype=np.float64)
    x = pkg.ldu_amg_vcycle(M, dev(b)).cpu().numpy()
    xd = np.linalg.solve(amg.csr_of(s).toarray(), b)
    assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))
    for precision in ("fp64", "mixed"):
        _, it, relres, st = pkg.amg_pcg_solve(M, dev(b), tol=1e-10, precision=precision)
        assert st == 0 and relres <= 1e-10
        assert it == 1 if precision == "fp64" else it <= 4
    with pytest.raises(ValueError):
        pkg.ldu_amg_aggregates(M, 0)
    M.close()


def test_max_levels_and_max_coarse(pkg, amg):
    s = lc.poisson_box(24)
    A = amg.csr_of(s)
    for ml, mc in ((1, 500), (12, 2000), (12, 60)):
        M = pkg.amg_from_system(s, max_levels=ml, max_coarse=mc)
        levels, coarse = amg.hierarchy(A, max_coarse=mc, max_levels=ml)
        assert M.info()["rows"] == [L[0].shape[0] for L in levels] + [coarse.shape[0]]
        b = np.asarray(s.b, dtype=np.float64)
        x = pkg.ldu_amg_vcycle(M, dev(b)).cpu().numpy()
        xo = amg.vcycle(levels, coarse, b)
        assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
        M.close()


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_lanes_per_row_keeps_the_cycle(pkg, amg, lanes):
    """The lanes sharing a row of R and of the coarse matrices only change
    the order of each row's sum."""
    s = CASES["lognormal_rcm24"]()
    M = pkg.amg_from_system(s, lanes_per_row=lanes)
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    b = np.random.default_rng(9).uniform(-1, 1, s.n)
    x = pkg.ldu_amg_vcycle(M, dev(b)).cpu().numpy()
    xo = amg.vcycle(levels, coarse, b)
    assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
    M.close()


def test_zero_rhs_and_bad_arguments(pkg):
    s = lc.poisson_box(12)
    M = pkg.amg_from_system(s)
    x0 = torch.ones(s.n, dtype=torch.float64, device="cuda")
    x, it, relres, st = pkg.amg_pcg_solve(M, torch.zeros_like(x0), x=x0)
    assert st == 0 and it == 0 and relres == 0.0 and float(x.abs().max()) == 0.0
    x0 = torch.ones(s.n, dtype=torch.float64, device="cuda")
    x, it, relres, st = pkg.amg_pcg_solve(M, torch.zeros_like(x0), x=x0, precision="mixed")
    assert st == 0 and it == 0 and float(x.abs().max()) == 0.0
    # maxit reached: NOT_CONVERGED with the iterate so far
    x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-14, maxit=2, check=False)
    assert st == 1 and it == 2 and relres > 1e-14
    M.close()
    with pytest.raises(pkg.LduError):
        pkg.amg_from_system(s, max_coarse=5000)
    with pytest.raises(pkg.LduError):
        pkg.amg_from_system(s, max_levels=-1)
    with pytest.raises(pkg.LduError):
        pkg.amg_from_system(s, lanes_per_row=3)
    # coarsening stopped above the dense-inverse limit
    with pytest.raises(pkg.LduError) as e:
        pkg.amg_from_system(lc.poisson_box(48), max_levels=1)
    assert e.value.status == -7


def test_full_size_128_converges(pkg):
    """The 128^3 graded Dirichlet Poisson system (Table 2's largest cube):
    properties that hold at any size, without the oracle."""
    s = configs.config2(128)
    M = pkg.amg_from_system(s)
    info = M.info()
    assert info["rows"][0] == s.n and info["rows"][-1] <= 500
    assert all(a > b for a, b in zip(info["rows"], info["rows"][1:]))
    for precision in ("fp64", "mixed"):
        x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-8, maxit=200,
                                              precision=precision)
        assert st == 0 and relres <= 1e-8
        assert it <= 60   # Table 2 reports 32 for the paper's aggregation AMG at 128^3
    M.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_pipelined_amg_pcg_matches_oracle(pkg, amg, name):
    s = CASES[name]()
    M = pkg.amg_from_system(s)
    r = amg.amg_pipecg(s, tol=1e-8, maxit=200)
    x, it, relres, st = pkg.amg_pipecg_solve(M, dev(s.b), tol=1e-8, maxit=200)
    assert st == 0 and relres <= 1e-8
    assert abs(it - r.iters) <= 1, (it, r.iters)
    A = amg.csr_of(s)
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) <= 1.0001e-8 * np.linalg.norm(s.b)
    M.close()


def test_pipelined_iterates_equal_pcg_iterates(pkg):
    """After k steps the pipelined and the plain AMG-PCG hold the same
    iterate up to rounding (both on the device, FP64 cycle)."""
    s = CASES["lognormal_20x17x13"]()
    M = pkg.amg_from_system(s)
    for k in (1, 4, 9):
        x1, it1, _, st1 = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-30, maxit=k, check=False)
        x2, it2, _, st2 = pkg.amg_pipecg_solve(M, dev(s.b), tol=1e-30, maxit=k, check=False)
        assert st1 == st2 == 1 and it1 == it2 == k
        a, b = x1.cpu().numpy(), x2.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(a)), k
    M.close()


def test_pipelined_edge_cases(pkg, amg):
    s = lc.poisson_box(7, 6, 5, diffusivity="lognormal", seed=2)   # its own coarsest level
    M = pkg.amg_from_system(s)
    x, it, relres, st = pkg.amg_pipecg_solve(M, dev(s.b), tol=1e-10)
    assert st == 0 and it == 1 and relres <= 1e-10
    x, it, relres, st = pkg.amg_pipecg_solve(M, torch.zeros(s.n, dtype=torch.float64,
                                                            device="cuda"))
    assert st == 0 and it == 0 and float(x.abs().max()) == 0.0
    M.close()
    s = lc.poisson_box(12)
    M = pkg.amg_from_system(s)
    x0 = np.random.default_rng(5).uniform(-1, 1, s.n)
    x, it, relres, st = pkg.amg_pipecg_solve(M, dev(s.b), x=dev(x0), tol=1e-9)
    assert st == 0 and relres <= 1e-9
    A = amg.csr_of(s)
    assert np.linalg.norm(s.b - A @ x.cpu().numpy()) <= 1.0001e-9 * np.linalg.norm(s.b)
    M.close()


def test_pipelined_full_size_128(pkg):
    s = configs.config2(128)
    M = pkg.amg_from_system(s)
    _, it1, rr1, st1 = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-8, precision="fp64")
    _, it2, rr2, st2 = pkg.amg_pipecg_solve(M, dev(s.b), tol=1e-8)
    assert st1 == st2 == 0 and rr2 <= 1e-8 and abs(it1 - it2) <= 1
    M.close()


def test_full_size_hierarchy_matches_oracle(pkg, amg):
    """The 128^3 headline system: every level's row count and aggregates
    bit-exact against the oracle's hierarchy.  The device builds it in
    parallel (independent-set rounds, hash-table sparse products) and the
    oracle with scipy, so the coarse values differ in their last bits; the
    patterns are structural and the strength ties are relative to a row's
    largest entry, so the integer results agree all the same."""
    s = configs.config2(128)
    M = pkg.amg_from_system(s)
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    assert M.info()["rows"] == [L[0].shape[0] for L in levels] + [coarse.shape[0]]
    for lev in range(len(levels)):
        agg_o, _ = amg.aggregate(levels[lev][0])
        assert np.array_equal(pkg.ldu_amg_aggregates(M, lev), agg_o), lev
    # structural patterns: every level stores exactly the oracle's entries
    last_A, last_P, _ = levels[-1]
    assert M.info()["nnz"] == [L[0].nnz for L in levels] + [amg.galerkin(last_A, last_P).nnz]
    # the coarse levels' values, formed here by block-per-row fixed-point sums
    # for their long rows, through one FP64 cycle against the oracle's
    b = np.random.default_rng(6).uniform(-1, 1, s.n)
    x = pkg.ldu_amg_vcycle(M, dev(b)).cpu().numpy()
    xo = amg.vcycle(levels, coarse, b)
    assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
    M.close()


def test_device_setup_is_deterministic(pkg):
    """Two hierarchies of the same matrix are the same bit for bit: every sum
    of the construction is formed in a fixed order (duplicates by face, each
    product row in expansion order), whatever the thread scheduling."""
    s = CASES["lognormal_rcm24"]()
    b = dev(np.random.default_rng(3).uniform(-1, 1, s.n))
    outs = []
    for _ in range(2):
        M = pkg.amg_from_system(s)
        aggs = [pkg.ldu_amg_aggregates(M, k).copy() for k in range(M.info()["levels"] - 1)]
        outs.append((M.info()["rows"], M.info()["nnz"], aggs, pkg.ldu_amg_vcycle(M, b).cpu()))
        M.close()
    (r0, z0, a0, x0), (r1, z1, a1, x1) = outs
    assert r0 == r1 and z0 == z1
    assert all(np.array_equal(u, v) for u, v in zip(a0, a1))
    assert torch.equal(x0, x1)


def test_unsorted_faces_give_the_same_hierarchy(pkg, amg):
    """Faces need not be sorted: shuffling them (and so the order in which
    duplicate-free rows are assembled) changes nothing."""
    s = CASES["lognormal_20x17x13"]()
    perm = np.random.default_rng(11).permutation(s.nfaces)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)  # noqa: E731
    M = pkg.ldu_amg_create(s.n, t(s.owner[perm], torch.int32), t(s.neighbour[perm], torch.int32),
                           t(s.diag, torch.float64), t(s.upper[perm], torch.float64),
                           t(s.lower[perm], torch.float64))
    levels, coarse = amg.hierarchy(amg.csr_of(s))
    assert M.info()["rows"] == [L[0].shape[0] for L in levels] + [coarse.shape[0]]
    agg_o, _ = amg.aggregate(levels[0][0])
    assert np.array_equal(pkg.ldu_amg_aggregates(M, 0), agg_o)
    M.close()


def test_create_validates_like_ldu_create(pkg):
    s = lc.poisson_box(6, 5, 4)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)  # noqa: E731
    own, nbr = s.owner.copy(), s.neighbour.copy()
    own[3], nbr[3] = nbr[3], own[3]                       # owner > neighbour
    with pytest.raises(pkg.LduError) as e:
        pkg.ldu_amg_create(s.n, t(own, torch.int32), t(nbr, torch.int32), t(s.diag, torch.float64),
                           t(s.upper, torch.float64), t(s.lower, torch.float64))
    assert e.value.status == -2
    nbr2 = s.neighbour.copy()
    nbr2[5] = s.n                                          # index outside [0, n)
    with pytest.raises(pkg.LduError) as e:
        pkg.ldu_amg_create(s.n, t(s.owner, torch.int32), t(nbr2, torch.int32),
                           t(s.diag, torch.float64), t(s.upper, torch.float64),
                           t(s.lower, torch.float64))
    assert e.value.status == -2
    d = s.diag.copy()
    d[7] = 0.0                                             # non-positive diagonal
    with pytest.raises(pkg.LduError) as e:
        pkg.ldu_amg_create(s.n, t(s.owner, torch.int32), t(s.neighbour, torch.int32),
                           t(d, torch.float64), t(s.upper, torch.float64), t(s.lower, torch.float64))
    assert e.value.status == -3
    up = s.upper.copy()
    up[2] = np.nan                                         # non-finite value
    with pytest.raises(pkg.LduError) as e:
        pkg.ldu_amg_create(s.n, t(s.owner, torch.int32), t(s.neighbour, torch.int32),
                           t(s.diag, torch.float64), t(up, torch.float64), t(s.lower, torch.float64))
    assert e.value.status == -3


@pytest.mark.parametrize("solver", ["fp64", "mixed", "pipelined"])
def test_unreachable_tolerance_restarts_and_stops_at_the_cap(pkg, amg, solver):
    """tol = 1e-16 lies below what FP64 can confirm: the recursive residual
    passes it, the true residual does not, the search restarts from the true
    residual (the confirmation path), and the loop ends at the iteration cap
    with NOT_CONVERGED and the reported residual equal to the recomputed one."""
    s = CASES["lognormal_rcm24"]()
    M = pkg.amg_from_system(s)
    if solver == "pipelined":
        x, it, relres, st = pkg.amg_pipecg_solve(M, dev(s.b), tol=1e-16, maxit=80, check=False)
    else:
        x, it, relres, st = pkg.amg_pcg_solve(M, dev(s.b), tol=1e-16, maxit=80,
                                              precision=solver, check=False)
    assert st in (0, 1) and it <= 80
    A = amg.csr_of(s)
    true = np.linalg.norm(s.b - A @ x.cpu().numpy()) / np.linalg.norm(s.b)
    # both residuals are formed at rounding level here: they agree to a few 1e-17
    assert abs(true - relres) <= max(1e-3 * true, 1e-16)
    # attainable accuracy: PCG reaches FP64's; the pipelined recurrences (four
    # coupled updates, no periodic replacement) drift from the true residual
    # to about 1e-10 before the confirmation restarts them
    assert true <= (1e-9 if solver == "pipelined" else 1e-13)
    M.close()
