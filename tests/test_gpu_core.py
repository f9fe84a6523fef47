"""GPU parity of the C-ABI path against the oracle: SpMV, Jacobi-PCG,
pipelined PCG (FP64 and mixed), face gradient, value refresh, edge cases.

Tolerances (floating point, from the arithmetic):
  * SpMV FP64: |y - y_ref| <= 1e-13 * (|A| |x|)_i per row (componentwise
    backward-error form; a few ulps of the row's absolute sum).
  * SpMV FP32: <= 1e-6 * (|A| |x|)_i on float inputs.
  * Solves: the true ||b - A x||/||b|| of the returned x, recomputed by the
    oracle's own FP64 SpMV, is <= tol (1% slack for the difference between
    the scaled-space and original-space rounding); iteration counts of the
    FP64 methods within 2% + 2 of the oracle's; solutions at a tight
    tolerance within 1e-9 of the oracle's.
"""
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


def cuda(a, dt=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t if dt is None else t.to(dt)


def abs_bound(oracle_mod, s, x):
    return oracle_mod.spmv(s, np.abs(x), diag=np.abs(s.diag), upper=np.abs(s.upper),
                           lower=np.abs(s.lower))


def shuffled_faces(s, seed=5):
    g = np.random.default_rng(seed)
    order = g.permutation(s.nfaces)
    t = lc.LduSystem(n=s.n, owner=s.owner[order], neighbour=s.neighbour[order], diag=s.diag,
                     upper=s.upper[order], lower=s.lower[order], b=s.b, coef=s.coef[order],
                     diag_extra=s.diag_extra, shape=s.shape, name=s.name + "-shuffled")
    return t


def nonsymmetric(s, seed=9):
    g = np.random.default_rng(seed)
    t = lc.LduSystem(n=s.n, owner=s.owner, neighbour=s.neighbour,
                     diag=s.diag * g.uniform(1.0, 2.0, s.n),
                     upper=s.upper * g.uniform(0.5, 1.5, s.nfaces),
                     lower=s.lower * g.uniform(0.5, 1.5, s.nfaces), b=s.b, coef=s.coef,
                     diag_extra=s.diag_extra, shape=s.shape, name=s.name + "-nonsym")
    return t


SPMV_CASES = {
    "c1-8": lambda: lc.config1(s=8),
    "c2-13-ragged": lambda: lc.config2(s=13),
    "c3-10": lambda: lc.config3(s=10),
    "box-5x6x7": lambda: lc.poisson_box(5, 6, 7, diffusivity="lognormal"),
    "one-cell": lambda: lc.poisson_box(1, 1, 1),
    "line-1x1x9": lambda: lc.poisson_box(9, 1, 1),
    "shuffled": lambda: shuffled_faces(lc.config2(s=7)),
    "nonsym": lambda: nonsymmetric(lc.config2(s=9)),
}


@pytest.mark.parametrize("case", list(SPMV_CASES))
@pytest.mark.parametrize("C", [32, 64, 128])
def test_spmv_parity(pkg, oracle_mod, case, C):
    s = SPMV_CASES[case]()
    A = pkg.from_system(s, slice_rows=C)
    g = np.random.default_rng(3)
    x = g.uniform(-1, 1, s.n)
    y = pkg.ldu_spmv(A, cuda(x)).cpu().numpy()
    y_ref = oracle_mod.spmv(s, x)
    bound = abs_bound(oracle_mod, s, x)
    assert np.all(np.abs(y - y_ref) <= 1e-13 * bound + 1e-300)
    x32 = x.astype(np.float32)
    y32 = pkg.ldu_spmv(A, cuda(x32), precision="fp32").cpu().numpy().astype(np.float64)
    y32_ref = oracle_mod.spmv(s, x32.astype(np.float64))
    bound32 = abs_bound(oracle_mod, s, x32.astype(np.float64))
    assert np.all(np.abs(y32 - y32_ref) <= 1e-6 * bound32 + 1e-30)
    info = A.info()
    assert info["n"] == s.n and info["n_padded"] % C == 0 and info["n_padded"] >= s.n
    A.close()


def test_spmv_and_solves_share_a_handle(pkg):
    """The double product passes through one of the handle's work vectors
    (D^1/2 x, then the product): products between solves leave the solves'
    results unchanged, solves leave the products unchanged, and coefficient
    updates reach the float product's copy of the scaling factors."""
    s = lc.config2(s=24)
    A = pkg.from_system(s)
    g = np.random.default_rng(11)
    x = cuda(g.uniform(-1, 1, s.n))
    x32 = x.float()
    b = cuda(s.b)
    y64 = pkg.ldu_spmv(A, x).clone()
    y32 = pkg.ldu_spmv(A, x32, precision="fp32").clone()
    sol = []
    for _ in range(2):
        xs, st, it, rr = pkg.pipecg_solve(A, b, tol=1e-10, precision="mixed", deflate=True)
        assert st == 0
        sol.append((xs.clone(), it, rr))
        assert torch.equal(pkg.ldu_spmv(A, x), y64)
        assert torch.equal(pkg.ldu_spmv(A, x32, precision="fp32"), y32)
        xp, st, _, _ = pkg.pcg_solve(A, b, tol=1e-10)
        assert st == 0
    assert torch.equal(sol[0][0], sol[1][0]) and sol[0][1:] == sol[1][1:]
    # new values: both products follow them (against the oracle's product)
    import oracle as om
    vals = {"diag": 1.5 * s.diag, "upper": 0.7 * s.upper, "lower": 0.7 * s.lower}
    pkg.ldu_update_values(A, cuda(vals["diag"]), cuda(vals["upper"]), cuda(vals["lower"]))
    xn = g.uniform(-1, 1, s.n)
    ref = om.spmv(s, xn, **vals)
    scale = np.abs(ref).max()
    assert np.max(np.abs(pkg.ldu_spmv(A, cuda(xn)).cpu().numpy() - ref)) <= 1e-12 * scale
    xn32 = xn.astype(np.float32)
    y32n = pkg.ldu_spmv(A, cuda(xn32), precision="fp32").cpu().numpy()
    ref32 = om.spmv(s, xn32.astype(np.float64), **vals)
    assert np.max(np.abs(y32n - ref32)) <= 1e-5 * scale
    A.close()


SOLVE_CASES = {
    "c1-32": lambda: lc.config1(),   # the 32^3 unit-diffusivity Poisson case at its full size
    "c1-16": lambda: lc.config1(s=16),
    "c2-20": lambda: lc.config2(s=20),
    "c3-16": lambda: lc.config3(s=16),
    "box-7x5x9": lambda: lc.poisson_box(7, 5, 9, diffusivity="lognormal", seed=4),
    "shuffled-c2-9": lambda: shuffled_faces(lc.config2(s=9)),
}


@pytest.mark.parametrize("case", list(SOLVE_CASES))
@pytest.mark.parametrize("C", [32, 128])
def test_pcg_parity(pkg, oracle_mod, case, C):
    s = SOLVE_CASES[case]()
    A = pkg.from_system(s, slice_rows=C)
    b = cuda(s.b)
    ref = oracle_mod.pcg(s, tol=1e-8)
    x, st, it, rr = pkg.pcg_solve(A, b, tol=1e-8)
    xh = x.cpu().numpy()
    true_rr = oracle_mod.true_relres(s, xh)
    assert st == 0
    assert true_rr <= 1.01e-8
    assert abs(rr - true_rr) <= 1e-3 * true_rr + 1e-15
    assert abs(it - ref.iters) <= 0.02 * ref.iters + 2
    # tight solve: the same solution as the oracle's
    xt, st, _, _ = pkg.pcg_solve(A, b, tol=1e-12)
    xs = oracle_mod.pcg(s, tol=1e-12).x
    assert st == 0
    assert np.linalg.norm(xt.cpu().numpy() - xs) <= 1e-9 * np.linalg.norm(xs)
    A.close()


@pytest.mark.parametrize("case", list(SOLVE_CASES))
def test_pipecg_fp64_parity(pkg, oracle_mod, case):
    s = SOLVE_CASES[case]()
    A = pkg.from_system(s)
    b = cuda(s.b)
    ref = oracle_mod.pipecg(s, tol=1e-8)
    x, st, it, rr = pkg.pipecg_solve(A, b, tol=1e-8, precision="fp64")
    true_rr = oracle_mod.true_relres(s, x.cpu().numpy())
    assert st == 0 and true_rr <= 1.01e-8
    assert abs(it - ref.iters) <= 0.02 * ref.iters + 2
    pcg_it = oracle_mod.pcg(s, tol=1e-8).iters
    assert abs(it - pcg_it) <= 0.02 * pcg_it + 2      # pipelined == PCG in exact arithmetic
    A.close()


@pytest.mark.parametrize("case", list(SOLVE_CASES))
@pytest.mark.parametrize("mode", [dict(rr_period=16), dict(rr_period=0, tau=1e-3, restart=True),
                                  dict(rr_period=16, deflate=True), dict(rr_period=16, tau=0.3)])
def test_mixed_parity(pkg, oracle_mod, case, mode):
    s = SOLVE_CASES[case]()
    A = pkg.from_system(s)
    b = cuda(s.b)
    ref = oracle_mod.mixed_pipecg(s, tol=1e-8, period=mode["rr_period"],
                                  tau=mode.get("tau", 0.0), restart=mode.get("restart", False),
                                  deflate=mode.get("deflate", False))
    x, st, it, rr = pkg.pipecg_solve(A, b, tol=1e-8, precision="mixed", **mode)
    xh = x.cpu().numpy()
    true_rr = oracle_mod.true_relres(s, xh)
    assert st == 0 and true_rr <= 1.01e-8, (st, it, rr, true_rr)
    # float rounding differs in order between the two, so iteration counts
    # agree loosely; the error against the tight FP64 solution is reported
    assert it <= 1.25 * ref.iters + 8
    xs = oracle_mod.pcg(s, tol=1e-13).x
    err = np.linalg.norm(xh - xs) / np.linalg.norm(xs)
    err_ref = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert err <= max(10 * err_ref, 1e-6)
    A.close()


def test_mixed_default_rule_is_period_16_tau_03(pkg):
    """With rr_period and tau both 0 the mixed solve replaces every 16
    iterations and on a 0.3^2 drop: bitwise the same run as those options."""
    s = lc.config2(s=24)
    A = pkg.from_system(s, slice_rows=64)
    b = cuda(s.b)
    x0, st0, it0, rr0 = pkg.pipecg_solve(A, b, tol=1e-9, precision="mixed")
    reps0 = A.stats()["replacements"]
    x1, st1, it1, rr1 = pkg.pipecg_solve(A, b, tol=1e-9, precision="mixed", rr_period=16, tau=0.3)
    assert st0 == st1 == 0 and it0 == it1 and reps0 == A.stats()["replacements"]
    assert torch.equal(x0, x1) and rr0 == rr1
    A.close()


def test_mixed_reaches_tight_tolerance(pkg, oracle_mod):
    s = lc.config2(s=12)
    A = pkg.from_system(s)
    x, st, it, rr = pkg.pipecg_solve(A, cuda(s.b), tol=1e-12, precision="mixed")
    assert st == 0 and oracle_mod.true_relres(s, x.cpu().numpy()) <= 1.01e-12
    assert A.stats()["replacements"] >= 3
    A.close()


@pytest.mark.parametrize("solver", ["pcg", "pipe", "mixed"])
def test_edge_cases(pkg, oracle_mod, solver):
    s = lc.config2(s=6)
    A = pkg.from_system(s)

    def solve(b, x0=None, **kw):
        if solver == "pcg":
            return pkg.pcg_solve(A, b, x0, check=False, **kw)
        return pkg.pipecg_solve(A, b, x0, precision="fp64" if solver == "pipe" else "mixed",
                                check=False, **kw)

    # zero right-hand side: x = 0 whatever the initial guess
    x, st, it, rr = solve(torch.zeros(s.n, dtype=torch.float64, device="cuda"),
                          torch.ones(s.n, dtype=torch.float64, device="cuda"))
    assert st == 0 and rr == 0.0 and it == 0 and float(x.abs().max()) == 0.0
    # exact initial guess: no iterations
    xs = oracle_mod.pcg(s, tol=1e-14).x
    x, st, it, rr = solve(cuda(s.b), cuda(xs), tol=1e-8)
    assert st == 0 and it == 0 and rr <= 1e-8
    # iteration cap
    x, st, it, rr = solve(cuda(s.b), tol=1e-14, maxit=3)
    assert st == 1 and it == 3 and rr > 1e-14
    assert abs(oracle_mod.true_relres(s, x.cpu().numpy()) - rr) <= 1e-6 * rr
    # deterministic: two runs agree bitwise
    x1, *_ = solve(cuda(s.b), tol=1e-10)
    x2, *_ = solve(cuda(s.b), tol=1e-10)
    assert torch.equal(x1, x2)
    A.close()


def test_empty_and_tiny(pkg, oracle_mod):
    s = lc.poisson_box(1, 1, 1)
    A = pkg.from_system(s)
    x, st, it, rr = pkg.pcg_solve(A, cuda(s.b), tol=1e-12)
    assert st == 0 and abs(float(x[0]) - s.b[0] / s.diag[0]) <= 1e-15 * abs(s.b[0] / s.diag[0])
    A.close()
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    ei = torch.zeros(0, dtype=torch.int32, device="cuda")
    A0 = pkg.ldu_create(0, ei, ei, e, e, e)
    x, st, it, rr = pkg.pcg_solve(A0, e)
    assert st == 0 and it == 0
    A0.close()


def test_not_spd_and_bad_addressing(pkg):
    s = lc.poisson_box(6, 5, 4)
    ones = np.ones(s.n)
    # unit diagonal, off-diagonals -1: I - adjacency is indefinite
    t = lc.LduSystem(n=s.n, owner=s.owner, neighbour=s.neighbour, diag=ones,
                     upper=-np.ones(s.nfaces), lower=-np.ones(s.nfaces), b=s.b, coef=s.coef,
                     diag_extra=s.diag_extra)
    A = pkg.from_system(t)
    for call in (lambda: pkg.pcg_solve(A, cuda(s.b), check=False),
                 lambda: pkg.pipecg_solve(A, cuda(s.b), check=False)):
        _, st, _, _ = call()
        assert st == pkg.ldupcg.ERR_NOT_SPD
    A.close()
    with pytest.raises(pkg.LduError) as e:
        bad = lc.LduSystem(n=s.n, owner=s.neighbour, neighbour=s.owner, diag=s.diag,
                           upper=s.upper, lower=s.lower, b=s.b, coef=s.coef,
                           diag_extra=s.diag_extra)
        pkg.from_system(bad)
    assert e.value.status == pkg.ldupcg.ERR_BAD_ADDRESSING
    with pytest.raises(pkg.LduError) as e:
        nb = s.neighbour.copy()
        nb[3] = s.n + 7
        bad = lc.LduSystem(n=s.n, owner=s.owner, neighbour=nb, diag=s.diag, upper=s.upper,
                           lower=s.lower, b=s.b, coef=s.coef, diag_extra=s.diag_extra)
        pkg.from_system(bad)
    assert e.value.status == pkg.ldupcg.ERR_BAD_ADDRESSING
    with pytest.raises(pkg.LduError) as e:
        d = s.diag.copy()
        d[0] = 0.0
        bad = lc.LduSystem(n=s.n, owner=s.owner, neighbour=s.neighbour, diag=d, upper=s.upper,
                           lower=s.lower, b=s.b, coef=s.coef, diag_extra=s.diag_extra)
        pkg.from_system(bad)
    assert e.value.status == pkg.ldupcg.ERR_NOT_SPD


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_barrier_timeout_is_reported_and_recoverable(pkg, oracle_mod, precision):
    """Block 0 leaves before its first barrier; the others time out.  The
    block limit is lifted so that this small system still has other blocks."""
    s = lc.config1(s=10)
    A = pkg.from_system(s, min_slices=-1)
    _, st, _, _ = pkg.pipecg_solve(A, cuda(s.b), precision=precision, barrier_timeout_s=0.2,
                                   fault_inject=1, check=False)
    assert st == pkg.ldupcg.ERR_BARRIER_TIMEOUT
    # the context and the handle stay usable
    x, st, it, rr = pkg.pipecg_solve(A, cuda(s.b), precision=precision, tol=1e-8)
    assert st == 0 and oracle_mod.true_relres(s, x.cpu().numpy()) <= 1.01e-8
    A.close()


def test_face_grad_bitwise(pkg, oracle_mod):
    s = lc.config2(s=11)
    A = pkg.from_system(s)
    g = np.random.default_rng(2)
    lam = g.standard_normal(s.n)
    x = g.standard_normal(s.n)
    got = pkg.ldu_face_grad(A, cuda(lam), cuda(x)).cpu().numpy()
    ref = oracle_mod.face_grad(s.owner, s.neighbour, lam, x)
    assert np.array_equal(got, ref)
    A.close()


def test_set_face_coeffs_matches_assembly(pkg, oracle_mod):
    s = lc.config2(s=10)
    A = pkg.from_system(s)
    g = np.random.default_rng(4)
    coef = s.coef * g.uniform(0.5, 2.0, s.nfaces)
    pkg.ldu_set_face_coeffs(A, cuda(coef), cuda(s.diag_extra))
    d, u, lo = oracle_mod.matrix_from_coef(s, coef)
    x = g.uniform(-1, 1, s.n)
    y = pkg.ldu_spmv(A, cuda(x)).cpu().numpy()
    y_ref = oracle_mod.spmv(s, x, diag=d, upper=u, lower=lo)
    bound = oracle_mod.spmv(s, np.abs(x), diag=np.abs(d), upper=np.abs(u), lower=np.abs(lo))
    assert np.all(np.abs(y - y_ref) <= 1e-13 * bound)
    # update_values with the same matrix gives the same product
    pkg.ldu_update_values(A, cuda(d), cuda(u), cuda(lo))
    y2 = pkg.ldu_spmv(A, cuda(x)).cpu().numpy()
    assert np.all(np.abs(y2 - y_ref) <= 1e-13 * bound)
    A.close()


@pytest.fixture(scope="module")
def mixed_mid(oracle_mod):
    """config 2 at 96^3 (884,736 cells): several slices per warp at every
    slice height, so the staged pipeline refills its stages."""
    s = lc.config2(s=96)
    ref = oracle_mod.mixed_pipecg(s, tol=1e-8, period=12)
    xs = oracle_mod.pcg(s, tol=1e-11).x
    return s, ref, xs


@pytest.mark.parametrize("staging", [0, -1])
@pytest.mark.parametrize("C,bps", [(32, 0), (32, 3), (32, 4), (64, 0), (64, 3), (128, 0)])
def test_mixed_launch_shapes(pkg, oracle_mod, mixed_mid, C, bps, staging):
    """Every build of the mixed kernel (slice height x resident blocks per SM
    x staged or plain matrix loads) against the oracle on the same case."""
    s, ref, xs = mixed_mid
    A = pkg.from_system(s, slice_rows=C, blocks_per_sm=bps, staging=staging)
    x, st, it, rr = pkg.pipecg_solve(A, cuda(s.b), tol=1e-8, precision="mixed", rr_period=12)
    stats = A.stats()
    xh = x.cpu().numpy()
    true_rr = oracle_mod.true_relres(s, xh)
    assert st == 0 and true_rr <= 1.01e-8, (st, it, rr, true_rr)
    assert abs(rr - true_rr) <= 1e-3 * true_rr
    assert it <= 1.25 * ref.iters + 8, (it, ref.iters)
    err = np.linalg.norm(xh - xs) / np.linalg.norm(xs)
    err_ref = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert err <= max(10 * err_ref, 1e-6)
    if staging == -1:
        assert stats["staged"] == 0
    if bps:
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert stats["grid_blocks"] == bps * nsm
    A.close()


@pytest.mark.parametrize("ny,fits", [(32767, True), (32768, False), (20, True)])
def test_col16_offsets_at_the_int16_limit(pkg, oracle_mod, ny, fits):
    """A 1 x ny x 2 box numbers its z-neighbour ny rows away: 32767 is the
    largest offset the 16-bit columns hold, 32768 sends the handle back to
    int32 columns.  Both solve the same as the oracle (the diagonal is
    scaled by 4, a strongly dominant diagonal, so a few iterations do)."""
    s = lc.poisson_box(1, ny, 2, diffusivity="lognormal", seed=2)
    s.diag = 4.0 * s.diag
    A = pkg.from_system(s, slice_rows=64)
    assert A.info()["col16"] == (1 if fits else 0)
    ref = oracle_mod.mixed_pipecg(s, tol=1e-10, period=12)
    x, st, it, rr = pkg.pipecg_solve(A, cuda(s.b), tol=1e-10, precision="mixed", rr_period=12)
    assert A.stats()["staged"] == 1
    xh = x.cpu().numpy()
    assert st == 0 and oracle_mod.true_relres(s, xh) <= 1.01e-10
    assert it <= 1.25 * ref.iters + 8
    assert np.linalg.norm(xh - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    A.close()
    B = pkg.from_system(s, slice_rows=64, staging=-1)
    assert B.info()["col16"] == 0          # plain loads never read them
    B.close()


@pytest.mark.parametrize("solver", ["pcg", "mixed"])
def test_small_systems_use_fewer_blocks(pkg, oracle_mod, solver):
    """By default a single-system launch gives each block at least 8 slices:
    a 16^3 system (32 slices of 128 rows) runs on 4 blocks, and the same
    solve without the limit (one block per resident slot, most of them
    idle) reaches the same solution."""
    s = lc.config1(s=16)
    b = cuda(s.b)
    out = {}
    for ms in (0, -1):
        A = pkg.from_system(s, min_slices=ms)
        if solver == "pcg":
            x, st, it, rr = pkg.pcg_solve(A, b, tol=1e-10)
        else:
            x, st, it, rr = pkg.pipecg_solve(A, b, tol=1e-10, precision="mixed")
        assert st == 0 and oracle_mod.true_relres(s, x.cpu().numpy()) <= 1.01e-10
        out[ms] = (x.cpu().numpy(), it, A.stats()["grid_blocks"])
        A.close()
    assert out[0][2] == 4
    assert out[-1][2] > 4
    assert abs(out[0][1] - out[-1][1]) <= 2
    assert np.linalg.norm(out[0][0] - out[-1][0]) <= 1e-8 * np.linalg.norm(out[-1][0])


def smooth_field(s):
    """sin(pi x) sin(pi y) sin(pi z) at the cell centres of a unit box."""
    nx, ny, nz = s.shape
    c = np.asarray(s.cell_of)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    return (np.sin(np.pi * (i + 0.5) / nx) * np.sin(np.pi * (j + 0.5) / ny)
            * np.sin(np.pi * (k + 0.5) / nz))


def heat_system(s, mass):
    """The backward-Euler matrix M + A of a diffusion system."""
    return lc.LduSystem(n=s.n, owner=s.owner, neighbour=s.neighbour, diag=s.diag + mass,
                        upper=s.upper, lower=s.lower, b=s.b, coef=s.coef,
                        diag_extra=s.diag_extra + mass, shape=s.shape, name=s.name + "-heat")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_heat_steps_match_oracle(pkg, oracle_mod, precision):
    """Five implicit heat steps (M + A) T^(n+1) = M T^n from a smooth T^0,
    against the same steps solved by the oracle's dense LU; starting each
    step from the last temperature needs fewer iterations than starting
    from zero (by about a tenth at this step size: the stopping test is
    relative to ||b||, so a warm start saves only the first digits)."""
    s = lc.poisson_box(8, 8, 8, diffusivity="lognormal", seed=31)
    h = 1.0 / 8
    mass = np.full(s.n, h ** 3 / (0.05 * h * h))          # dt = 0.05 h^2 (k ~ 1)
    hs = heat_system(s, mass)
    A = pkg.from_system(hs)
    T0 = smooth_field(s)
    T = cuda(T0.copy())
    _, st, its, rr = pkg.ldu_heat_steps(A, cuda(mass), T, 5, tol=1e-12, precision=precision)
    assert st == 0 and rr <= 1.01e-12
    M = oracle_mod.dense(hs)
    Tref = T0.copy()
    for _ in range(5):
        Tref = oracle_mod.lu_solve(M, mass * Tref)
    assert np.linalg.norm(T.cpu().numpy() - Tref) <= 1e-9 * np.linalg.norm(Tref)
    # the same steps, each from zero
    cold = 0
    Tc = cuda(T0.copy())
    for _ in range(5):
        b = cuda(mass) * Tc
        x, st, it, _ = (pkg.pcg_solve(A, b, tol=1e-12) if precision == "fp64" else
                        pkg.pipecg_solve(A, b, tol=1e-12, precision="mixed"))
        cold += it
        Tc = x
    assert its < cold, (its, cold)
    A.close()


def test_heat_steps_edge_cases(pkg):
    s = lc.poisson_box(3, 3, 3)
    mass = np.ones(s.n)
    A = pkg.from_system(heat_system(s, mass))
    T = cuda(np.ones(s.n))
    _, st, its, rr = pkg.ldu_heat_steps(A, cuda(mass), T, 0)        # no steps: unchanged
    assert st == 0 and its == 0 and torch.all(T == 1)
    z = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    _, st, its, rr = pkg.ldu_heat_steps(A, cuda(mass), z, 3)        # T = 0 stays 0
    assert st == 0 and torch.all(z == 0) and rr == 0.0
    B = pkg.from_systems([s, s])
    _, st, _, _ = pkg.ldu_heat_steps(B, cuda(np.ones(2 * s.n)),
                                     cuda(np.ones(2 * s.n)), 1, check=False)
    assert st == pkg.ldupcg.ERR_UNSUPPORTED
    A.close()
    B.close()
