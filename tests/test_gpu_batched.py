"""Batched solve (many independent systems in one persistent launch) against
the oracle system by system, and against separate single-system solves.

Tolerances as in test_gpu_core: every system's true relative residual,
recomputed by the oracle's FP64 SpMV, is <= tol (1% slack); FP64 PCG
iteration counts within 2% + 2 of the oracle's."""
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


def small_batch():
    """Config-4 recipe at small sizes, plus edge cases: one cell, a line of
    cells, a non-cubic box, sizes that are and are not slice multiples."""
    sides = lc.config4_sides(nsys=20, lo=3, hi=12, seed=1)
    systems = [lc.poisson_box(int(sd), seed=1, sub=i, diffusivity="lognormal")
               for i, sd in enumerate(sides)]
    systems += [lc.poisson_box(1, 1, 1, seed=2, sub=0), lc.poisson_box(9, 1, 1, seed=2, sub=1),
                lc.poisson_box(4, 8, 4, seed=2, sub=2, diffusivity="lognormal"),
                lc.config3(s=8, seed=3)]
    return systems


def cat_b(systems):
    return torch.as_tensor(np.concatenate([s.b for s in systems]), device="cuda")


def split(x, systems):
    out, o = [], 0
    for s in systems:
        out.append(x[o:o + s.n])
        o += s.n
    return out


@pytest.mark.parametrize("C", [32, 64, 128])
@pytest.mark.parametrize("precision,staging", [("fp64", 0), ("mixed", 0), ("mixed", -1)])
def test_batched_parity(pkg, oracle_mod, C, precision, staging):
    """staging 0: the mixed solve's float sweeps stage the matrix in shared
    memory (each one-block team opens and drains its own pipeline per
    system); -1: plain loads."""
    systems = small_batch()
    A = pkg.from_systems(systems, slice_rows=C, staging=staging)
    b = cat_b(systems)
    x, worst, its, rrs, sts = pkg.pcg_solve_batched(A, b, tol=1e-8, precision=precision)
    assert worst == 0 and np.all(sts == 0)
    xs = split(x.cpu().numpy(), systems)
    for k, s in enumerate(systems):
        true_rr = oracle_mod.true_relres(s, xs[k])
        assert true_rr <= 1.01e-8, (k, s.name, its[k], rrs[k], true_rr)
        assert abs(rrs[k] - true_rr) <= 1e-3 * true_rr + 1e-15
        if precision == "fp64":
            ref = oracle_mod.pcg(s, tol=1e-8)
            assert abs(its[k] - ref.iters) <= 0.02 * ref.iters + 2, (k, its[k], ref.iters)
    A.close()


def test_batched_matches_separate_solves(pkg, oracle_mod):
    systems = small_batch()
    A = pkg.from_systems(systems, slice_rows=64)
    x, worst, its, rrs, sts = pkg.pcg_solve_batched(A, cat_b(systems), tol=1e-11,
                                                    precision="fp64")
    assert worst == 0
    xs = split(x.cpu().numpy(), systems)
    for k, s in enumerate(systems):
        Ak = pkg.from_system(s, slice_rows=64)
        xk, st, it, rr = pkg.pcg_solve(Ak, torch.as_tensor(s.b, device="cuda"), tol=1e-11)
        assert st == 0
        assert abs(it - its[k]) <= 0.02 * it + 2
        ref = xk.cpu().numpy()
        assert np.linalg.norm(xs[k] - ref) <= 1e-8 * max(np.linalg.norm(ref), 1e-300)
        Ak.close()
    A.close()


@pytest.mark.parametrize("max_team,scale", [(1, 1.0), (4, 0.25), (32, 0.05)])
def test_batched_schedules(pkg, oracle_mod, max_team, scale):
    systems = small_batch()
    A = pkg.from_systems(systems, slice_rows=32)
    pkg.ldu_batch_schedule(A, max_team=max_team, team_work_scale=scale)
    info = pkg.ldu_batch_info(A)
    assert info["nsys"] == len(systems) and info["max_team"] <= max_team
    x, worst, its, rrs, sts = pkg.pcg_solve_batched(A, cat_b(systems), tol=1e-8,
                                                    precision="mixed")
    assert worst == 0
    for k, (s, xk) in enumerate(zip(systems, split(x.cpu().numpy(), systems))):
        assert oracle_mod.true_relres(s, xk) <= 1.01e-8, (k, max_team, scale)
    A.close()


def test_batched_graph_capture(pkg, oracle_mod):
    systems = small_batch()
    A = pkg.from_systems(systems, slice_rows=64)
    b = cat_b(systems)
    x = torch.zeros_like(b)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pkg.pcg_solve_batched_async(A, b, x, tol=1e-8, precision="mixed", stream=s)   # warm-up
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        x.zero_()
        pkg.pcg_solve_batched_async(A, b, x, tol=1e-8, precision="mixed")
    for _ in range(2):
        x.fill_(7.0)
        g.replay()
        torch.cuda.synchronize()
        worst, its, rrs, sts = pkg.ldu_batch_results(A)
        assert worst == 0
        for k, (sy, xk) in enumerate(zip(systems, split(x.cpu().numpy(), systems))):
            assert oracle_mod.true_relres(sy, xk) <= 1.01e-8
    A.close()


def test_batched_bad_addressing(pkg):
    systems = [lc.poisson_box(3, 3, 3), lc.poisson_box(4, 4, 4)]
    nb = systems[0].neighbour.copy()
    nb[-1] = systems[0].n          # points into the next system
    bad = lc.LduSystem(n=systems[0].n, owner=systems[0].owner, neighbour=nb,
                       diag=systems[0].diag, upper=systems[0].upper, lower=systems[0].lower,
                       b=systems[0].b, coef=systems[0].coef, diag_extra=systems[0].diag_extra)
    with pytest.raises(pkg.LduError) as e:
        pkg.from_systems([bad, systems[1]])
    assert e.value.status == pkg.ldupcg.ERR_BAD_ADDRESSING


def test_batched_config4_full(pkg, oracle_mod):
    """512 systems, cube sides uniform in 8..48 (17.8M cells), mixed to 1e-8
    in one launch; every system checked by the oracle's SpMV, a sample of
    them against separate single-system solves."""
    systems = lc.config4()
    A = pkg.from_systems(systems, slice_rows=64)
    x, worst, its, rrs, sts = pkg.pcg_solve_batched(A, cat_b(systems), tol=1e-8,
                                                    precision="mixed")
    assert worst == 0 and np.all(sts == 0)
    xs = split(x.cpu().numpy(), systems)
    for k, s in enumerate(systems):
        assert oracle_mod.true_relres(s, xs[k]) <= 1.01e-8, (k, its[k])
    for k in (0, 7, 100, 311, 511):
        s = systems[k]
        Ak = pkg.from_system(s, slice_rows=64)
        xk, st, it, rr = pkg.pipecg_solve(Ak, torch.as_tensor(s.b, device="cuda"), tol=1e-8,
                                          precision="mixed")
        assert st == 0
        ref = xk.cpu().numpy()
        assert np.linalg.norm(xs[k] - ref) <= 1e-5 * np.linalg.norm(ref)
        Ak.close()
    A.close()
