"""Full-size GPU checks in the benchmark's launch configuration (default
layout and block shape): the 128^3 lognormal case and the 256^3 graded
pressure case.  The oracle checks every row of the FP64 SpMV and recomputes
the true residual of every returned solution with its own FP64 SpMV."""
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


@pytest.fixture(scope="module")
def case128():
    return lc.config2(s=128)


def test_spmv_128(pkg, oracle_mod, case128):
    s = case128
    A = pkg.from_system(s)
    x = np.random.default_rng(0).uniform(-1, 1, s.n)
    y = pkg.ldu_spmv(A, torch.as_tensor(x, device="cuda")).cpu().numpy()
    y_ref = oracle_mod.spmv(s, x)
    bound = oracle_mod.spmv(s, np.abs(x), diag=s.diag, upper=np.abs(s.upper),
                            lower=np.abs(s.lower))
    assert np.all(np.abs(y - y_ref) <= 1e-13 * bound)
    A.close()


def test_solvers_128(pkg, oracle_mod, case128):
    s = case128
    A = pkg.from_system(s)
    b = torch.as_tensor(s.b, device="cuda")
    its = {}
    for name, call in [("pcg", lambda: pkg.pcg_solve(A, b, tol=1e-8)),
                       ("pipe", lambda: pkg.pipecg_solve(A, b, tol=1e-8, precision="fp64")),
                       ("mixed", lambda: pkg.pipecg_solve(A, b, tol=1e-8, precision="mixed"))]:
        x, st, it, rr = call()
        true_rr = oracle_mod.true_relres(s, x.cpu().numpy())
        assert st == 0 and true_rr <= 1.01e-8, (name, st, it, rr, true_rr)
        its[name] = it
    # the oracle's FP64 PCG takes 752 iterations on this case (seed 0)
    assert abs(its["pcg"] - 752) <= 0.02 * 752 + 2
    assert abs(its["pipe"] - its["pcg"]) <= 0.02 * its["pcg"] + 2
    assert its["mixed"] <= 1.2 * its["pcg"]
    A.close()


def test_pressure_256(pkg, oracle_mod):
    s = lc.config3(s=256)
    A = pkg.from_system(s)
    x = np.random.default_rng(1).uniform(-1, 1, s.n)
    y = pkg.ldu_spmv(A, torch.as_tensor(x, device="cuda")).cpu().numpy()
    y_ref = oracle_mod.spmv(s, x)
    bound = oracle_mod.spmv(s, np.abs(x), diag=s.diag, upper=np.abs(s.upper),
                            lower=np.abs(s.lower))
    assert np.all(np.abs(y - y_ref) <= 1e-13 * bound)
    b = torch.as_tensor(s.b, device="cuda")
    for kw in (dict(precision="fp64"), dict(precision="mixed", deflate=True)):
        xs, st, it, rr = pkg.pipecg_solve(A, b, tol=1e-8, maxit=50000, **kw)
        true_rr = oracle_mod.true_relres(s, xs.cpu().numpy())
        assert st == 0 and true_rr <= 1.01e-8, (kw, st, it, rr, true_rr)
    A.close()
