"""pcg_solve_ldu_noalloc: the allocation-free solve for callers that cannot
call cudaMalloc (their device memory belongs to another allocator, or they
cannot take cudaMalloc's implicit device synchronisation).

It must give what pcg_solve gives on a default handle of the same matrix,
twice in a row (the fixed device scratch is shared by consecutive calls and
keeps the previous call's contents), from a zero and from a non-zero initial
guess, and refuse inputs beyond its fixed maximum: cells and faces before any
GPU work, stored slots after the device has counted them, after which the
next call must still solve correctly.  The file name makes pytest collect it
last, so a failure here does not hide the results of the other tests."""
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


def dev(a, dt=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t if dt is None else t.to(dt)


@pytest.mark.parametrize("make", [lambda: lc.config2(s=20), lambda: lc.config1(s=32),
                                  lambda: lc.config3(s=16)])
def test_noalloc_matches_pcg_solve_twice(pkg, make):
    s = make()
    A = pkg.from_system(s)
    b = dev(s.b)
    x_ref, st_ref, it_ref, rr_ref = pkg.pcg_solve(A, b, tol=1e-10)
    assert st_ref == 0
    arrays = (dev(s.owner, torch.int32), dev(s.neighbour, torch.int32), dev(s.diag),
              dev(s.upper), dev(s.lower))
    for call in range(2):
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        x, st, it, rr = pkg.pcg_solve_ldu_noalloc(s.n, *arrays, b, x, tol=1e-10)
        assert st == 0, (call, st)
        assert it == it_ref and abs(rr - rr_ref) <= 1e-3 * rr_ref
        err = torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)
        assert float(err) <= 1e-9, (call, float(err))
    A.close()


def test_noalloc_rejects_sizes_beyond_its_maximum(pkg):
    n = 32769
    z64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    e32 = torch.zeros(0, dtype=torch.int32, device="cuda")
    e64 = torch.zeros(0, dtype=torch.float64, device="cuda")
    _, st, _, _ = pkg.pcg_solve_ldu_noalloc(n, e32, e32, z64 + 1.0, e64, e64, z64, z64.clone(),
                                            check=False)
    assert st == pkg.ldupcg.ERR_UNSUPPORTED


def test_noalloc_warm_start_matches_pcg_solve(pkg):
    """The initial guess is read from x: both entry points start from the same
    non-zero x0 and must end at the same iterate."""
    s = lc.config2(s=18, seed=2)
    A = pkg.from_system(s)
    b = dev(s.b)
    x0 = dev(np.random.default_rng(7).uniform(-1, 1, s.n))
    x_ref, st_ref, it_ref, rr_ref = pkg.pcg_solve(A, b, x0.clone(), tol=1e-10)
    arrays = (dev(s.owner, torch.int32), dev(s.neighbour, torch.int32), dev(s.diag),
              dev(s.upper), dev(s.lower))
    for call in range(2):
        x, st, it, rr = pkg.pcg_solve_ldu_noalloc(s.n, *arrays, b, x0.clone(), tol=1e-10)
        assert st == 0 and it == it_ref, (call, st, it, it_ref)
        err = torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)
        assert float(err) <= 1e-9, (call, float(err))
    A.close()


def test_noalloc_refuses_rows_beyond_its_slot_capacity(pkg):
    """A star: cell 0 shares a face with each of the 4095 others, so the first
    128-row slice is 4095 slots wide (524,160 slots) while the scratch holds
    262,144.  The count happens on the device after validation; the call
    returns UNSUPPORTED before anything is written past the capacity, and a
    normal call afterwards still matches pcg_solve."""
    n = 4096
    own = np.zeros(n - 1, dtype=np.int32)
    nbr = np.arange(1, n, dtype=np.int32)
    diag = np.full(n, 2.0)
    diag[0] = float(n)
    off = -np.ones(n - 1)
    b = dev(np.ones(n))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st, _, _ = pkg.pcg_solve_ldu_noalloc(n, dev(own), dev(nbr), dev(diag), dev(off), dev(off),
                                            b, x, check=False)
    assert st == pkg.ldupcg.ERR_UNSUPPORTED
    s = lc.config2(s=16)
    A = pkg.from_system(s)
    x_ref, st_ref, it_ref, _ = pkg.pcg_solve(A, dev(s.b), tol=1e-10)
    x, st, it, _ = pkg.pcg_solve_ldu_noalloc(
        s.n, dev(s.owner, torch.int32), dev(s.neighbour, torch.int32), dev(s.diag),
        dev(s.upper), dev(s.lower), dev(s.b), torch.zeros(s.n, dtype=torch.float64,
                                                         device="cuda"), tol=1e-10)
    assert st == 0 and it == it_ref
    assert float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)) <= 1e-9
    A.close()
