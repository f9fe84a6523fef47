"""Pins of the mixed-precision oracle's control logic, step by step.

The end-to-end pins (the solution against dense LU, the iteration count
against FP64 PCG) would not notice a slip that still converges.  These pin
each piece of the replacement policy of or_mixed_pipecg on its own, from the
oracle's event trace:
  (a) the float recurrences: on a unit-diffusivity box with h = 2^-4 every
      matrix value is exact in float, and with a replacement after every
      step the iterates must follow FP64 pipelined PCG (Sec. 4.1) step for
      step, within float rounding;
  (b) the float unit sigma: a power of two changes no float result except its
      exponent, so forcing sigma = 1 must give bitwise the same solution and
      the same iteration and replacement counts;
  (c) deflation of the constant vector (Saad, Yeung, Erhel & Guyomarc'h
      2000): every new direction is A-orthogonal to W = 1, (A W, p) = 0, and
      every replaced residual is orthogonal to W;
  (d) the period rule: with tau = 0 every replacement but the first (forced)
      and the last (predicted convergence or the cap) comes exactly `period`
      steps after the previous one;
  (e) the tau rule: no step is ever taken with (r, u) at or below tau^2 times
      its value at the last replacement, and steps between tau^2 and tau are
      taken (the test compares with tau^2, not tau);
  (f) the predicted-convergence rule: the relres predicted from the recursive
      (r, u) and the ratio ||r64||^2 / (r64, M^-1 r64) agrees with the true
      relres then formed in FP64;
  (g) the step length: the pipelined denominator delta - beta gamma /
      alpha_old (- (a1, u)^2 / c with deflation) that alpha divides by is
      (p, A p) of the new direction in exact arithmetic, and must match it
      to float drift at every step.
Tracing itself changes nothing: a traced run gives bitwise the untraced x.
"""
import numpy as np
import pytest

import ldu_cases as lc


def scaled(s, c):
    """The same system with every matrix value and the right-hand side
    multiplied by c (the same solution; the ratio of (f) scales by c)."""
    return lc.LduSystem(n=s.n, owner=s.owner, neighbour=s.neighbour, diag=c * s.diag,
                        upper=c * s.upper, lower=c * s.lower, b=c * s.b, coef=s.coef,
                        diag_extra=s.diag_extra, shape=s.shape, name=s.name + "-scaled")


def steps_and_reps(oracle_mod, r):
    t = r.trace
    return t[t[:, oracle_mod.TRACE_EVENT] == 0], t[t[:, oracle_mod.TRACE_EVENT] == 1]


@pytest.mark.parametrize("k", [1, 2, 5, 13, 30])
def test_a_period_one_tracks_fp64_pipelined(oracle_mod, k):
    s = lc.config1(s=16)
    for v in (s.diag, s.upper, s.lower):
        assert np.array_equal(v.astype(np.float32).astype(np.float64), v)
    ref = oracle_mod.pipecg(s, tol=1e-30, maxit=k)
    got = oracle_mod.mixed_pipecg(s, tol=1e-30, maxit=k, period=1, tau=0.0)
    assert ref.iters == got.iters == k
    assert np.linalg.norm(got.x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


CASES = [lambda: lc.config2(s=16), lambda: lc.config3(s=16),
         lambda: lc.poisson_box(9, 7, 11, diffusivity="lognormal", seed=5)]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("mode", [dict(period=16, tau=0.3), dict(period=12),
                                  dict(period=16, deflate=True),
                                  dict(period=0, tau=1e-3, restart=True)])
def test_b_sigma_is_exact_scaling(oracle_mod, make, mode):
    s = make()
    a = oracle_mod.mixed_pipecg(s, tol=1e-10, **mode)
    b = oracle_mod.mixed_pipecg(s, tol=1e-10, sigma1=True, **mode)
    assert a.status == b.status == 0
    assert (a.iters, a.replacements) == (b.iters, b.replacements)
    assert np.array_equal(a.x, b.x)


@pytest.mark.parametrize("make", [lambda: lc.config3(s=16), lambda: lc.config2(s=16)])
def test_c_deflation_orthogonality(oracle_mod, make):
    s = make()
    r = oracle_mod.mixed_pipecg(s, tol=1e-10, period=16, deflate=True, trace=True)
    assert r.status == 0
    steps, reps = steps_and_reps(oracle_mod, r)
    assert len(steps) == r.iters and len(reps) == r.replacements
    assert np.max(np.abs(steps[:, oracle_mod.TRACE_STEP_AP])) <= 1e-6
    assert np.max(np.abs(reps[:, oracle_mod.TRACE_REP_WR])) <= 1e-12


@pytest.mark.parametrize("period", [7, 16])
@pytest.mark.parametrize("make", CASES)
def test_d_period_rule(oracle_mod, make, period):
    s = make()
    r = oracle_mod.mixed_pipecg(s, tol=1e-10, period=period, tau=0.0, trace=True)
    assert r.status == 0
    _, reps = steps_and_reps(oracle_mod, r)
    its = reps[:, oracle_mod.TRACE_IT].astype(int)
    trig = reps[:, oracle_mod.TRACE_REP_TRIGGER].astype(int)
    assert its[0] == 0 and trig[0] & oracle_mod.TRIG_FORCED
    assert np.all(np.diff(its[:-1]) == period)
    assert np.all(trig[1:-1] & oracle_mod.TRIG_PERIOD)
    assert 0 < its[-1] - its[-2] <= period
    assert r.replacements == 1 + r.iters // period + (1 if r.iters % period else 0)


@pytest.mark.parametrize("make", CASES)
def test_e_tau_rule(oracle_mod, make):
    s = make()
    tau = 0.3
    r = oracle_mod.mixed_pipecg(s, tol=1e-10, period=0, tau=tau, trace=True)
    assert r.status == 0
    steps, reps = steps_and_reps(oracle_mod, r)
    ratio = steps[:, oracle_mod.TRACE_STEP_GRATIO]
    assert np.all(ratio > tau * tau)
    assert np.any(ratio <= tau)
    trig = reps[1:-1, oracle_mod.TRACE_REP_TRIGGER].astype(int)
    assert np.all(trig & (oracle_mod.TRIG_TAU | oracle_mod.TRIG_FORCED))


@pytest.mark.parametrize("c", [1.0, 100.0, 1e-3])
@pytest.mark.parametrize("make", [lambda: lc.config2(s=16), lambda: lc.config1(s=12)])
def test_f_predicted_relres_matches_true(oracle_mod, make, c):
    s = scaled(make(), c)
    r = oracle_mod.mixed_pipecg(s, tol=1e-10, period=16, trace=True)
    assert r.status == 0
    _, reps = steps_and_reps(oracle_mod, r)
    q = reps[1:, oracle_mod.TRACE_REP_PREDICTED] / reps[1:, oracle_mod.TRACE_REP_RELRES]
    assert np.all((q > 2.0 / 3.0) & (q < 1.5)), q
    # convergence is declared on the FP64 residual the last replacement formed
    assert reps[-1, oracle_mod.TRACE_REP_RELRES] <= 1e-10 and r.relres <= 1e-10


@pytest.mark.parametrize("make,mode,bound", [
    (lambda: lc.config3(s=16), dict(period=16, deflate=True), 1e-3),
    (lambda: lc.config2(s=16), dict(period=16, deflate=True), 1e-3),
    (lambda: lc.config1(s=12), dict(period=16, deflate=True), 1e-3),
    (lambda: lc.config2(s=16), dict(period=16), 1e-2),
    (lambda: lc.config1(s=12), dict(period=16, tau=0.3), 1e-2),
])
def test_g_denominator_is_p_A_p(oracle_mod, make, mode, bound):
    s = make()
    r = oracle_mod.mixed_pipecg(s, tol=1e-10, trace=True, **mode)
    plain = oracle_mod.mixed_pipecg(s, tol=1e-10, **mode)
    assert r.status == 0 and np.array_equal(r.x, plain.x)
    steps, _ = steps_and_reps(oracle_mod, r)
    assert np.max(np.abs(steps[:, oracle_mod.TRACE_STEP_DENOM] - 1.0)) <= bound
