"""Oracle of the aggregation-AMG preconditioned CG (Sec. 5, the AMG-CG of
Table 2): a plain CPU restatement, step by step, of the method as this
project reads it.  TEST INFRASTRUCTURE ONLY (tests and the CPU baseline).

The paper applies a V-cycle of an aggregation-based AMG, aggregates built
around a distance-2 maximal independent set, with weighted Jacobi
(omega = 4/3) as the smoother, and takes the AMG from CUSP, whose
aggregation forms that independent set in parallel (Bell, Dalton & Olson,
SIAM J. Sci. Comput. 34 (2012)).  The reading taken here:

* graph: the stored off-diagonal entries of A (every stored connection
  counts, whatever its value; sparsity patterns are structural throughout,
  so a coarse entry that cancels to zero is kept);
* priorities: row i of a level has the 64-bit priority h_i, output number
  i + 1 of the SplitMix64 stream with state 0 (Steele, Lea & Flood 2014),
  mix64((i + 1) * 0x9E3779B97F4A7C15) -- distinct for distinct rows;
* distance-2 maximal independent set, Luby-style rounds: every row holds
  the pair (state, h) with state 0 excluded, 1 undecided, 2 root, ordered
  lexicographically.  A round takes, for every row, the largest pair within
  distance 2 (two sweeps of the largest pair over the row and its
  neighbours); an undecided row whose largest pair is its own becomes a
  root, an undecided row whose largest pair is a root's is excluded.  Rounds
  repeat until no row is undecided;
* aggregates: the roots, numbered in increasing row order; then every
  non-root row with a root neighbour joins that root (a row has at most one:
  roots are more than two steps apart); then every row still unassigned
  joins the aggregate of the assigned neighbour it is most strongly
  connected to (largest |a_ij|; values within 1e-12 of the row's largest
  |a_ij| of the best count as ties, which go to the lower aggregate number,
  so that rounding in the coarse matrices cannot flip the choice).  The
  independent set is maximal, so every row is then assigned;
* prolongator: the tentative P_t (P_t[i, agg(i)] = 1) smoothed by one
  weighted-Jacobi step, P = (I - w D^-1 A) P_t, with w = 4 / (3 rho) and rho
  the Gershgorin bound max_i sum_j |a_ij| / a_ii of D^-1 A, so that the
  paper's 4/3 becomes a convergent weight;
* coarse matrices by Galerkin projection, A_c = P^T A P, until a level has at
  most `max_coarse` rows, which is solved exactly;
* V(1,1) cycle with the same weighted Jacobi as smoother, started from zero;
* PCG (Saad Alg. 9.1) with z = V(r), stopping on the recursive ||r||/||b||
  and confirming with the true residual, as the Jacobi oracle does;
* the pipelined form of the same PCG (Table 2's AMG-PipeCG), `amg_pipecg`.
"""
import numpy as np
import scipy.sparse as sp

from ldu_cases import rng

TIE = 1e-12   # relative to a row's strongest connection: strengths this close count as equal
STATE_EXCLUDED, STATE_UNDECIDED, STATE_ROOT = 0, 1, 2


def csr_of(s, diag=None):
    """The system's matrix as a scipy CSR matrix (both triangles, explicit
    zeros kept)."""
    n = s.n
    d = s.diag if diag is None else diag
    rows = np.concatenate([np.arange(n), s.owner, s.neighbour])
    cols = np.concatenate([np.arange(n), s.neighbour, s.owner])
    vals = np.concatenate([d, s.upper, s.lower])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    return A


def priorities(n):
    """h_i = mix64((i + 1) * golden): SplitMix64 outputs 1..n of state 0."""
    return rng.raw(np.uint64(0), n)


def _pattern_with_diagonal(A):
    n = A.shape[0]
    P = sp.csr_matrix((np.ones(A.nnz), A.indices.copy(), A.indptr.copy()), shape=A.shape)
    P = (P + sp.identity(n, format="csr")).tocsr()
    P.sort_indices()
    return P


def _largest_pair(pat, state, h):
    """For every row, the largest (state, h) over the row and its neighbours."""
    st = state[pat.indices]
    ms = np.maximum.reduceat(st, pat.indptr[:-1])
    hh = np.where(st == np.repeat(ms, np.diff(pat.indptr)), h[pat.indices], np.uint64(0))
    mh = np.maximum.reduceat(hh, pat.indptr[:-1])
    return ms, mh


def mis2(A):
    """Roots of the distance-2 maximal independent set (boolean per row) and
    the number of rounds it took."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    pat = _pattern_with_diagonal(A)
    h = priorities(n)
    state = np.full(n, STATE_UNDECIDED, dtype=np.int64)
    rounds = 0
    while np.any(state == STATE_UNDECIDED):
        s1, h1 = _largest_pair(pat, state, h)          # distance 1
        s2, h2 = _largest_pair(pat, s1, h1)            # distance 2
        und = state == STATE_UNDECIDED
        own = und & (s2 == state) & (h2 == h)
        excl = und & ~own & (s2 == STATE_ROOT)
        state[own] = STATE_ROOT
        state[excl] = STATE_EXCLUDED
        rounds += 1
    return state == STATE_ROOT, rounds


def aggregate(A):
    """Aggregate number of every row (see the module docstring) and the count."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    n = A.shape[0]
    root, _ = mis2(A)
    agg = np.full(n, -1, dtype=np.int64)
    roots = np.flatnonzero(root)
    agg[roots] = np.arange(roots.size)
    indptr, indices, data = A.indptr, A.indices, A.data
    rows = np.repeat(np.arange(n), np.diff(indptr))
    first = agg.copy()
    # neighbours of roots (each row has at most one root neighbour)
    hit = root[indices] & ~root[rows] & (indices != rows)
    first[rows[hit]] = agg[indices[hit]]
    out = first.copy()
    for i in np.flatnonzero(first < 0):                  # the rest: strongest assigned neighbour
        row = slice(indptr[i], indptr[i + 1])
        js, vs = indices[row], np.abs(data[row])
        off = js != i
        tol = TIE * (vs[off].max() if off.any() else 0.0)
        best, best_v = -1, -1.0
        for j, a in zip(js, vs):
            if j == i or first[j] < 0:
                continue
            if best < 0 or a > best_v + tol:
                best, best_v = first[j], a
            elif a >= best_v - tol and first[j] < best:
                best, best_v = first[j], max(a, best_v)
        out[i] = best
    if np.any(out < 0):
        raise AssertionError("a row is more than two steps from every root")
    return out, int(roots.size)


def jacobi_weight(A):
    """w = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii (Gershgorin)."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    rowsum = np.asarray(abs(A).sum(axis=1)).ravel()
    return 4.0 / (3.0 * np.max(rowsum / d))


def pattern_of(M):
    """The pattern of M (every stored entry, zeros included) as a matrix of ones."""
    M = sp.csr_matrix(M)
    return sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape)


def on_pattern(pat, M):
    """The values of M on the pattern of pat (zero where M stores nothing)."""
    pat = sp.csr_matrix(pat)
    pat.sort_indices()
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    vals = np.asarray(sp.csr_matrix(M)[rows, pat.indices]).ravel()
    return sp.csr_matrix((vals, pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def structural_product(*mats):
    """The product of sparse matrices on the structural pattern of the
    product of their patterns: entries that cancel to zero are kept."""
    val = sp.csr_matrix(mats[0])
    pat = pattern_of(mats[0])
    for M in mats[1:]:
        val = val @ sp.csr_matrix(M)
        pat = pat @ pattern_of(M)        # sums of ones: no cancellation
    return on_pattern(pat, val)


def prolongator(A, agg, na, w):
    """P = (I - w D^-1 A) P_t, on the structural pattern of (I + A) P_t."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    Pt = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    IA = pattern_of(A) + sp.identity(n, format="csr")        # ones: no cancellation
    pat = IA @ Pt
    num = Pt - w * (sp.diags(1.0 / A.diagonal()) @ (A @ Pt))
    return on_pattern(pat, num)


def galerkin(A, P):
    """A_c = P^T A P on the structural pattern of the triple product."""
    return structural_product(sp.csr_matrix(P.T), sp.csr_matrix(A), sp.csr_matrix(P))


def hierarchy(A, max_coarse=500, max_levels=12):
    """[(A_l, P_l, w_l)] for every level above the coarsest, and the
    coarsest matrix (dense)."""
    levels = []
    A = sp.csr_matrix(A)
    while A.shape[0] > max_coarse and len(levels) < max_levels:
        agg, na = aggregate(A)
        if na >= A.shape[0]:
            break
        w = jacobi_weight(A)
        P = prolongator(A, agg, na, w)
        levels.append((A, P, w))
        A = galerkin(A, P)
    return levels, A.toarray()


def vcycle(levels, coarse, b, lev=0):
    """x = V(b): V(1,1) cycle from zero."""
    if lev == len(levels):
        return np.linalg.solve(coarse, b)
    A, P, w = levels[lev]
    d = A.diagonal()
    x = w * b / d                                        # pre-smoothing from zero
    r = b - A @ x
    x = x + P @ vcycle(levels, coarse, P.T @ r, lev + 1)
    x = x + w * (b - A @ x) / d                          # post-smoothing
    return x


class Result:
    def __init__(self, x, iters, relres, levels):
        self.x, self.iters, self.relres, self.levels = x, iters, relres, levels


def amg_pcg(s, b=None, tol=1e-8, maxit=500, max_coarse=500):
    """PCG with the V-cycle preconditioner."""
    A = csr_of(s)
    b = np.asarray(s.b if b is None else b, dtype=np.float64)
    levels, coarse = hierarchy(A, max_coarse)
    bn = np.linalg.norm(b)
    x = np.zeros(s.n)
    if bn == 0.0:
        return Result(x, 0, 0.0, len(levels) + 1)
    r = b.copy()
    z = vcycle(levels, coarse, r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= tol * bn:
            r = b - A @ x
            if np.linalg.norm(r) <= tol * bn:
                break
            z = vcycle(levels, coarse, r)
            p = z.copy()
            rz = r @ z
            continue
        z = vcycle(levels, coarse, r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    relres = np.linalg.norm(b - A @ x) / bn
    return Result(x, it, relres, len(levels) + 1)


def amg_pipecg(s, b=None, tol=1e-8, maxit=500, max_coarse=500):
    """Pipelined PCG (Ghysels & Vanroose 2014, the preconditioned variant the
    paper's Sec. 4.1 builds on) with M = the V-cycle: one cycle and one
    product per iteration and the three dot products (r, u), (w, u), (r, r)
    of a step formed together.  Recurrences: u = M r, w = A u, m = M w,
    n = A m; z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p;
    x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z.  Stops on the
    recursive ||r|| and confirms with the true residual (a disagreement
    restarts the recurrences from it)."""
    A = csr_of(s)
    b = np.asarray(s.b if b is None else b, dtype=np.float64)
    levels, coarse = hierarchy(A, max_coarse)
    bn = np.linalg.norm(b)
    x = np.zeros(s.n)
    if bn == 0.0:
        return Result(x, 0, 0.0, len(levels) + 1)
    r = b.copy()
    it = 0
    while True:
        # (re)start of the recurrences from the current residual
        u = vcycle(levels, coarse, r)
        w = A @ u
        z = np.zeros(s.n)
        q = np.zeros(s.n)
        sv = np.zeros(s.n)
        p = np.zeros(s.n)
        gamma_old = alpha_old = None
        gamma, delta = r @ u, w @ u
        converged = False
        while it < maxit:
            m = vcycle(levels, coarse, w)
            nv = A @ m
            if gamma_old is None:
                beta, alpha = 0.0, gamma / delta
            else:
                beta = gamma / gamma_old
                alpha = gamma / (delta - beta * gamma / alpha_old)
            z = nv + beta * z
            q = m + beta * q
            sv = w + beta * sv
            p = u + beta * p
            x = x + alpha * p
            r = r - alpha * sv
            u = u - alpha * q
            w = w - alpha * z
            it += 1
            gamma_old, alpha_old = gamma, alpha
            gamma, delta = r @ u, w @ u
            if np.linalg.norm(r) <= tol * bn:
                converged = True
                break
        if not converged:
            break
        r = b - A @ x
        if np.linalg.norm(r) <= tol * bn or it >= maxit:
            break
    relres = np.linalg.norm(b - A @ x) / bn
    return Result(x, it, relres, len(levels) + 1)
