"""Oracle of the aggregation-AMG preconditioned CG (Sec. 5, the AMG-CG of
Table 2): a plain CPU restatement, step by step, of the method as this
project reads it.  TEST INFRASTRUCTURE ONLY (tests and the CPU baseline).

The paper applies a V-cycle of an aggregation-based AMG, aggregates built
around a distance-2 maximal independent set, with weighted Jacobi
(omega = 4/3) as the smoother.  The reading taken here:

* graph: the off-diagonal non-zeros of A (every connection counts);
* aggregation, rows visited in increasing order:
    phase 1  a row whose neighbours are all unaggregated becomes a root, and
             it and its neighbours form a new aggregate (the roots are a
             greedy distance-2 independent set);
    phase 2  every row still unaggregated joins the phase-1 aggregate of the
             neighbour it is most strongly connected to (largest |a_ij|;
             values within a relative 1e-12 of the best count as ties,
             which go to the lower aggregate number, so that rounding in
             the coarse matrices cannot flip the choice);
    phase 3  rows with no aggregated neighbour (isolated rows) become
             aggregates of their own;
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


TIE = 1e-12   # relative: connection strengths this close count as equal


def csr_of(s, diag=None):
    """The system's matrix as a scipy CSR matrix (both triangles)."""
    n = s.n
    d = s.diag if diag is None else diag
    rows = np.concatenate([np.arange(n), s.owner, s.neighbour])
    cols = np.concatenate([np.arange(n), s.neighbour, s.owner])
    vals = np.concatenate([d, s.upper, s.lower])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def aggregate(A):
    """Aggregate number of every row (phases 1-3 above) and the count.
    Neighbours are visited in increasing column order."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    n = A.shape[0]
    indptr, indices, data = A.indptr, A.indices, A.data
    nbrs = [indices[indptr[i]:indptr[i + 1]] for i in range(n)]
    vals = [data[indptr[i]:indptr[i + 1]] for i in range(n)]
    agg = np.full(n, -1, dtype=np.int64)
    na = 0
    for i in range(n):                                   # phase 1
        nb = [j for j in nbrs[i] if j != i]
        if agg[i] >= 0 or not nb or any(agg[j] >= 0 for j in nb):
            continue
        agg[i] = na
        for j in nb:
            agg[j] = na
        na += 1
    phase1 = agg.copy()
    for i in range(n):                                   # phase 2
        if phase1[i] >= 0:
            continue
        best, best_v = -1, -1.0
        for j, v in zip(nbrs[i], vals[i]):
            if j == i or phase1[j] < 0:
                continue
            a = abs(v)
            if best < 0 or a > best_v * (1.0 + TIE):
                best, best_v = phase1[j], a
            elif a >= best_v * (1.0 - TIE) and phase1[j] < best:
                best, best_v = phase1[j], max(a, best_v)
        agg[i] = best
    for i in range(n):                                   # phase 3
        if agg[i] < 0:
            agg[i] = na
            na += 1
    return agg, na


def jacobi_weight(A):
    """w = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii (Gershgorin)."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    rowsum = np.asarray(abs(A).sum(axis=1)).ravel()
    return 4.0 / (3.0 * np.max(rowsum / d))


def prolongator(A, agg, na, w):
    """P = (I - w D^-1 A) P_t."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    Pt = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    Dinv = sp.diags(1.0 / A.diagonal())
    return sp.csr_matrix(Pt - w * (Dinv @ (A @ Pt)))


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
        A = sp.csr_matrix(P.T @ A @ P)
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
