"""Cell renumbering of an LDU system: random permutation and reverse
Cuthill-McKee (RCM, George and Liu 1981; here scipy's implementation).

After renumbering each face is re-oriented so owner < neighbour (swapping
upper and lower when the orientation flips) and faces are re-sorted by
(owner, neighbour), as lduAddressing requires.  Input preparation only.
"""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from .mesh import LduSystem
from . import rng


def renumber(sys_, new_of_old):
    """Return the system with cell c moved to row new_of_old[c]."""
    new_of_old = np.asarray(new_of_old, dtype=np.int64)
    n = sys_.n
    o = new_of_old[sys_.owner]
    nb = new_of_old[sys_.neighbour]
    swap = o > nb
    lo = np.where(swap, nb, o)
    hi = np.where(swap, o, nb)
    up = np.where(swap, sys_.lower, sys_.upper)
    lw = np.where(swap, sys_.upper, sys_.lower)
    order = np.lexsort((hi, lo))
    inv = np.empty(n, dtype=np.int64)
    inv[new_of_old] = np.arange(n, dtype=np.int64)

    def perm_cells(v):
        return None if v is None else np.asarray(v)[inv]

    return LduSystem(
        n=n, owner=lo[order].astype(np.int32), neighbour=hi[order].astype(np.int32),
        diag=perm_cells(sys_.diag), upper=up[order], lower=lw[order], b=perm_cells(sys_.b),
        coef=sys_.coef[order], diag_extra=perm_cells(sys_.diag_extra), shape=sys_.shape,
        cell_of=perm_cells(sys_.cell_of), name=sys_.name, meta=dict(sys_.meta))


def random_order(n, seed):
    """new_of_old for a uniformly random relabelling of n cells."""
    order = rng.permutation(rng.stream_base(seed, "perm"), n)   # new position -> old cell
    new_of_old = np.empty(n, dtype=np.int64)
    new_of_old[order] = np.arange(n, dtype=np.int64)
    return new_of_old


def adjacency(sys_):
    n = sys_.n
    o = sys_.owner.astype(np.int64)
    nb = sys_.neighbour.astype(np.int64)
    data = np.ones(2 * o.shape[0], dtype=np.int8)
    return sp.csr_matrix((data, (np.concatenate([o, nb]), np.concatenate([nb, o]))), shape=(n, n))


def rcm_order(sys_):
    """new_of_old for the RCM ordering of the system's face graph."""
    order = np.asarray(reverse_cuthill_mckee(adjacency(sys_), symmetric_mode=True), dtype=np.int64)
    new_of_old = np.empty(sys_.n, dtype=np.int64)
    new_of_old[order] = np.arange(sys_.n, dtype=np.int64)
    return new_of_old


def bandwidth(sys_):
    if sys_.nfaces == 0:
        return 0
    return int(np.max(sys_.neighbour.astype(np.int64) - sys_.owner.astype(np.int64)))
