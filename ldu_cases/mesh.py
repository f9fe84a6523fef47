"""Hexahedral box meshes in OpenFOAM-style LDU face addressing, and the
finite-volume Laplacian coefficients the solver is given.

Cells of an nx x ny x nz block are numbered c = i + nx*(j + ny*k).  Internal
faces are listed per owner cell in ascending order, each owner's faces in
the order +x, +y, +z, so that owner < neighbour and faces are sorted by
(owner, neighbour) -- the lduAddressing convention the paper's lduMatrix
uses (Sec. 5).  The matrix is assembled positive (semi)definite: for a face
with coefficient c_f, upper = lower = -c_f and c_f is added to both adjacent
diagonals; Dirichlet walls add 2*k_P*|S|/w_P to the diagonal of the wall cell
(boundary value 0, so the right-hand side is unchanged).

This is input generation only: nothing here is part of the solve.
"""
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np


@dataclass
class LduSystem:
    """One symmetric system A x = b in LDU form (all arrays host numpy)."""
    n: int
    owner: np.ndarray          # int32 [F], owner < neighbour
    neighbour: np.ndarray      # int32 [F]
    diag: np.ndarray           # float64 [n]
    upper: np.ndarray          # float64 [F]   A[owner, neighbour]
    lower: np.ndarray          # float64 [F]   A[neighbour, owner]
    b: np.ndarray              # float64 [n]
    coef: np.ndarray           # float64 [F]   c_f >= 0, upper = lower = -c_f
    diag_extra: np.ndarray     # float64 [n]   boundary / reference-cell part of diag
    shape: Tuple[int, int, int] = (0, 0, 0)
    cell_of: Optional[np.ndarray] = None   # original (i,j,k) cell of each row
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nfaces(self):
        return int(self.owner.shape[0])


def uniform_widths(m):
    return np.full(m, 1.0 / m)


def graded_widths(m, ratio):
    """Symmetric double grading: m/2 cells per half with widths growing
    geometrically from the wall to the centre, the centre cell `ratio` times
    the wall cell, mirrored and normalised so the widths sum to 1."""
    if m % 2 or m < 4:
        raise ValueError("graded axis needs an even number of cells >= 4")
    h = m // 2
    r = ratio ** (1.0 / (h - 1))
    half = r ** np.arange(h, dtype=np.float64)
    w = np.concatenate([half, half[::-1]])
    return w / w.sum()


def box_faces(nx, ny, nz):
    """Internal faces of the block: (owner, neighbour, axis), sorted."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    own, nbr, ax = [], [], []
    for a, (sl_o, sl_n) in enumerate([
            ((slice(None), slice(None), slice(0, nx - 1)), (slice(None), slice(None), slice(1, nx))),
            ((slice(None), slice(0, ny - 1), slice(None)), (slice(None), slice(1, ny), slice(None))),
            ((slice(0, nz - 1), slice(None), slice(None)), (slice(1, nz), slice(None), slice(None)))]):
        o = idx[sl_o].ravel()
        own.append(o)
        nbr.append(idx[sl_n].ravel())
        ax.append(np.full(o.shape[0], a, dtype=np.int8))
    own = np.concatenate(own)
    nbr = np.concatenate(nbr)
    ax = np.concatenate(ax)
    # stable sort by owner keeps the +x, +y, +z (ascending neighbour) order
    order = np.argsort(own, kind="stable")
    return own[order], nbr[order], ax[order]


class BoxGeometry:
    """Cell widths, face areas and centre-to-face distances of a box block."""

    def __init__(self, wx, wy, wz):
        self.w = [np.asarray(wx, float), np.asarray(wy, float), np.asarray(wz, float)]
        self.nx, self.ny, self.nz = (len(v) for v in self.w)
        self.n = self.nx * self.ny * self.nz
        self.owner, self.neighbour, self.axis = box_faces(self.nx, self.ny, self.nz)

    def ijk(self, c):
        c = np.asarray(c, dtype=np.int64)
        return c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)

    def cell_width(self, c, axis):
        i, j, k = self.ijk(c)
        return self.w[axis][(i, j, k)[axis]]

    def face_area(self, c, axis):
        """Area of a face normal to `axis` belonging to cell c."""
        i, j, k = self.ijk(c)
        t = [(1, 2), (0, 2), (0, 1)][axis]
        ijk = (i, j, k)
        return self.w[t[0]][ijk[t[0]]] * self.w[t[1]][ijk[t[1]]]

    def internal_face_geometry(self):
        """(area, d_P, d_N) per internal face: d_* is centre-to-face distance."""
        o, nb, ax = self.owner, self.neighbour, self.axis
        area = np.empty(o.shape[0])
        dP = np.empty(o.shape[0])
        dN = np.empty(o.shape[0])
        for a in range(3):
            m = ax == a
            area[m] = self.face_area(o[m], a)
            dP[m] = 0.5 * self.cell_width(o[m], a)
            dN[m] = 0.5 * self.cell_width(nb[m], a)
        return area, dP, dN

    def wall_cells(self, axis, side):
        """Cells on the wall normal to `axis` (side 0: min, 1: max)."""
        idx = np.arange(self.n, dtype=np.int64).reshape(self.nz, self.ny, self.nx)
        sl = [slice(None)] * 3
        sl[2 - axis] = 0 if side == 0 else -1
        return idx[tuple(sl)].ravel()


def assemble(geo, coef, diag_extra, b, name="", meta=None):
    """Positive LDU assembly from face coefficients and boundary diagonal terms."""
    n = geo.n
    diag = np.array(diag_extra, dtype=np.float64, copy=True)
    diag += np.bincount(geo.owner, weights=coef, minlength=n)
    diag += np.bincount(geo.neighbour, weights=coef, minlength=n)
    up = -np.asarray(coef, dtype=np.float64)
    return LduSystem(
        n=n,
        owner=geo.owner.astype(np.int32), neighbour=geo.neighbour.astype(np.int32),
        diag=diag, upper=up.copy(), lower=up.copy(), b=np.asarray(b, dtype=np.float64),
        coef=np.asarray(coef, dtype=np.float64), diag_extra=np.asarray(diag_extra, np.float64),
        shape=(geo.nx, geo.ny, geo.nz), cell_of=np.arange(n, dtype=np.int64),
        name=name, meta=dict(meta or {}))


def diffusion_coefficients(geo, k_cell, dirichlet_axes=((0, 0), (0, 1))):
    """Face coefficients c_f = k_f |S_f| / |d_PN| with the harmonic-mean face
    diffusivity k_f = 2 k_P k_N / (k_P + k_N), and the Dirichlet wall terms
    2 k_P |S_b| / w_P (wall at half a cell from the centre) for each
    (axis, side) in `dirichlet_axes`; other walls are zero-gradient."""
    area, dP, dN = geo.internal_face_geometry()
    kP = k_cell[geo.owner]
    kN = k_cell[geo.neighbour]
    kf = 2.0 * kP * kN / (kP + kN)
    coef = kf * area / (dP + dN)
    extra = np.zeros(geo.n)
    for axis, side in dirichlet_axes:
        cells = geo.wall_cells(axis, side)
        extra[cells] += 2.0 * k_cell[cells] * geo.face_area(cells, axis) / geo.cell_width(cells, axis)
    return coef, extra


def harmonic_factors(geo, dirichlet_axes=((0, 0), (0, 1))):
    """The geometry of diffusion_coefficients without the diffusivity:
    g_f = |S_f| / |d_PN| per internal face and bfac_P = sum over the
    Dirichlet walls of cell P of 2 |S_b| / w_P, so that for any cell
    diffusivity k the face coefficients are g_f * 2 k_P k_N / (k_P + k_N) and
    the boundary diagonal terms k_P * bfac_P."""
    area, dP, dN = geo.internal_face_geometry()
    g = area / (dP + dN)
    bfac = np.zeros(geo.n)
    for axis, side in dirichlet_axes:
        cells = geo.wall_cells(axis, side)
        bfac[cells] += 2.0 * geo.face_area(cells, axis) / geo.cell_width(cells, axis)
    return g, bfac


def pressure_coefficients(geo, aP):
    """icoFoam-style pressure coefficients c_f = |S_f| / |d_PN| * (1/a)_f with
    1/a interpolated linearly to the face, weight d_N/(d_P+d_N) on the owner."""
    area, dP, dN = geo.internal_face_geometry()
    wgt = dN / (dP + dN)
    inv_a_f = wgt / aP[geo.owner] + (1.0 - wgt) / aP[geo.neighbour]
    return area / (dP + dN) * inv_a_f


def flux_divergence(geo, phi):
    """b_P = sum of phi over faces P owns minus phi over faces where P is
    the neighbour (a discrete divergence; sums to zero)."""
    return (np.bincount(geo.owner, weights=phi, minlength=geo.n)
            - np.bincount(geo.neighbour, weights=phi, minlength=geo.n))
