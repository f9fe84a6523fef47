"""Pins of the seeded input generators (no solver arithmetic involved)."""
import json
import os

import numpy as np
import pytest

import ldu_cases as lc
from ldu_cases import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")))
    got = rng.raw(1234567, 5)
    assert [int(v) for v in got] == [int(v) for v in ref["outputs"]]


def test_rng_counter_form_and_ranges():
    base = rng.stream_base(0, "rhs")
    a = rng.raw(base, 100)
    assert np.array_equal(a[37:60], rng.raw(base, 23, start=37))
    u = rng.uniform01(base, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = rng.normal(base, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    p = rng.permutation(base, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000))
    k = rng.integers(base, 100000, 8, 48)
    assert k.min() == 8 and k.max() == 48


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 4, 5), (32, 32, 32)])
def test_face_count_and_ordering(shape):
    s = lc.poisson_box(*shape)
    nx, ny, nz = shape
    assert s.nfaces == (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    if nx == ny == nz:
        assert s.nfaces == 3 * nx * nx * (nx - 1)
    o = s.owner.astype(np.int64)
    nb = s.neighbour.astype(np.int64)
    assert np.all(o < nb) and o.min() >= 0 and nb.max() < s.n
    key = o * s.n + nb
    assert np.all(np.diff(key) > 0)          # sorted by (owner, neighbour), no duplicates


def test_config1_sizes():
    s = lc.config1()
    assert (s.n, s.nfaces) == (32768, 95232)


def test_graded_widths():
    w = lc.graded_widths(256, 4.0)
    assert abs(w.sum() - 1.0) < 1e-14
    assert abs(w[127] / w[0] - 4.0) < 1e-12
    assert np.array_equal(w, w[::-1])
    assert np.all(np.diff(w[:128]) > 0)


@pytest.mark.parametrize("make", [
    lambda: lc.config2(s=10),
    lambda: lc.config3(s=8),
    lambda: lc.poisson_box(5, 6, 7, diffusivity="lognormal"),
])
def test_assembly_invariants(make):
    s = make()
    assert np.array_equal(s.upper, s.lower)                 # symmetric storage, bitwise
    assert np.all(s.upper < 0) and np.all(s.diag > 0)
    off = (np.bincount(s.owner, weights=np.abs(s.upper), minlength=s.n)
           + np.bincount(s.neighbour, weights=np.abs(s.lower), minlength=s.n))
    excess = s.diag - off
    scale = s.diag.max()
    assert np.all(excess >= -1e-13 * scale)                 # diagonally dominant
    plain = s.diag_extra == 0
    assert np.all(np.abs(excess[plain]) <= 1e-13 * scale)   # equality without wall terms
    assert np.all(excess[~plain] > 0)                       # strict on wall / pinned rows


def test_pressure_case_neumann_and_divergence():
    s = lc.config3(s=8)
    assert abs(s.b.sum()) <= 1e-12 * np.abs(s.b).sum()      # b is a divergence
    assert np.count_nonzero(s.diag_extra) == 1 and s.diag_extra[0] > 0
    cells = s.meta["widths"]
    assert abs(np.sum(cells) - 1.0) < 1e-14


def test_renumbering_is_a_relabelling():
    s0 = lc.config2(s=9, reorder=False)
    s1 = lc.config2(s=9, reorder=True)
    assert np.array_equal(np.sort(s1.cell_of), np.arange(s0.n))
    # every cell keeps its diagonal and rhs, every face its coefficient
    assert np.array_equal(s1.diag, s0.diag[s1.cell_of])
    assert np.array_equal(s1.b, s0.b[s1.cell_of])
    key0 = set(zip(s0.owner.tolist(), s0.neighbour.tolist(), s0.coef.tolist()))
    co = s1.cell_of
    key1 = set((int(min(co[a], co[b])), int(max(co[a], co[b])), c)
               for a, b, c in zip(s1.owner, s1.neighbour, s1.coef))
    assert key0 == key1


def test_rcm_reduces_bandwidth():
    s0 = lc.config2(s=16, reorder=False)
    srand = lc.renumber(s0, lc.random_order(s0.n, 0))
    srcm = lc.renumber(srand, lc.rcm_order(srand))
    assert lc.bandwidth(srcm) < lc.bandwidth(srand)
    assert lc.bandwidth(srcm) <= lc.bandwidth(s0) * 2


def test_batched_sides():
    sides = lc.config4_sides()
    assert sides.shape == (512,) and sides.min() >= 8 and sides.max() <= 48
    # seeded: same draw twice
    assert np.array_equal(sides, lc.config4_sides())
