"""Pin the oracle's cluster labelling (Sec. I step 2, Hoshen-Kopelman of
Sec. II.A, min-label rule of Sec. II.B) to scipy's connected components.

Two sites are in one cluster iff a path of bonds joins them; the label of a
site is the minimum site index of its cluster.
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def _edges(L, bond):
    """Bonded links as (i, j) pairs, periodic, from bond bytes."""
    N = L * L
    i = np.arange(N)
    x, y = i % L, i // L
    right = y * L + (x + 1) % L
    down = ((y + 1) % L) * L + x
    mr = (bond & 1).astype(bool)
    md = (bond & 2).astype(bool)
    a = np.concatenate([i[mr], i[md]])
    b = np.concatenate([right[mr], down[md]])
    return a, b


def _scipy_min_labels(L, a, b):
    N = L * L
    g = coo_matrix((np.ones(a.size), (a, b)), shape=(N, N))
    nc, comp = connected_components(g, directed=False)
    mins = np.full(nc, N, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(N))
    return mins[comp].astype(np.int32), nc


@pytest.mark.parametrize("L", [2, 3, 5, 8, 33])
@pytest.mark.parametrize("p", [0.0, 0.3, 0.5, 0.59, 0.8, 1.0])
def test_labels_equal_scipy_components(orc, L, p):
    rng = np.random.default_rng(1000 * L + int(p * 100))
    nsets = 300 if L <= 8 else 60
    for _ in range(nsets):
        bond = ((rng.random(L * L) < p).astype(np.uint8)
                | ((rng.random(L * L) < p).astype(np.uint8) << 1))
        lab, nc = orc.label(L, bond)
        ref, nref = _scipy_min_labels(L, *_edges(L, bond))
        np.testing.assert_array_equal(lab, ref)
        assert nc == nref


@pytest.mark.parametrize("L", [2, 5, 16, 33])
def test_zero_probability_every_site_alone(orc, L):
    spin = orc.hot_start(L, 7)
    bond, nb = orc.bonds(L, 7, 0, 0, spin)
    assert nb == 0 and not bond.any()
    lab, nc = orc.label(L, bond)
    np.testing.assert_array_equal(lab, np.arange(L * L))
    assert nc == L * L


@pytest.mark.parametrize("L", [2, 3, 5, 16, 33])
def test_unit_probability_gives_like_spin_domains(orc, L):
    spin = orc.hot_start(L, 11)
    bond, nb = orc.bonds(L, 11, 3, 1 << 32, spin)
    # every link between equal spins is bonded, no other
    i = np.arange(L * L)
    x, y = i % L, i // L
    eq_r = spin == spin[y * L + (x + 1) % L]
    eq_d = spin == spin[((y + 1) % L) * L + x]
    np.testing.assert_array_equal(bond & 1, eq_r.astype(np.uint8))
    np.testing.assert_array_equal((bond >> 1) & 1, eq_d.astype(np.uint8))
    assert nb == int(eq_r.sum() + eq_d.sum())
    lab, nc = orc.label(L, bond)
    ref, nref = _scipy_min_labels(L, *_edges(L, bond))
    np.testing.assert_array_equal(lab, ref)
    assert nc == nref


@pytest.mark.parametrize("L", [2, 3, 64])
def test_uniform_field_at_unit_probability_is_one_cluster(orc, L):
    spin = np.ones(L * L, dtype=np.uint8)
    bond, nb = orc.bonds(L, 5, 0, 1 << 32, spin)
    assert nb == 2 * L * L
    lab, nc = orc.label(L, bond)
    assert nc == 1 and not lab.any()


def test_batch_counts_match_single_calls(orc):
    rng = np.random.default_rng(3)
    L = 5
    sets = (rng.random((40, L * L)) < 0.5).astype(np.uint8) | \
           ((rng.random((40, L * L)) < 0.5).astype(np.uint8) << 1)
    counts = orc.count_clusters_batch(L, sets)
    for s, c in zip(sets, counts):
        assert orc.label(L, s)[1] == c
