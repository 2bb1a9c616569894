"""Pin the oracle's topological rule (Sec. III: a cluster percolates when it
winds around the box).

A cluster winds in x exactly when some cycle of it has non-zero x winding d;
its lift to the m-fold cover of the torus in x is then connected to its own
copy shifted by L for every m coprime to d, and is not for any m when d = 0.
The 2-fold and 3-fold covers (scipy components) therefore decide the rule
on every lattice with L <= 5 (there d <= L < 6) and on random bond sets at
larger L, independently of the oracle's breadth-first unwrapping.
"""
import math

import numpy as np
import pytest


def _cover_connected(L, bond, m, axis):
    """Is some site connected to its own copy shifted by L in the m-fold cover
    (along x for axis 0, y for axis 1) of the torus with these bonds?"""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    W, H = (m * L, L) if axis == 0 else (L, m * L)
    n = W * H
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    X, Y = X.ravel(), Y.ravel()
    b = bond[(Y % L) * L + (X % L)]
    i = Y * W + X
    r = (b & 1).astype(bool)
    d = (b & 2).astype(bool)
    src = np.concatenate([i[r], i[d]])
    dst = np.concatenate([Y[r] * W + (X[r] + 1) % W, ((Y[d] + 1) % H) * W + X[d]])
    g = coo_matrix((np.ones(src.size), (src, dst)), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    base = np.flatnonzero((X < L) & (Y < L))
    shifted = (Y[base] * W + X[base] + L) if axis == 0 else ((Y[base] + L) * W + X[base])
    return bool((comp[base] == comp[shifted]).any())


def _covers(L, bond):
    return tuple(int(_cover_connected(L, bond, 2, a) or _cover_connected(L, bond, 3, a)) for a in (0, 1))


@pytest.mark.parametrize("L", [2, 3, 4, 5, 8, 13])
def test_windings_equal_covering_lattice_components(orc, L):
    rng = np.random.default_rng(100 + L)
    seen = set()
    for k in range(150):
        p = float(rng.uniform(0.2, 1.0))
        spin = rng.integers(0, 2, L * L).astype(np.uint8) if k % 2 else np.ones(L * L, np.uint8)
        bond, _ = orc.bonds(L, int(rng.integers(1 << 30)), k, orc.threshold_p(p), spin)
        got = orc.windings(L, bond)
        assert got == _covers(L, bond), (L, k)
        seen.add(got)
    assert {(0, 0), (1, 1)} <= seen


def test_windings_of_simple_shapes(orc):
    L = 7
    row = np.zeros(L * L, np.uint8)
    row[3 * L: 4 * L] = 1                       # a closed row: winds in x only
    assert orc.windings(L, row) == (1, 0)
    open_row = row.copy()
    open_row[3 * L + L - 1] = 0                 # the same row cut once: no cycle
    assert orc.windings(L, open_row) == (0, 0)
    col = np.zeros(L * L, np.uint8)
    col[np.arange(L) * L + 2] = 2               # a closed column: winds in y only
    assert orc.windings(L, col) == (0, 1)
    stair = np.zeros(L * L, np.uint8)           # a staircase closing after one turn both ways
    for t in range(L):
        stair[t * L + t] |= 1                   # right from (t, t)
        stair[t * L + (t + 1) % L] |= 2         # then down from (t+1, t)
    assert orc.windings(L, stair) == (1, 1)
    loop = np.zeros(L * L, np.uint8)            # a small contractible loop
    loop[0] = 3
    loop[1] = 2
    loop[L] = 1
    assert orc.windings(L, loop) == (0, 0)


def test_winding_implies_extension(orc):
    rng = np.random.default_rng(9)
    for L in (4, 9, 16):
        for k in range(60):
            spin = rng.integers(0, 2, L * L).astype(np.uint8)
            bond, _ = orc.bonds(L, k, k, orc.threshold_p(float(rng.uniform(0.5, 1.0))), spin)
            lab, _ = orc.label(L, bond)
            wx, wy = orc.windings(L, bond)
            sx, sy = orc.spans(L, lab)
            assert wx <= sx and wy <= sy


def test_wind_flag_reports_without_changing_the_chain(orc):
    a = orc.sw_chain(24, 1.0, 2.269185, 3)
    b = orc.sw_chain(24, 1.0, 2.269185, 3, wind=True)
    oa, ob = a.run(20), b.run(20)
    for f in ("bond_sum", "mag", "nclusters", "nbonds", "threshold"):
        np.testing.assert_array_equal(oa[f], ob[f])
    assert (oa["spans_x"] == 0).all() and (ob["spans_x"] | ob["spans_y"]).any()


def test_topological_pcc_approaches_fk_threshold(orc):
    """PCC on the winding rule also drives p to 2 - sqrt(2) (the rules agree
    in the thermodynamic limit, Sec. III), up to an O(1/L) shift."""
    L = 128
    ch = orc.pcc_chain(L, 1, wind=True)
    obs = ch.run(4000)
    p_late = obs["threshold"][-1000:].astype(np.float64) / 2.0 ** 32
    assert abs(p_late.mean() - (2 - math.sqrt(2))) < 2.0 / L
