"""Pin the oracle's topological rule in d dimensions (Sec. III: a cluster
percolates when it winds around the periodic box along an axis):

* on 2D bond sets it equals the 2D rule, itself pinned by covering-lattice
  components;
* in 3D it equals brute force on the K-fold covering lattice along each axis
  (K a prime above L^2): a cluster that winds with winding number g along the
  axis lifts to gcd(g, K) = 1 component, one that does not to K components;
* hand-built clusters: a closed line along one axis winds along that axis
  only, a closed layer along the two axes of its plane, a broken line or no
  bond along none; open boundaries never wind;
* the chain reports the rule every sweep and, under PCC, feeds it back.
"""
import numpy as np
import pytest

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import connected_components  # noqa: E402


def _coords(dim, L):
    i = np.arange(L ** dim)
    return [i % L, (i // L) % L, i // (L * L)][:dim]


def _next_prime(n):
    k = n + 1
    while any(k % d == 0 for d in range(2, int(k ** 0.5) + 1)):
        k += 1
    return k


def _cover_wraps(dim, L, bond, ncl):
    """Winding along each axis from the components of the K-fold cover."""
    N = L ** dim
    cs = _coords(dim, L)
    K = _next_prime(L ** (dim - 1))
    out = []
    for a in range(dim):
        rows, cols = [], []
        for d in range(dim):
            has = ((bond >> d) & 1).astype(bool)
            i = np.nonzero(has)[0]
            step = L ** d
            wrap = cs[d][i] == L - 1
            j = np.where(wrap, i - (L - 1) * step, i + step)
            for c in range(K):
                cj = (c + 1) % K if d == a else c
                rows.append(c * N + i)
                cols.append(np.where(wrap, cj, c) * N + j)
        r = np.concatenate(rows)
        cc = np.concatenate(cols)
        g = scipy_sparse.coo_matrix((np.ones(len(r), np.int8), (r, cc)), shape=(K * N, K * N))
        n, _ = connected_components(g, directed=False)
        out.append(int(n < K * ncl))
    return tuple(out)


def _random_bonds(rng, dim, L, p):
    bond = np.zeros(L ** dim, dtype=np.uint8)
    for d in range(dim):
        bond |= ((rng.random(L ** dim) < p).astype(np.uint8) << d)
    return bond


@pytest.mark.parametrize("L", [2, 3, 5, 8])
def test_windings_nd_equals_the_2d_rule(orc, L):
    rng = np.random.default_rng(L)
    for p in (0.3, 0.5, 0.6, 0.8):
        for _ in range(20):
            b = _random_bonds(rng, 2, L, p)
            wx, wy = orc.windings(L, b)
            assert orc.windings_nd(2, L, b) == (wx, wy)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_windings_nd_3d_covering_lattice(orc, L):
    rng = np.random.default_rng(50 + L)
    seen = set()
    for p in (0.25, 0.4, 0.55, 0.7):
        for _ in range(10):
            b = _random_bonds(rng, 3, L, p)
            _, ncl = orc.label_nd(3, L, b)
            got = orc.windings_nd(3, L, b)
            assert got == _cover_wraps(3, L, b, ncl)
            seen.add(got)
    assert len(seen) > 2   # several outcomes occur


def test_windings_nd_2d_covering_lattice(orc):
    rng = np.random.default_rng(7)
    for _ in range(30):
        b = _random_bonds(rng, 2, 5, 0.55)
        _, ncl = orc.label_nd(2, 5, b)
        assert orc.windings_nd(2, 5, b) == _cover_wraps(2, 5, b, ncl)


def test_windings_nd_hand_built(orc):
    L = 6
    N = L ** 3
    x, y, z = _coords(3, L)
    line = np.zeros(N, np.uint8)
    line[(x == 2) & (y == 3)] |= 4          # every z link of the column (2, 3): a closed line
    assert orc.windings_nd(3, L, line) == (0, 0, 1)
    broken = line.copy()
    broken[2 + L * 3 + L * L * 4] = 0      # one link of the line missing
    assert orc.windings_nd(3, L, broken) == (0, 0, 0)
    layer = np.zeros(N, np.uint8)
    layer[z == 1] |= 3                      # every x and y link of the layer z = 1
    assert orc.windings_nd(3, L, layer) == (1, 1, 0)
    assert orc.windings_nd(3, L, np.zeros(N, np.uint8)) == (0, 0, 0)
    # a closed diagonal staircase (+x then +y, L times) winds along x and y
    stair = np.zeros(N, np.uint8)
    for k in range(L):
        stair[k + L * k] |= 1                  # (k, k) -> (k+1, k)
        stair[(k + 1) % L + L * k] |= 2        # (k+1, k) -> (k+1, k+1)
    assert orc.windings_nd(3, L, stair) == (1, 1, 0)


@pytest.mark.parametrize("dim,L", [(2, 9), (3, 5)])
def test_open_boundaries_never_wind(orc, dim, L):
    rng = np.random.default_rng(dim * 10 + L)
    spin = np.zeros(L ** dim, np.uint8)     # all states equal: bonds wherever the link draws one
    for k in range(10):
        b, _ = orc.potts_bonds(dim, L, 3, k, orc.threshold_p(0.9), spin, open=True)
        assert orc.windings_nd(dim, L, b) == (0,) * dim
    periodic, _ = orc.potts_bonds(dim, L, 3, 0, orc.threshold_p(0.9), spin)
    assert orc.windings_nd(dim, L, periodic) == (1,) * dim   # dense bonds wind everywhere
    del rng


@pytest.mark.parametrize("dim,L", [(2, 12), (3, 5)])
@pytest.mark.parametrize("pcc", [False, True])
def test_chain_reports_and_feeds_back_the_rule(orc, dim, L, pcc):
    ch = orc.PottsChain(dim, L, 3, 1.0, 1.0 if dim == 2 else 1.8, 11, pcc=pcc, wind=True)
    t = ch.threshold
    flags = []
    for k in range(60):
        o = ch.run(1)[0]
        w = orc.windings_nd(dim, L, ch.bond)
        assert (int(o["spans_x"]), int(o["spans_y"])) == (w[0], int(any(w[1:])))
        assert int(o["threshold"]) == t
        if pcc:
            t = orc.pcc_update(t, k, bool(w[0] or any(w[1:])))
        flags.append(int(o["spans_x"]) | int(o["spans_y"]))
    assert ch.threshold == t
    assert 0 < sum(flags) < len(flags)
