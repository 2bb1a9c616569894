"""Pin the oracle's q-state Potts / d-dimensional SW chain (the cluster
update of Sec. I with "equal spins" read as "equal states", on the periodic
d-dimensional lattice the paper states its method for, Sec. II).

* Labels: scipy connected components on random 2D and 3D bond sets.
* The exact SW transition matrix on tiny lattices (2D L=2 with q=3, 3D L=2
  with q=2, every link pair doubled by the wrap): rows sum to one (any wrong
  cluster count breaks it) and the Boltzmann weights of H = -J sum delta are
  in detailed balance and stationary.
* Chain statistics: <bond_sum> and <mag^2> of the chain against brute-force
  enumeration (2D q=3 L=3, 3^9 states; 3D q=2 L=2).
* The state draw is uniform over the q states; q=2 takes the Ising
  threshold at J_Ising = J/2.
"""
import math

import numpy as np
import pytest


def _links(dim, L):
    N = L ** dim
    i = np.arange(N)
    x, y, z = i % L, (i // L) % L, i // (L * L)
    a, b = [], []
    for d in range(dim):
        xx, yy, zz = x.copy(), y.copy(), z.copy()
        (xx, yy, zz)[d][:] = ((xx, yy, zz)[d] + 1) % L
        a.append(i)
        b.append(xx + L * yy + (L * L * zz if dim == 3 else 0))
    # link l = dim*i + d
    A = np.stack(a, axis=1).ravel()
    B = np.stack(b, axis=1).ravel()
    return A, B


def _enumerate(dim, L, q, J, T):
    N = L ** dim
    states = np.arange(q ** N, dtype=np.int64)
    s = (states[:, None] // (q ** np.arange(N))) % q
    a, b = _links(dim, L)
    eq = (s[:, a] == s[:, b])
    bs = (2 * eq - 1).sum(axis=1)
    E = -J * eq.sum(axis=1)
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    mag = (q * (s == 0) - 1).sum(axis=1).astype(np.float64)
    return float((w * bs).sum() / Z), float((w * mag ** 2).sum() / Z)


def _binned(x, nbins):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nbins
    b = x[: m * nbins].reshape(nbins, m).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


@pytest.mark.parametrize("dim,L", [(2, 2), (2, 5), (2, 9), (3, 2), (3, 3), (3, 6)])
def test_label_nd_equals_scipy_components(orc, dim, L):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(dim * 100 + L)
    N = L ** dim
    a, b = _links(dim, L)
    for k in range(40):
        bond = (rng.random((N, dim)) < rng.uniform(0.05, 0.9)).astype(np.uint8)
        bytes_ = (bond << np.arange(dim)).sum(axis=1).astype(np.uint8)
        lab, nc = orc.label_nd(dim, L, bytes_)
        on = bond.ravel().astype(bool)
        g = coo_matrix((np.ones(on.sum()), (a[on], b[on])), shape=(N, N))
        ncomp, comp = connected_components(g, directed=False)
        assert nc == ncomp
        # labels are the component minima
        mins = np.full(ncomp, N)
        np.minimum.at(mins, comp, np.arange(N))
        np.testing.assert_array_equal(lab, mins[comp])


@pytest.mark.parametrize("dim,L,q,T", [(2, 2, 3, 1.0), (2, 2, 3, 0.6), (3, 2, 2, 2.0)])
def test_exact_potts_transition_matrix(orc, dim, L, q, T):
    J = 1.0
    N = L ** dim
    a, b = _links(dim, L)
    nl = a.size
    P = -math.expm1(-J / T)
    masks = np.arange(1 << nl, dtype=np.int64)
    bits = ((masks[:, None] >> np.arange(nl)) & 1).astype(np.uint8)
    bond_bytes = np.zeros((masks.size, N), dtype=np.uint8)
    for l in range(nl):
        bond_bytes[:, l // dim] |= bits[:, l] << (l % dim)
    c = orc.count_clusters_nd(dim, L, bond_bytes)
    del bond_bytes
    nb = bits.sum(axis=1)
    del bits
    G = (P / (1 - P)) ** nb * float(q) ** (-c.astype(np.float64))
    for bit in range(nl):
        G = G.reshape(-1, 2, 1 << bit)
        G[:, 1, :] += G[:, 0, :]
    G = G.reshape(-1)
    states = np.arange(q ** N, dtype=np.int64)
    s = (states[:, None] // (q ** np.arange(N))) % q
    eq = (s[:, a] == s[:, b]).astype(np.int64)
    A = (eq << np.arange(nl)).sum(axis=1)
    W = (1 - P) ** eq.sum(axis=1)[:, None] * G[A[:, None] & A[None, :]]
    np.testing.assert_allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    pi = np.exp((J / T) * (eq.sum(axis=1) - eq.sum(axis=1).max()))
    pi /= pi.sum()
    flow = pi[:, None] * W
    assert np.abs(flow - flow.T).max() < 1e-12
    np.testing.assert_allclose(pi @ W, pi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim,L,q,T", [(2, 3, 3, 1.0), (2, 3, 3, 0.9), (3, 2, 2, 1.5), (2, 3, 2, 1.2)])
def test_potts_chain_matches_enumeration(orc, dim, L, q, T):
    bs_exact, m2_exact = _enumerate(dim, L, q, 1.0, T)
    ch = orc.PottsChain(dim, L, q, 1.0, T, seed=3)
    ch.run(1000)
    obs = ch.run(400_000)
    bs, bs_se = _binned(obs["bond_sum"], 1000)
    m2, m2_se = _binned(obs["mag"].astype(np.float64) ** 2, 1000)
    assert abs(bs - bs_exact) < 4 * bs_se, (bs, bs_exact, bs_se)
    assert abs(m2 - m2_exact) < 4 * m2_se, (m2, m2_exact, m2_se)


def test_potts_states_are_uniform(orc):
    for q in (2, 3, 5, 7):
        lab = np.arange(200_000, dtype=np.int32)   # every site its own root
        L = int(math.isqrt(lab.size))
        s = orc.potts_assign(2, L, q, 9, 4, lab[: L * L])
        counts = np.bincount(s, minlength=q)
        assert counts.size == q
        exp = s.size / q
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        assert chi2 < 3 * q + 30, (q, counts)


def test_potts_conventions(orc):
    for T in (1.0, 2.269185, 3.0):
        assert orc.threshold_potts(1.0, T) == orc.threshold_T(0.5, T)
    h = orc.potts_hot_start(3, 5, 4, 1)
    assert h.max() < 4 and set(np.unique(h)) == {0, 1, 2, 3}
    up = np.zeros(27, np.uint8)
    assert orc.potts_measure(3, 3, 4, up) == (81, 27 * 3)
