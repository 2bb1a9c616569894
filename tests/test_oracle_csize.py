"""Pin the oracle's cluster estimator sum_C |C|^2 (obs["csize2"]).

Every cluster of a sweep takes an independent fair sign (Sec. I step 3), so
given the clusters E[M^2] = sum_C |C|^2: the mean of csize2 over the chain is
the exact <M^2> of the Ising model.  That identity is checked against
brute-force enumeration of the 4x4 lattice (periodic and open), and the
function itself against its limits and a direct count on random labels.
"""
import math

import numpy as np
import pytest


def _m2_exact(L, T, open_bc, J=1.0):
    N = L * L
    states = np.arange(1 << N, dtype=np.int64)
    sig = 2 * ((states[:, None] >> np.arange(N)) & 1) - 1
    i = np.arange(N)
    x, y = i % L, i // L
    if open_bc:
        r, d = x < L - 1, y < L - 1
        a = np.concatenate([i[r], i[d]])
        b = np.concatenate([i[r] + 1, i[d] + L])
    else:
        a = np.concatenate([i, i])
        b = np.concatenate([y * L + (x + 1) % L, ((y + 1) % L) * L + x])
    E = -J * (sig[:, a] * sig[:, b]).sum(axis=1)
    w = np.exp(-(E - E.min()) / T)
    return float((w * sig.sum(axis=1).astype(np.float64) ** 2).sum() / w.sum())


def _binned(x, nbins):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nbins
    b = x[: m * nbins].reshape(nbins, m).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


def test_csize2_limits_and_scipy_components(orc):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(5)
    for L in (2, 3, 8, 33):
        N = L * L
        lab, _ = orc.label(L, np.zeros(N, np.uint8))
        assert orc.csize2(L, lab) == N                      # P = 0: singletons
        bond, _ = orc.bonds(L, 1, 0, 1 << 32, np.ones(N, np.uint8))
        lab, _ = orc.label(L, bond)
        assert orc.csize2(L, lab) == N * N                  # P = 1, equal spins: one cluster
        for k in range(5):
            spin = rng.integers(0, 2, N).astype(np.uint8)
            bond, _ = orc.bonds(L, 3 + k, k, orc.threshold_p(0.7), spin)
            lab, _ = orc.label(L, bond)
            i = np.arange(N)
            x, y = i % L, i // L
            r = np.flatnonzero(bond & 1)
            d = np.flatnonzero(bond & 2)
            src = np.concatenate([r, d])
            dst = np.concatenate([y[r] * L + (x[r] + 1) % L, ((y[d] + 1) % L) * L + x[d]])
            g = coo_matrix((np.ones(src.size), (src, dst)), shape=(N, N))
            _, comp = connected_components(g, directed=False)
            assert orc.csize2(L, lab) == int((np.bincount(comp) ** 2).sum())


@pytest.mark.parametrize("open_bc", [False, True])
@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_csize2_mean_is_exact_m2_4x4(orc, T, open_bc):
    L = 4
    m2 = _m2_exact(L, T, open_bc)
    ch = orc.sw_chain(L, 1.0, T, seed=7, open=open_bc, csize=True)
    ch.run(1000)
    obs = ch.run(400_000)
    c_mean, c_se = _binned(obs["csize2"], 1000)
    m_mean, m_se = _binned(obs["mag"].astype(np.float64) ** 2, 1000)
    assert abs(c_mean - m2) < 4 * c_se, (c_mean, m2, c_se)
    assert abs(m_mean - m2) < 4 * m_se, (m_mean, m2, m_se)
    # the estimator has the smaller variance (why it is used)
    assert c_se < m_se


def test_csize2_off_by_default(orc):
    ch = orc.sw_chain(16, 1.0, 2.3, seed=1)
    assert (ch.run(3)["csize2"] == 0).all()


@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_bond_count_energy_estimator_4x4(orc, T):
    """<sum sigma sigma> = 2 <nbonds> / P - n_links: each link bonds with
    probability P exactly when its spins agree, so the bond count is an
    energy estimator too (exact value from enumeration)."""
    L = 4
    N = L * L
    states = np.arange(1 << N, dtype=np.int64)
    sig = 2 * ((states[:, None] >> np.arange(N)) & 1) - 1
    i = np.arange(N)
    x, y = i % L, i // L
    a = np.concatenate([i, i])
    b = np.concatenate([y * L + (x + 1) % L, ((y + 1) % L) * L + x])
    bs = (sig[:, a] * sig[:, b]).sum(axis=1)
    w = np.exp((bs - bs.max()) / T)
    exact = float((w * bs).sum() / w.sum())
    P = orc.threshold_T(1.0, T) / 2.0 ** 32
    ch = orc.sw_chain(L, 1.0, T, seed=11)
    ch.run(1000)
    obs = ch.run(400_000)
    est, se = _binned(2.0 * obs["nbonds"] / P - 2 * N, 1000)
    assert abs(est - exact) < 4 * se, (est, exact, se)
