"""Pin the oracle's open-boundary chain and its open-boundary span rule
(Sec. III: for open boundaries a spanning cluster touches both opposite
borders).

* Brute-force enumeration of the 4x4 open lattice: the open chain must
  reproduce <E>/N and <|M|>/N of the free-boundary Ising model (a wrong link
  set -- a wrap link kept, a border link dropped -- shifts <E>).
* The exact 3x3 SW transition matrix on the 12 links of the open lattice,
  built from the oracle's labeller, is stochastic and in detailed balance
  with the free-boundary Boltzmann weights.
* The touches-both-borders rule equals the extension rule (every column
  occupied) on clusters made without wrap links -- such a cluster's column
  projection is an interval -- so the open rule is checked against the
  pinned periodic span test on open bond sets.
"""
import math

import numpy as np
import pytest


def _open_links(L):
    """Endpoints (i, j) of the links of the open L x L lattice."""
    i = np.arange(L * L)
    x, y = i % L, i // L
    r = x < L - 1
    d = y < L - 1
    a = np.concatenate([i[r], i[d]])
    b = np.concatenate([i[r] + 1, i[d] + L])
    return a, b


def _enumerate_open(L, T, J=1.0):
    N = L * L
    states = np.arange(1 << N, dtype=np.int64)
    sig = 2 * ((states[:, None] >> np.arange(N)) & 1) - 1
    a, b = _open_links(L)
    E = -J * (sig[:, a] * sig[:, b]).sum(axis=1)
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return float((w * E).sum() / Z / N), float((w * np.abs(sig.sum(axis=1))).sum() / Z / N)


def _binned(x, nbins):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nbins
    b = x[: m * nbins].reshape(nbins, m).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


def test_open_bonds_are_the_periodic_draws_without_wrap_links(orc):
    rng = np.random.default_rng(3)
    for L in (2, 3, 5, 16, 33):
        i = np.arange(L * L)
        keep = np.where(i % L < L - 1, 1, 0) | np.where(i // L < L - 1, 2, 0)
        for k in range(4):
            spin = rng.integers(0, 2, L * L).astype(np.uint8)
            t = orc.threshold_p(float(rng.uniform(0.2, 1.0)))
            per, _ = orc.bonds(L, 7 + k, k, t, spin)
            opn, nb = orc.bonds(L, 7 + k, k, t, spin, open=True)
            np.testing.assert_array_equal(opn, per & keep)
            assert nb == int((opn & 1).sum() + ((opn >> 1) & 1).sum())


def test_open_energy_counts_each_interior_link_once(orc):
    for L in (2, 3, 7):
        up = np.ones(L * L, dtype=np.uint8)
        assert orc.measure(L, up, open=True) == (2 * L * (L - 1), L * L)
        # a checkerboard (odd L: not proper across the wrap) has every open link unequal
        cb = ((np.arange(L * L) % L + np.arange(L * L) // L) % 2).astype(np.uint8)
        assert orc.measure(L, cb, open=True)[0] == -2 * L * (L - 1)


@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_open_chain_matches_enumeration_4x4(orc, T):
    L = 4
    e_exact, m_exact = _enumerate_open(L, T)
    chain = orc.sw_chain(L, 1.0, T, seed=2, open=True)
    chain.run(1000)
    obs = chain.run(1_000_000)
    e = orc.energy_per_site(obs, L)
    m = np.abs(obs["mag"]).astype(np.float64) / (L * L)
    e_mean, e_se = _binned(e, 1000)
    m_mean, m_se = _binned(m, 1000)
    assert e_se < 2e-3 and m_se < 2e-3
    assert abs(e_mean - e_exact) < 4 * e_se, (e_mean, e_exact, e_se)
    assert abs(m_mean - m_exact) < 4 * m_se, (m_mean, m_exact, m_se)


@pytest.mark.parametrize("T", [2.0, 3.0])
def test_exact_open_sw_transition_matrix_3x3(orc, T):
    L, J = 3, 1.0
    N = L * L
    a, b = _open_links(L)
    nl = a.size                       # 12 links
    K = J / T
    P = -math.expm1(-2 * K)
    masks = np.arange(1 << nl, dtype=np.int64)
    bits = (masks[:, None] >> np.arange(nl)) & 1
    # bond bytes: link q is site a[q]'s right link (b = a+1) or down link (b = a+L)
    bond_bytes = np.zeros((masks.size, N), dtype=np.uint8)
    for q in range(nl):
        d = 0 if b[q] == a[q] + 1 else 1
        bond_bytes[:, a[q]] |= (bits[:, q] << d).astype(np.uint8)
    c = orc.count_clusters_batch(L, bond_bytes)
    nb = bits.sum(axis=1)
    G = (P / (1 - P)) ** nb * 2.0 ** (-c.astype(np.float64))
    for bit in range(nl):
        G = G.reshape(-1, 2, 1 << bit)
        G[:, 1, :] += G[:, 0, :]
    G = G.reshape(-1)
    states = np.arange(1 << N, dtype=np.int64)
    s = (states[:, None] >> np.arange(N)) & 1
    active = (s[:, a] == s[:, b]).astype(np.int64)
    A = (active << np.arange(nl)).sum(axis=1)
    nA = active.sum(axis=1)
    W = (1 - P) ** nA[:, None] * G[A[:, None] & A[None, :]]
    np.testing.assert_allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    sig = 2 * s - 1
    bsum = (sig[:, a] * sig[:, b]).sum(axis=1)
    pi = np.exp(K * (bsum - bsum.max()))
    pi /= pi.sum()
    flow = pi[:, None] * W
    assert np.abs(flow - flow.T).max() < 1e-12
    np.testing.assert_allclose(pi @ W, pi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("L", [2, 3, 4, 7, 16, 31])
def test_open_spans_equal_extension_rule_on_open_clusters(orc, L):
    rng = np.random.default_rng(L)
    seen = set()
    for k in range(300):
        p = float(rng.uniform(0.3, 1.0))
        spin = rng.integers(0, 2, L * L).astype(np.uint8) if k % 3 else np.ones(L * L, np.uint8)
        bond, _ = orc.bonds(L, int(rng.integers(1 << 30)), k, orc.threshold_p(p), spin, open=True)
        lab, _ = orc.label(L, bond)
        got = orc.spans_open(L, lab)
        assert got == orc.spans(L, lab)
        seen.add(got)
    assert (0, 0) in seen and (1, 1) in seen


def test_open_spans_limits(orc):
    for L in (2, 5, 9):
        lab, _ = orc.label(L, np.zeros(L * L, np.uint8))
        assert orc.spans_open(L, lab) == (0, 0)
        up = np.ones(L * L, np.uint8)
        bond, _ = orc.bonds(L, 1, 0, 1 << 32, up, open=True)
        lab, _ = orc.label(L, bond)
        assert orc.spans_open(L, lab) == (1, 1)
        # one full row of right bonds spans x only; one full column spans y only
        row = np.zeros(L * L, np.uint8)
        row[2 % L * L: 2 % L * L + L - 1] = 1
        lab, _ = orc.label(L, row)
        assert orc.spans_open(L, lab) == (1, 0)
        col = np.zeros(L * L, np.uint8)
        col[np.arange(L - 1) * L + 1 % L] = 2
        lab, _ = orc.label(L, col)
        assert orc.spans_open(L, lab) == (0, 1)


def test_open_pcc_approaches_fk_threshold(orc):
    """Open-boundary PCC drives p to the bond threshold of the critical FK
    clusters, 2 - sqrt(2), up to a finite-size shift of order 1/L."""
    L = 128
    ch = orc.pcc_chain(L, 1, open=True)
    obs = ch.run(4000)
    p_late = obs["threshold"][-1000:].astype(np.float64) / 2.0 ** 32
    assert abs(p_late.mean() - (2 - math.sqrt(2))) < 2.0 / L
    flags = obs["spans_x"] | obs["spans_y"]
    assert 0.2 < flags[-1000:].mean() < 0.8
