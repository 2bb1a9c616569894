"""Pin the oracle's Swendsen-Wang chain (Sec. I steps 1-4) to exact results.

* The exact SW transition matrix of the 3x3 periodic lattice, built from the
  oracle's labeller: rows sum to one only if every cluster count is right,
  and the Boltzmann distribution must satisfy detailed balance.
* Brute-force enumeration of the 4x4 lattice (2^16 states): the oracle's
  chain must reproduce <E>/N and <|M|>/N.
* Kaufman's exact partition function of the finite L x L torus: the oracle's
  chain must reproduce <E>/N at L = 64.
"""
import math

import numpy as np
import pytest


# ---------------------------------------------------------------- helpers

def _links(L):
    """Endpoints (i, j) of link l = 2i + d, in link order."""
    i = np.arange(L * L)
    x, y = i % L, i // L
    right = y * L + (x + 1) % L
    down = ((y + 1) % L) * L + x
    a = np.repeat(i, 2)
    b = np.empty(2 * L * L, dtype=np.int64)
    b[0::2], b[1::2] = right, down
    return a, b


def _enumerate(L, T, J=1.0):
    """Exact <E>/N and <|M|>/N of the L x L periodic Ising model."""
    N = L * L
    states = np.arange(1 << N, dtype=np.int64)
    sig = 2 * ((states[:, None] >> np.arange(N)) & 1) - 1
    a, b = _links(L)
    bs = (sig[:, a] * sig[:, b]).sum(axis=1)
    E = -J * bs
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return float((w * E).sum() / Z / N), float((w * np.abs(sig.sum(axis=1))).sum() / Z / N)


def _kaufman_energy(L, T, J=1.0, dps=40):
    """<E>/N from Kaufman's partition function of the L x L torus:
    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4), K = J/T,
    Z1 = prod_r 2cosh(L g_{2r+1}/2), Z2 = prod_r 2sinh(L g_{2r+1}/2),
    Z3 = prod_r 2cosh(L g_{2r}/2),   Z4 = prod_r 2sinh(L g_{2r}/2),
    cosh g_l = cosh2K coth2K - cos(l pi / L) (l >= 1), g_0 = 2K + ln tanh K."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = dps

    def lnZ(K):
        c = mp.cosh(2 * K) / mp.tanh(2 * K)

        def g(l):
            if l == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(l * mp.pi / L))

        odd = [g(2 * r + 1) for r in range(L)]
        even = [g(2 * r) for r in range(L)]
        z1 = mp.fprod(2 * mp.cosh(L * x / 2) for x in odd)
        z2 = mp.fprod(2 * mp.sinh(L * x / 2) for x in odd)
        z3 = mp.fprod(2 * mp.cosh(L * x / 2) for x in even)
        z4 = mp.fprod(2 * mp.sinh(L * x / 2) for x in even)
        return mp.log(mp.mpf(1) / 2) + (L * L / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K)) \
            + mp.log(z1 + z2 + z3 + z4)

    K = mp.mpf(J) / mp.mpf(T)
    dlnZ = mp.diff(lnZ, K)
    return float(-J * dlnZ / (L * L))


def _binned(x, nbins):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nbins
    b = x[: m * nbins].reshape(nbins, m).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


# ------------------------------------------------------ exact 3x3 matrix

@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_exact_sw_transition_matrix_3x3(orc, T):
    L, J = 3, 1.0
    N, nl = L * L, 2 * L * L
    K = J / T
    P = -math.expm1(-2 * K)
    # cluster count c(B) of every bond set B (an 18-bit mask over links)
    masks = np.arange(1 << nl, dtype=np.int64)
    bits = (masks[:, None] >> np.arange(nl)) & 1
    bond_bytes = (bits[:, 0::2] | (bits[:, 1::2] << 1)).astype(np.uint8)
    c = orc.count_clusters_batch(L, bond_bytes)
    nb = bits.sum(axis=1)
    # W(s -> s') = (1-P)^|A(s)| sum_{B subset of A(s) & A(s')} (P/(1-P))^|B| 2^-c(B)
    G = (P / (1 - P)) ** nb * 2.0 ** (-c.astype(np.float64))
    for bit in range(nl):          # subset sums (zeta transform)
        G = G.reshape(-1, 2, 1 << bit)
        G[:, 1, :] += G[:, 0, :]
    G = G.reshape(-1)
    a, b = _links(L)
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


# -------------------------------------------------- 4x4 enumeration

def test_kaufman_formula_matches_enumeration_4x4():
    for T in (2.0, 2.269185, 3.0):
        e_exact, _ = _enumerate(4, T)
        assert abs(_kaufman_energy(4, T) - e_exact) < 1e-10


@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_chain_matches_enumeration_4x4(orc, T):
    L = 4
    e_exact, m_exact = _enumerate(L, T)
    chain = orc.sw_chain(L, 1.0, T, seed=1)
    chain.run(1000)
    obs = chain.run(1_000_000)
    e = orc.energy_per_site(obs, L)
    m = np.abs(obs["mag"]).astype(np.float64) / (L * L)
    e_mean, e_se = _binned(e, 1000)
    m_mean, m_se = _binned(m, 1000)
    assert e_se < 2e-3 and m_se < 2e-3
    assert abs(e_mean - e_exact) < 4 * e_se, (e_mean, e_exact, e_se)
    assert abs(m_mean - m_exact) < 4 * m_se, (m_mean, m_exact, m_se)


# -------------------------------------------------- Kaufman at L = 64

def test_chain_matches_kaufman_energy_64(orc):
    L, T = 64, 2.269185
    e_exact = _kaufman_energy(L, T)
    assert abs(e_exact - (-1.42393907865)) < 1e-9
    chain = orc.sw_chain(L, 1.0, T, seed=1)
    chain.run(100)
    obs = chain.run(40_000)
    e_mean, e_se = _binned(orc.energy_per_site(obs, L), 100)
    assert e_se < 2e-3
    assert abs(e_mean - e_exact) < 4 * e_se, (e_mean, e_exact, e_se)
