"""Check the oracle's sweep against the method's definition assembled from
library routines: the (pinned) Philox blocks, numpy for the bond test and the
observables, and scipy's connected components for the clusters.

Definition (a reading: the paper leaves the random numbers unspecified):
  hot start  s_i  = bit (i mod 128) of Philox(floor(i/128), 0, 0, INIT)
  bonds      b_l  = [s_i = s_j] and [word (l mod 4) of Philox(floor(l/4), k, 0, BOND) < t]
  clusters   root(i) = minimum site index of i's cluster
  flip       s_i  = bit (root mod 128) of Philox(floor(root/128), k, 0, SPIN)
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def _words(orc, seed, idx, sweep, stream):
    ctr = np.zeros((idx.size, 4), dtype=np.uint32)
    ctr[:, 0] = idx
    ctr[:, 1] = sweep & 0xFFFFFFFF
    ctr[:, 2] = sweep >> 32
    ctr[:, 3] = stream
    return orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])


def _bit(words, b):
    return ((words[np.arange(b.size), b // 32] >> (b % 32).astype(np.uint32)) & 1).astype(np.uint8)


def _reference_sweep(orc, L, seed, k, t, spin):
    N = L * L
    i = np.arange(N)
    x, y = i % L, i // L
    nbr = np.stack([y * L + (x + 1) % L, ((y + 1) % L) * L + x], axis=1)
    l = 2 * i[:, None] + np.arange(2)[None, :]
    w = _words(orc, seed, (l // 4).ravel(), k, orc.STREAM_BOND)
    u = w[np.arange(l.size), (l % 4).ravel()].reshape(N, 2).astype(np.uint64)
    bonded = (spin[:, None] == spin[nbr]) & (u < np.uint64(t))
    bond = (bonded[:, 0] | (bonded[:, 1] << 1)).astype(np.uint8)
    a = np.concatenate([i[bonded[:, 0]], i[bonded[:, 1]]])
    b = np.concatenate([nbr[bonded[:, 0], 0], nbr[bonded[:, 1], 1]])
    nc, comp = connected_components(coo_matrix((np.ones(a.size), (a, b)), shape=(N, N)),
                                    directed=False)
    mins = np.full(nc, N, dtype=np.int64)
    np.minimum.at(mins, comp, i)
    root = mins[comp]
    ws = _words(orc, seed, root // 128, k, orc.STREAM_SPIN)
    new = _bit(ws, root % 128)
    sig = 2 * new.astype(np.int64) - 1
    obs = dict(bond_sum=int((sig[:, None] * sig[nbr]).sum()), mag=int(sig.sum()),
               nclusters=int(nc), nbonds=int(bonded.sum()), threshold=int(t))
    return bond, root.astype(np.int32), new, obs


@pytest.mark.parametrize("L", [2, 3, 5, 8, 13])
@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_sweeps_match_definition(orc, L, T):
    seed = 1 + L
    t = orc.threshold_T(1.0, T)
    ws = _words(orc, seed, np.arange(L * L) // 128, 0, orc.STREAM_INIT)
    spin_ref = _bit(ws, np.arange(L * L) % 128)
    chain = orc.sw_chain(L, 1.0, T, seed)
    np.testing.assert_array_equal(chain.spin, spin_ref)
    for k in range(6):
        bond_ref, lab_ref, spin_ref, obs_ref = _reference_sweep(orc, L, seed, k, t, spin_ref)
        obs = chain.run(1)[0]
        np.testing.assert_array_equal(chain.bond, bond_ref)
        np.testing.assert_array_equal(chain.label, lab_ref)
        np.testing.assert_array_equal(chain.spin, spin_ref)
        for key, v in obs_ref.items():
            assert int(obs[key]) == v, key


def test_sweep_counter_high_word_is_used(orc):
    """Sweeps beyond 2^32 use the counter's third word: they must differ from
    the sweep with the same low word."""
    L, seed, t = 8, 3, orc.threshold_p(0.6)
    spin = orc.hot_start(L, seed)
    b0, _ = orc.bonds(L, seed, 5, t, spin)
    b1, _ = orc.bonds(L, seed, 5 + (1 << 32), t, spin)
    assert (b0 != b1).any()
    _, _, _, ref = _reference_sweep(orc, L, seed, 5 + (1 << 32), t, spin)
    assert orc.bonds(L, seed, 5 + (1 << 32), t, spin)[1] == ref["nbonds"]


def test_resume_equals_straight_run(orc):
    """State = (spins, seed, sweep, threshold): n sweeps then m sweeps equal
    n + m sweeps in one go."""
    L, seed = 16, 9
    a = orc.sw_chain(L, 1.0, 2.269185, seed)
    oa = np.concatenate([a.run(7), a.run(5)])
    b = orc.sw_chain(L, 1.0, 2.269185, seed)
    ob = b.run(12)
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(a.spin, b.spin)
    c = orc.Chain(L, seed, orc.threshold_T(1.0, 2.269185), spin=b.spin.copy(), sweep=b.sweep)
    d = orc.sw_chain(L, 1.0, 2.269185, seed)
    d.run(12)
    np.testing.assert_array_equal(c.run(3), d.run(3))
