"""Pin the oracle's Potts / d-dimensional open boundaries and PCC (Sec. III
states the percolation criteria for any dimension and for open as well as
periodic boundaries):

* the d-dimensional extension rule equals the 2D span test (itself pinned by
  the paper's worked example) on 2D labellings, brute force in 3D, and the
  paper's worked example laid along each axis of a 3D lattice;
* open-boundary bonds are the periodic draws with the links that leave the
  lattice removed, and the energy sum drops exactly those links;
* under open boundaries occupying every hyperplane is touching both faces;
* the PCC chain applies the feedback to its own flags, and the threshold of
  the 2D q=3 Potts chain settles near the FK percolation point of the
  critical q-state Potts model, p_c = sqrt(q) / (1 + sqrt(q)).
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "range_operator_example.json")


def _coords(dim, L):
    i = np.arange(L ** dim)
    return [i % L, (i // L) % L, i // (L * L)][:dim]


def _random_bonds(rng, dim, L, p, open=False):
    bond = np.zeros(L ** dim, dtype=np.uint8)
    cs = _coords(dim, L)
    for d in range(dim):
        on = rng.random(L ** dim) < p
        if open:
            on &= cs[d] < L - 1
        bond |= (on.astype(np.uint8) << d)
    return bond


def _brute_spans(dim, L, lab):
    cs = _coords(dim, L)
    out = []
    for a in range(dim):
        cover = {}
        for r, c in zip(lab.tolist(), cs[a].tolist()):
            cover.setdefault(r, set()).add(c)
        out.append(int(any(len(v) == L for v in cover.values())))
    return tuple(out)


@pytest.mark.parametrize("L", [2, 3, 5, 8, 13])
def test_spans_nd_equals_the_2d_span_test(orc, L):
    rng = np.random.default_rng(L)
    for p in (0.3, 0.5, 0.6, 0.8, 1.0):
        for _ in range(20):
            lab, _ = orc.label_nd(2, L, _random_bonds(rng, 2, L, p))
            assert orc.spans_nd(2, L, lab) == orc.spans(L, lab)


@pytest.mark.parametrize("L", [2, 3, 4, 6])
def test_spans_nd_3d_brute_force(orc, L):
    rng = np.random.default_rng(100 + L)
    seen = set()
    for p in (0.2, 0.35, 0.5, 0.7):
        for _ in range(15):
            lab, _ = orc.label_nd(3, L, _random_bonds(rng, 3, L, p))
            got = orc.spans_nd(3, L, lab)
            assert got == _brute_spans(3, L, lab)
            seen.add(got)
    assert len(seen) > 1   # both outcomes occur


def test_paper_range_operator_example_along_each_axis(orc):
    """Sec. III's example (a cluster on columns [0,3] U [5,15] of a 16-wide
    lattice does not span; with column 4 it does) laid along x, y and z."""
    with open(GOLDEN) as f:
        g = json.load(f)
    L = g["L"]
    cols = set()
    for lo, hi in g["after_merge"]["P_x(1)"]:
        cols.update(range(lo, hi + 1))
    for axis in range(3):
        for extra, want in ((set(), 0), ({4}, 1)):
            lab = np.arange(L ** 3, dtype=np.int32)
            sites = []
            for c in sorted(cols | extra):
                xyz = [0, 0, 0]
                xyz[axis] = c
                sites.append(xyz[0] + L * xyz[1] + L * L * xyz[2])
            lab[sites] = min(sites)
            sp = orc.spans_nd(3, L, lab)
            assert sp[axis] == want and sum(sp) == want


@pytest.mark.parametrize("dim,L", [(2, 7), (3, 5)])
def test_open_bonds_are_periodic_draws_without_the_leaving_links(orc, dim, L):
    q, seed, thr = 3, 11, orc.threshold_potts(1.0, 0.9)
    spin = orc.potts_hot_start(dim, L, q, seed)
    per, _ = orc.potts_bonds(dim, L, seed, 4, thr, spin)
    opn, nb = orc.potts_bonds(dim, L, seed, 4, thr, spin, open=True)
    cs = _coords(dim, L)
    keep = np.zeros(L ** dim, dtype=np.uint8)
    for d in range(dim):
        keep |= ((cs[d] < L - 1).astype(np.uint8) << d)
    np.testing.assert_array_equal(opn, per & keep)
    assert nb == int(np.unpackbits(opn).sum())
    # the energy sum over the links that exist
    bs, mag = orc.potts_measure(dim, L, q, spin, open=True)
    want = 0
    i = np.arange(L ** dim)
    for d in range(dim):
        j = i.copy()
        step = L ** d
        j = np.where(cs[d] < L - 1, i + step, i)
        m = cs[d] < L - 1
        want += int((2 * (spin[i[m]] == spin[j[m]]) - 1).sum())
    assert bs == want and mag == int((q * (spin == 0) - 1).sum())


@pytest.mark.parametrize("dim,L", [(2, 6), (2, 11), (3, 4), (3, 5)])
def test_open_spanning_is_touching_both_faces(orc, dim, L):
    rng = np.random.default_rng(7 * L + dim)
    cs = _coords(dim, L)
    for p in (0.4, 0.55, 0.7, 0.9):
        for _ in range(15):
            lab, _ = orc.label_nd(dim, L, _random_bonds(rng, dim, L, p, open=True))
            touch = []
            for a in range(dim):
                lo = set(lab[cs[a] == 0].tolist())
                hi = set(lab[cs[a] == L - 1].tolist())
                touch.append(int(bool(lo & hi)))
            assert orc.spans_nd(dim, L, lab) == tuple(touch)


@pytest.mark.parametrize("dim,L,open", [(2, 24, False), (2, 24, True), (3, 6, False)])
def test_pcc_chain_applies_the_feedback(orc, dim, L, open):
    ch = orc.PottsChain(dim, L, 3, 1.0, 1.0, 5, open=open, pcc=True)
    obs = ch.run(300)
    t = 1 << 31
    for k in range(300):
        assert int(obs["threshold"][k]) == t
        t = orc.pcc_update(t, k, bool(obs["spans_x"][k] or obs["spans_y"][k]))
    assert ch.threshold == t
    flags = obs["spans_x"] | obs["spans_y"]
    assert flags.any() and not flags.all()


def test_pcc_2d_q3_settles_near_the_fk_threshold(orc):
    """The feedback drives p to where a spanning cluster appears half the time:
    the FK percolation point of the critical 2D q-state Potts model,
    sqrt(q) / (1 + sqrt(q)) (0.634 for q = 3), up to an O(1/L) shift of the
    extension rule."""
    L, q = 64, 3
    ch = orc.PottsChain(2, L, q, 1.0, 1.0, 9, pcc=True)
    obs = ch.run(4000)
    p = obs["threshold"][2000:].astype(np.float64) / 2.0 ** 32
    pc = math.sqrt(q) / (1 + math.sqrt(q))
    assert abs(p.mean() - pc) < 2.0 / L, (p.mean(), pc)
