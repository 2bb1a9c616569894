"""Pin the oracle's PCC pieces: the extension-rule span test under periodic
boundaries (Sec. III) and the feedback on the bond threshold."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "range_operator_example.json")


def _labels_for_column_set(L, columns, other_rows=True):
    """A valid min-root labelling in which one cluster occupies exactly the
    given columns of row 0 (and nothing else), every other site alone."""
    lab = np.arange(L * L, dtype=np.int32)
    cols = sorted(columns)
    root = cols[0]
    for c in cols:
        lab[c] = root
    return lab


def test_paper_range_operator_example(orc):
    """Sec. III: after the merge P_x(1) = [0,3] U [5,15] on a 16-wide lattice;
    column 4 is missing, so the cluster does not span; filling it does."""
    with open(GOLDEN) as f:
        g = json.load(f)
    L = g["L"]
    cols = set()
    for lo, hi in g["after_merge"]["P_x(1)"]:
        cols.update(range(lo, hi + 1))
    assert len(cols) == L - 1 and 4 not in cols
    sx, sy = orc.spans(L, _labels_for_column_set(L, cols))
    assert bool(sx) is g["after_merge"]["percolating"] and sy == 0
    # the two pieces before the merge: neither spans either
    before = g["before_merge"]
    for name in ("P_x(1)", "P_x(8)"):
        piece = set()
        for lo, hi in before[name]:
            piece.update(range(lo, hi + 1))
        assert orc.spans(L, _labels_for_column_set(L, piece)) == (0, 0)
    sx, sy = orc.spans(L, _labels_for_column_set(L, cols | {4}))
    assert sx == 1 and sy == 0


def _brute_spans(L, lab):
    grid = lab.reshape(L, L)
    roots = np.unique(lab)
    sx = any(all((grid[:, x] == r).any() for x in range(L)) for r in roots)
    sy = any(all((grid[y, :] == r).any() for y in range(L)) for r in roots)
    return int(sx), int(sy)


@pytest.mark.parametrize("L", [2, 3, 5, 8, 12])
def test_spans_equal_brute_force(orc, L):
    rng = np.random.default_rng(L)
    for p in (0.2, 0.5, 0.6, 0.7, 0.9, 1.0):
        for _ in range(40):
            spin = (rng.random(L * L) < 0.5).astype(np.uint8)
            bond, _ = orc.bonds(L, int(rng.integers(1 << 30)), 0, orc.threshold_p(p), spin)
            lab, _ = orc.label(L, bond)
            assert orc.spans(L, lab) == _brute_spans(L, lab)


def test_spans_row_and_column_are_transposes(orc):
    rng = np.random.default_rng(5)
    L = 16
    for _ in range(50):
        spin = (rng.random(L * L) < 0.5).astype(np.uint8)
        bond, _ = orc.bonds(L, 3, int(rng.integers(100)), orc.threshold_p(0.8), spin)
        lab, _ = orc.label(L, bond)
        labT = lab.reshape(L, L).T.ravel()
        # relabel the transpose to min-root form
        fixed = np.empty_like(labT)
        first = {}
        for i, r in enumerate(labT):
            fixed[i] = first.setdefault(int(r), i)
        sx, sy = orc.spans(L, lab)
        assert orc.spans(L, fixed) == (sy, sx)


def test_pcc_step_schedule(orc):
    assert orc.pcc_delta(0) == 1 << 24       # delta p = 2^-8
    assert orc.pcc_delta(999) == 1 << 24
    assert orc.pcc_delta(1000) == 1 << 23    # halved every 1000 sweeps
    assert orc.pcc_delta(11999) == 1 << 13
    assert orc.pcc_delta(12000) == 1 << 12   # floor 2^-20
    assert orc.pcc_delta(10 ** 9) == 1 << 12
    assert orc.pcc_update(1 << 31, 0, True) == (1 << 31) - (1 << 24)
    assert orc.pcc_update(1 << 31, 0, False) == (1 << 31) + (1 << 24)
    assert orc.pcc_update(5, 0, True) == 0
    assert orc.pcc_update((1 << 32) - 5, 0, False) == 1 << 32


def test_pcc_chain_feedback_is_applied(orc):
    L, seed = 32, 1
    c = orc.pcc_chain(L, seed)
    obs = c.run(300)
    t = 1 << 31
    for k, o in enumerate(obs):
        assert int(o["threshold"]) == t
        t = orc.pcc_update(t, k, bool(o["spans_x"] or o["spans_y"]))
    assert c.threshold == t


def test_pcc_approaches_fk_threshold(orc):
    """At T_c the Fortuin-Kasteleyn clusters of the square-lattice Ising
    model percolate at p = 1 - exp(-2K_c) = 2 - sqrt 2; the feedback must
    drive p there up to a finite-size shift of order 1/L."""
    L = 128
    c = orc.pcc_chain(L, seed=1)
    obs = c.run(4000)
    p = obs["threshold"][2000:].astype(np.float64) / 2.0 ** 32
    assert abs(p.mean() - (2 - math.sqrt(2))) < 2.0 / L, p.mean()
