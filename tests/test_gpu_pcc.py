"""PCC on the GPU vs the oracle: the span test of Sec. III (extension rule
under periodic boundaries) and the threshold feedback, bit for bit."""
import math

import numpy as np
import pytest

from gpu_util import assert_obs_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0808_2109_gb300 import swgpu
    swgpu.lib()
    return swgpu


def _spans_numpy(L, lab):
    """Extension rule by its definition: some root occupies every column
    (every row)."""
    grid = lab.reshape(L, L)
    cols = [set(np.unique(grid[:, x]).tolist()) for x in range(L)]
    rows = [set(np.unique(grid[y, :]).tolist()) for y in range(L)]
    sx = bool(set.intersection(*cols))
    sy = bool(set.intersection(*rows))
    return int(sx), int(sy)


@pytest.mark.parametrize("L,n", [(2, 300), (3, 300), (5, 300), (16, 400), (33, 300), (64, 300),
                                 (128, 150), (129, 100), (200, 60), (257, 40)])
def test_pcc_small_bit_exact(sw, orc, L, n):
    ref = orc.pcc_chain(L, seed=L + 7)
    ref_obs = ref.run(n)
    with sw.Lattice(L, seed=L + 7, pcc=True) as lat:
        lat.sweep(n)
        obs = lat.observables()
        assert_obs_equal(obs, ref_obs)
        np.testing.assert_array_equal(lat.spins(), ref.spin)
        np.testing.assert_array_equal(lat.labels(), ref.label)
        assert lat.state()["threshold"] == ref.threshold
    # both outcomes of the span test occur in these runs
    flags = ref_obs["spans_x"] | ref_obs["spans_y"]
    if L >= 16:
        assert flags.any() and not flags.all()


def test_pcc_split_calls(sw, orc):
    L = 100
    ref = orc.pcc_chain(L, seed=3)
    with sw.Lattice(L, seed=3, pcc=True) as lat:
        for n in (1, 7, 30, 2):
            lat.sweep(n)
            assert_obs_equal(lat.observables(), ref.run(n))
        np.testing.assert_array_equal(lat.spins(), ref.spin)


def test_pcc_L2048_first_sweeps_bit_exact(sw, orc):
    L, n = 2048, 30
    ref = orc.pcc_chain(L, seed=1)
    ref_obs = ref.run(n)
    with sw.Lattice(L, seed=1, pcc=True) as lat:
        lat.sweep(n)
        assert_obs_equal(lat.observables(), ref_obs)
        np.testing.assert_array_equal(lat.spins(), ref.spin)
        np.testing.assert_array_equal(lat.labels(), ref.label)


def test_pcc_L2048_10000_sweeps(sw, orc):
    """The configured PCC run: every threshold follows from the previous one
    and that sweep's span flag by the feedback rule; p settles near the FK
    percolation threshold of the critical Ising model, 2 - sqrt 2; the last
    sweep's flags match the definition on its labels."""
    L, n = 2048, 10000
    with sw.Lattice(L, seed=1, pcc=True) as lat:
        lat.sweep(n)
        obs = lat.observables()
        lab = lat.labels()
        st = lat.state()
    assert len(obs) == n
    t = 1 << 31
    for k in range(n):
        assert int(obs["threshold"][k]) == t, k
        t = orc.pcc_update(t, k, bool(obs["spans_x"][k] or obs["spans_y"][k]))
    assert st["threshold"] == t
    p = obs["threshold"][9000:].astype(np.float64) / 2.0 ** 32
    assert abs(p.mean() - (2 - math.sqrt(2))) < 0.005, p.mean()
    assert _spans_numpy(L, lab) == (int(obs["spans_x"][-1]), int(obs["spans_y"][-1]))
