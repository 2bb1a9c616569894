"""The topological rule on the Potts / 3D path (Sec. III: a cluster percolates
when it winds around the periodic box) against the oracle, bit for bit: the
per-sweep winding flags, and under PCC the thresholds they feed back, with
the states, labels and bond bytes, in 2D and 3D, on lattices of one tile and
of several tiles per axis (ragged last tiles, sides that 4 does not divide)."""
import numpy as np
import pytest

from gpu_util import assert_obs_equal

pytestmark = pytest.mark.gpu
FIELDS = ("bond_sum", "mag", "nclusters", "nbonds", "spans_x", "spans_y", "threshold", "csize2")


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0808_2109_gb300 import swgpu
    swgpu.lib()
    return swgpu


def _compare(sw, orc, dim, L, q, T, seed, calls, pcc=False, open=False):
    ref = orc.PottsChain(dim, L, q, 1.0, T, seed, csize=True, pcc=pcc, open=open, wind=True)
    obs = []
    with sw.PottsLattice(dim, L, q, T=T, seed=seed, csize=True, pcc=pcc, open=open, wind=True) as lat:
        for n in calls:
            lat.sweep(n)
            o = lat.observables()
            assert_obs_equal(o, ref.run(n), FIELDS)
            obs.append(o)
            np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="states")
            np.testing.assert_array_equal(lat.labels(), ref.label, err_msg="labels")
            np.testing.assert_array_equal(lat.bonds(), ref.bond, err_msg="bonds")
        assert lat.state()["threshold"] == ref.threshold
    return np.concatenate(obs)


@pytest.mark.parametrize("dim,L,T", [(2, 2, 1.0), (2, 3, 1.0), (2, 16, 0.9), (2, 33, 1.0), (2, 130, 1.0),
                                     (2, 200, 0.95), (3, 2, 1.8), (3, 3, 1.8), (3, 8, 1.7), (3, 17, 1.8),
                                     (3, 33, 1.8), (3, 40, 1.75), (3, 50, 1.8)])
@pytest.mark.parametrize("q", [2, 3])
def test_potts_wind_bit_exact(sw, orc, dim, L, T, q):
    obs = _compare(sw, orc, dim, L, q, T, seed=L + q, calls=(3, 2))
    assert obs["spans_x"].dtype.kind in "iu"


@pytest.mark.parametrize("dim,L,n", [(2, 24, 200), (2, 129, 100), (3, 8, 150), (3, 36, 40), (3, 50, 30)])
def test_potts_pcc_wind_bit_exact(sw, orc, dim, L, n):
    """PCC with the topological rule as its criterion: every threshold."""
    obs = _compare(sw, orc, dim, L, 3, 1.0, seed=L, calls=(n // 2, n - n // 2), pcc=True)
    flags = obs["spans_x"] | obs["spans_y"]
    assert flags.any() and not flags.all()


@pytest.mark.parametrize("dim,L", [(2, 40), (3, 20)])
def test_potts_open_wind_never_winds(sw, orc, dim, L):
    obs = _compare(sw, orc, dim, L, 2, 0.5 if dim == 2 else 1.0, seed=3, calls=(4,), open=True)
    assert not obs["spans_x"].any() and not obs["spans_y"].any()


def test_potts_wind_checkpoint_resumes(sw, orc):
    dim, L, q = 3, 20, 3
    ref = orc.PottsChain(dim, L, q, 1.0, 1.0, 5, pcc=True, wind=True)
    ref_obs = ref.run(60)
    with sw.PottsLattice(dim, L, q, seed=5, pcc=True, wind=True) as a:
        a.sweep(30)
        blob = a.save()
    with sw.PottsLattice(dim, L, q, seed=8, pcc=True, wind=True) as b:
        b.load(blob)
        b.sweep(30)
        assert_obs_equal(b.observables(), ref_obs[30:], FIELDS[:-1])
        np.testing.assert_array_equal(b.spins(), ref.spin)
    with sw.PottsLattice(dim, L, q, seed=5, pcc=True) as c:   # another kind of lattice refuses it
        with pytest.raises(sw.SwError):
            c.load(blob)


@pytest.mark.parametrize("dim,L,pcc,open,wind", [(2, 130, True, False, False), (3, 40, True, False, False),
                                                 (2, 130, True, True, False), (3, 36, True, True, False),
                                                 (2, 130, False, True, True), (3, 36, True, True, True)])
def test_potts_feature_combinations(sw, orc, dim, L, pcc, open, wind):
    """Cluster sizes with PCC, open boundaries and the topological rule in
    combination, on lattices of several tiles: every field bit for bit."""
    T = 1.0 if dim == 2 else 1.8
    ref = orc.PottsChain(dim, L, 3, 1.0, T, 9, csize=True, pcc=pcc, open=open, wind=wind)
    with sw.PottsLattice(dim, L, 3, T=T, seed=9, csize=True, pcc=pcc, open=open, wind=wind) as lat:
        for n in (7, 5):
            lat.sweep(n)
            assert_obs_equal(lat.observables(), ref.run(n), FIELDS)
            np.testing.assert_array_equal(lat.spins(), ref.spin)
            np.testing.assert_array_equal(lat.labels(), ref.label)
        assert lat.state()["threshold"] == ref.threshold
