"""The q-state Potts / 3D path (sw_create_potts) against the oracle, bit for
bit: per-sweep observables (with sum |C|^2), states, labels and bond bytes,
in 2D and 3D, for several q and temperatures, including lattices with
doubled links (L = 2) and sizes that are not multiples of anything."""
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


def _compare(sw, orc, dim, L, q, T, seed=1, calls=(3, 2)):
    ref = orc.PottsChain(dim, L, q, 1.0, T, seed, csize=True)
    with sw.PottsLattice(dim, L, q, T=T, seed=seed, csize=True) as lat:
        np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="hot start")
        for n in calls:
            lat.sweep(n)
            assert_obs_equal(lat.observables(), ref.run(n), FIELDS)
            np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="states")
            np.testing.assert_array_equal(lat.labels(), ref.label, err_msg="labels")
            np.testing.assert_array_equal(lat.bonds(), ref.bond, err_msg="bonds")
        st = lat.state()
        assert (st["dim"], st["q"], st["sweep"], st["threshold"]) == (dim, q, sum(calls), ref.threshold)


@pytest.mark.parametrize("q", [2, 3, 4, 7])
@pytest.mark.parametrize("L", [2, 3, 16, 33, 100])
def test_potts_2d_bit_exact(sw, orc, L, q):
    for T in (0.7, 1.0, 1.6):
        _compare(sw, orc, 2, L, q, T, seed=L * 10 + q)


@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("L", [2, 3, 8, 17, 32])
def test_potts_3d_bit_exact(sw, orc, L, q):
    for T in (1.5, 2.26, 4.0):   # 3D Ising (q=2): J_c/T_c ~ 0.443 per J/2 coupling
        _compare(sw, orc, 3, L, q, T, seed=L * 10 + q)


def test_potts_larger_lattices(sw, orc):
    _compare(sw, orc, 3, 64, 2, 2.26, seed=1, calls=(2,))
    _compare(sw, orc, 2, 1024, 3, 1.0 / np.log(1 + np.sqrt(3)), seed=2, calls=(2,))


# Tiles are 128 x 64 sites in 2D and 32 x 16 x 16 in 3D: lattices of several
# tile columns whose last tile is ragged, sides that 4 does not divide (rows
# then start inside a Philox block: per-site draws), and 2 mod 4.
@pytest.mark.parametrize("L", [129, 130, 200, 257])
def test_potts_2d_tiles(sw, orc, L):
    _compare(sw, orc, 2, L, 3, 1.0 / np.log(1 + np.sqrt(3)), seed=L)


@pytest.mark.parametrize("L", [33, 36, 40, 50, 65])
def test_potts_3d_tiles(sw, orc, L):
    _compare(sw, orc, 3, L, 3, 1.8164, seed=L, calls=(2, 1))


def test_potts_no_bonds_and_all_states(sw, orc):
    """T so high that the threshold is 0 (no bond: every site its own cluster)
    and q = 256 (every byte value a state)."""
    _compare(sw, orc, 2, 200, 5, 1e12, seed=3)
    _compare(sw, orc, 3, 40, 2, 1e12, seed=4)
    _compare(sw, orc, 2, 160, 256, 0.3, seed=5)
    _compare(sw, orc, 3, 36, 256, 0.3, seed=6)


def test_potts_set_spins_checks_states(sw):
    with sw.PottsLattice(3, 5, 3, T=1.0) as lat:
        s = np.zeros(125, np.uint8)
        s[7] = 3
        with pytest.raises(sw.SwError) as e:
            lat.set_spins(s)
        assert e.value.code == sw.SW_ERR_ARG
        s[7] = 2
        lat.set_spins(s)
        np.testing.assert_array_equal(lat.spins(), s)
        with pytest.raises(sw.SwError):
            sw.pcc_step(lat.h, 1)


def test_potts_argument_checks(sw):
    for args in ((4, 8, 2), (3, 1, 2), (2, 8, 1), (2, 8, 257), (3, 1025, 2)):
        with pytest.raises(sw.SwError) as e:
            sw.sw_create_potts(*args, 1.0, 1.0, 1)
        assert e.value.code == sw.SW_ERR_ARG
