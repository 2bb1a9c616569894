"""Open boundaries and PCC on the q-state Potts / 3D path (Sec. III states
its percolation criteria for any dimension and for open boundaries) against
the oracle, bit for bit: per-sweep observables (thresholds and span flags
included), states, labels and bond bytes, in 2D and 3D; lattices whose rows
are whole warps (L a multiple of 32) and lattices whose rows are not."""
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


def _compare(sw, orc, dim, L, q, T=1.0, seed=1, calls=(3, 2), open=False, pcc=False):
    ref = orc.PottsChain(dim, L, q, 1.0, T, seed, csize=True, open=open, pcc=pcc)
    with sw.PottsLattice(dim, L, q, T=T, seed=seed, csize=True, open=open, pcc=pcc) as lat:
        np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="hot start")
        obs = []
        for n in calls:
            lat.sweep(n)
            o = lat.observables()
            assert_obs_equal(o, ref.run(n), FIELDS)
            obs.append(o)
            np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="states")
            np.testing.assert_array_equal(lat.labels(), ref.label, err_msg="labels")
            np.testing.assert_array_equal(lat.bonds(), ref.bond, err_msg="bonds")
        st = lat.state()
        assert (st["dim"], st["q"], st["sweep"], st["threshold"]) == (dim, q, sum(calls), ref.threshold)
        assert st["pcc"] == int(pcc) and st["open"] == int(open)
    return np.concatenate(obs)


@pytest.mark.parametrize("dim,L", [(2, 2), (2, 3), (2, 16), (2, 33), (2, 64), (3, 2), (3, 3), (3, 8), (3, 17)])
@pytest.mark.parametrize("q", [2, 3])
def test_potts_open_bit_exact(sw, orc, dim, L, q):
    for T in ((0.7, 1.0, 1.6) if dim == 2 else (1.5, 2.26, 4.0)):
        _compare(sw, orc, dim, L, q, T, seed=L * 10 + q, open=True)


@pytest.mark.parametrize("dim,L,n", [(2, 2, 200), (2, 5, 200), (2, 16, 300), (2, 33, 200), (2, 64, 200),
                                     (2, 100, 100), (3, 2, 200), (3, 4, 200), (3, 8, 150), (3, 17, 60),
                                     (3, 32, 40)])
@pytest.mark.parametrize("open", [False, True])
def test_potts_pcc_bit_exact(sw, orc, dim, L, n, open):
    obs = _compare(sw, orc, dim, L, 3, seed=L + 7, calls=(n // 2, n - n // 2), open=open, pcc=True)
    if L >= 8:   # both outcomes of the span test occur
        flags = obs["spans_x"] | obs["spans_y"]
        assert flags.any() and not flags.all()


@pytest.mark.parametrize("dim,L,n", [(2, 200, 120), (2, 130, 150), (3, 40, 60), (3, 50, 40), (3, 66, 20)])
@pytest.mark.parametrize("open", [False, True])
def test_potts_pcc_several_tiles(sw, orc, dim, L, n, open):
    """Lattices of several tiles along every axis, ragged last tiles, sides
    that 4 does not divide."""
    _compare(sw, orc, dim, L, 3, seed=L + 1, calls=(n // 2, n - n // 2), open=open, pcc=True)


@pytest.mark.parametrize("dim,L", [(2, 200), (2, 257), (3, 40), (3, 50)])
def test_potts_open_several_tiles(sw, orc, dim, L):
    for T in ((0.9, 1.2) if dim == 2 else (1.6, 2.2)):
        _compare(sw, orc, dim, L, 2, T, seed=L, open=True)


def test_potts_pcc_2d_L256(sw, orc):
    """A lattice of 8 x 8 warps per row pattern and 2^16 sites, 300 sweeps."""
    _compare(sw, orc, 2, 256, 3, seed=3, calls=(150, 150), pcc=True)


def test_potts_pcc_checkpoint_resumes(sw, orc):
    """A PCC Potts chain saved and loaded into a new lattice continues with the
    threshold the feedback had reached."""
    dim, L, q = 3, 8, 2
    ref = orc.PottsChain(dim, L, q, 1.0, 1.0, 4, pcc=True)
    ref_obs = ref.run(90)
    with sw.PottsLattice(dim, L, q, seed=4, pcc=True) as a:
        a.sweep(50)
        blob = a.save()
    with sw.PottsLattice(dim, L, q, seed=99, pcc=True) as b:
        b.load(blob)
        b.sweep(40)
        assert_obs_equal(b.observables(), ref_obs[50:], FIELDS[:-1])
        np.testing.assert_array_equal(b.spins(), ref.spin)
        assert b.state()["threshold"] == ref.threshold
