"""Checkpoint / resume: a chain saved after n sweeps and resumed (in a fresh
context, even one made with another seed) for m more equals a straight run
of n + m sweeps bit for bit -- plain, PCC (threshold fed back), open
boundaries with the topological rule and cluster sizes, and Potts in 3D."""
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


def _resume_equals_straight(make, n, m):
    with make(1) as straight:
        straight.sweep(n + m)
        ref = straight.observables()
        ref_spins, ref_labels = straight.spins(), straight.labels()
        ref_state = straight.state()
    with make(1) as first:
        first.sweep(n)
        head = first.observables()
        blob = first.save()
    with make(99) as second:            # another seed: the saved one is taken
        second.load(blob)
        assert second.state()["sweep"] == n
        second.sweep(m)
        tail = second.observables()
        assert_obs_equal(np.concatenate([head, tail]), ref, FIELDS)
        np.testing.assert_array_equal(second.spins(), ref_spins)
        np.testing.assert_array_equal(second.labels(), ref_labels)
        st = second.state()
        assert (st["sweep"], st["threshold"], st["seed"]) == (ref_state["sweep"], ref_state["threshold"], 1)


def test_plain(sw):
    _resume_equals_straight(lambda s: sw.Lattice(130, T=2.269185, seed=s), 7, 5)


def test_pcc_threshold_resumes(sw):
    _resume_equals_straight(lambda s: sw.Lattice(64, pcc=True, seed=s), 9, 11)


def test_open_winding_cluster_sizes(sw):
    _resume_equals_straight(lambda s: sw.Lattice(100, T=2.3, seed=s, open=True, wind=True, csize=True), 4, 6)


def test_potts_3d(sw):
    _resume_equals_straight(lambda s: sw.PottsLattice(3, 12, 3, T=1.2, seed=s, csize=True), 5, 4)


def test_load_refuses_other_lattices_and_bad_buffers(sw):
    with sw.Lattice(64, T=2.3, seed=1) as a, sw.Lattice(65, T=2.3, seed=1) as b, \
            sw.Lattice(64, pcc=True, seed=1) as c:
        a.sweep(2)
        blob = a.save()
        for other in (b, c):
            with pytest.raises(sw.SwError) as e:
                other.load(blob)
            assert e.value.code == sw.SW_ERR_ARG
        bad = bytearray(blob)
        bad[0] ^= 0xFF
        with pytest.raises(sw.SwError):
            a.load(bytes(bad))
        spins = bytearray(blob)
        spins[-1] = 7                    # not a spin
        with pytest.raises(sw.SwError):
            a.load(bytes(spins))
        with pytest.raises(sw.SwError):
            a.load(blob[:-1])            # short
        a.load(blob)
        with pytest.raises(sw.SwError) as e:
            a.labels()                   # rebuilt by the next sweep
        assert e.value.code == sw.SW_ERR_STATE
        a.sweep(1)
        a.labels()
