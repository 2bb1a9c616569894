"""The Potts / 3D path at the benchmark's full sizes (2D L = 8192, 3D L = 512,
q = 3 at their critical points), with the oracle as the checker of the last
sweep, step by step on the GPU's own intermediates (Sec. I steps 1-4): the
bonds drawn from the GPU's states before the sweep, the oracle's clusters of the
GPU's bonds, the oracle's new states of the GPU's labels, and the sweep's
observables recomputed from them."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0808_2109_gb300 import swgpu
    swgpu.lib()
    return swgpu


@pytest.mark.parametrize("dim,L,T", [(2, 8192, 1.0 / math.log(1.0 + math.sqrt(3.0))), (3, 512, 1.8164)])
def test_potts_full_size_last_sweep(sw, orc, dim, L, T):
    q, seed = 3, 1
    thr = orc.threshold_potts(1.0, T)
    with sw.PottsLattice(dim, L, q, T=T, seed=seed) as lat:
        lat.sweep(3)
        before = lat.spins()
        lat.observables()
        lat.sweep(1)                      # sweep k = 3
        obs = lat.observables()
        bonds, labels, spins = lat.bonds(), lat.labels(), lat.spins()
    k = 3
    want_bonds, nb = orc.potts_bonds(dim, L, seed, k, thr, before)
    np.testing.assert_array_equal(bonds, want_bonds, err_msg="bonds of the GPU's states")
    want_labels, ncl = orc.label_nd(dim, L, bonds)
    np.testing.assert_array_equal(labels, want_labels, err_msg="clusters of the GPU's bonds")
    np.testing.assert_array_equal(spins, orc.potts_assign(dim, L, q, seed, k, labels),
                                  err_msg="new states of the GPU's labels")
    bs, mag = orc.potts_measure(dim, L, q, spins)
    o = obs[0]
    assert (int(o["bond_sum"]), int(o["mag"]), int(o["nclusters"]), int(o["nbonds"])) == (bs, mag, ncl, nb)
    assert int(o["threshold"]) == thr
