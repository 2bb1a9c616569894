"""GPU path vs the CPU oracle, through the C ABI.

Spins, labels, bonds and every per-sweep integer observable must be equal bit
for bit; derived FP64 averages within 1e-12 relative.  Sizes cover single and
multiple tiles, ragged right/bottom tiles, odd L (rows that start on an odd
site), L smaller than a tile (the periodic wrap joins a tile to itself) and
L = 2 (two links between the same pair of sites).
"""
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


def _compare(sw, orc, L, T=None, p=None, seed=1, calls=(5,), tile_h=0):
    kw = dict(T=T) if T is not None else dict(p=p)
    kw["tile_h"] = tile_h
    ref = orc.sw_chain(L, 1.0, T, seed) if T is not None else orc.sw_chain_p(L, p, seed)
    with sw.Lattice(L, seed=seed, **kw) as lat:
        np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="hot start")
        for n in calls:
            lat.sweep(n)
            obs = lat.observables()
            ref_obs = ref.run(n)
            assert_obs_equal(obs, ref_obs)
            np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="spins")
            np.testing.assert_array_equal(lat.labels(), ref.label, err_msg="labels")
            np.testing.assert_array_equal(lat.bonds(), ref.bond, err_msg="bonds")
        st = lat.state()
        assert st["sweep"] == sum(calls) and st["threshold"] == ref.threshold


@pytest.mark.parametrize("L", [2, 3, 4, 5, 7, 16, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129,
                               200, 255, 256, 257, 384])
def test_small_lattices_bit_exact(sw, orc, L):
    for T in (2.0, 2.269185, 3.0):
        _compare(sw, orc, L, T=T, seed=L, calls=(4,))


@pytest.mark.parametrize("tile_h", [32, 64, 96, 128])
@pytest.mark.parametrize("L", [5, 95, 97, 130, 200, 385])
def test_every_tile_height(sw, orc, L, tile_h):
    """Results do not depend on the tile height (ragged last tile rows,
    partial sub-tile rows, a lattice narrower than one tile)."""
    _compare(sw, orc, L, T=2.269185, seed=L + tile_h, calls=(3, 2), tile_h=tile_h)


@pytest.mark.parametrize("L", [17, 128, 300])
def test_split_calls_continue_the_chain(sw, orc, L):
    _compare(sw, orc, L, T=2.269185, seed=3, calls=(1, 2, 5, 1))


@pytest.mark.parametrize("L", [2, 33, 130])
@pytest.mark.parametrize("p", [0.0, 1.0, 2 - math.sqrt(2)])
def test_bond_probability_limits(sw, orc, L, p):
    _compare(sw, orc, L, p=p, seed=5, calls=(3,))


@pytest.mark.parametrize("L,T", [(1000, 2.0), (1001, 2.269185), (2048, 3.0), (777, 2.269185)])
def test_medium_lattices(sw, orc, L, T):
    _compare(sw, orc, L, T=T, seed=1, calls=(3,))


def test_critical_L64_1000_sweeps(sw, orc):
    """L=64, T=2.269185, seed 1, hot start, 1000 sweeps: per-sweep E, M and
    cluster counts and the final spins and labels, bit-exact; derived
    averages within 1e-12 relative."""
    L, T, n = 64, 2.269185, 1000
    ref = orc.sw_chain(L, 1.0, T, 1)
    ref_obs = ref.run(n)
    with sw.Lattice(L, T=T, seed=1) as lat:
        lat.sweep(n)
        obs = lat.observables()
        assert_obs_equal(obs, ref_obs)
        np.testing.assert_array_equal(lat.spins(), ref.spin)
        np.testing.assert_array_equal(lat.labels(), ref.label)
    N = L * L
    for field, f in (("bond_sum", lambda o: -o.astype(np.float64) / N),
                     ("mag", lambda o: np.abs(o).astype(np.float64) / N)):
        a = float(np.mean(f(obs[field])))
        b = float(np.mean(f(ref_obs[field])))
        assert abs(a - b) <= 1e-12 * abs(b)


@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_L4096_sweeps_bit_exact(sw, orc, T):
    _compare(sw, orc, 4096, T=T, seed=1, calls=(2, 1))


def test_L16384_first_sweep_bit_exact(sw, orc):
    """The full-size lattice (268M sites) in the benchmark's launch
    configuration: the first sweep from the hot start equals the oracle's."""
    L, T = 16384, 2.269185
    ref = orc.sw_chain(L, 1.0, T, 1)
    ref_obs = ref.run(1)
    with sw.Lattice(L, T=T, seed=1) as lat:
        lat.sweep(1)
        assert_obs_equal(lat.observables(), ref_obs)
        np.testing.assert_array_equal(lat.spins(), ref.spin)
        np.testing.assert_array_equal(lat.labels(), ref.label)
        np.testing.assert_array_equal(lat.bonds(), ref.bond)


def _check_last_sweep_with_oracle(orc, L, seed, k, thr, prev_spins, spins, labels, bonds, o):
    """The oracle as checker of sweep k, step by step on the GPU's own
    intermediates (Sec. I steps 1-4): the bonds it draws on the spins before
    the sweep, the clusters of the GPU's bonds, the flip of the GPU's labels,
    and the observables of the GPU's spins.  Each is compared bit for bit, so
    a labelling that over-merges or misses a bond, or a spin that is not its
    root's SPIN bit, fails here at any size."""
    want_bonds, nb = orc.bonds(L, seed, k, thr, prev_spins)
    np.testing.assert_array_equal(bonds, want_bonds, err_msg="bonds of the last sweep")
    want_labels, nc = orc.label(L, bonds)
    np.testing.assert_array_equal(labels, want_labels, err_msg="clusters of the GPU's bonds")
    np.testing.assert_array_equal(spins, orc.assign(L, seed, k, labels), err_msg="flip of the GPU's labels")
    bs, mag = orc.measure(L, spins)
    assert (int(o["bond_sum"]), int(o["mag"]), int(o["nclusters"]), int(o["nbonds"])) == (bs, mag, nc, nb)


@pytest.mark.parametrize("L,T,n", [(4096, 2.0, 200), (4096, 2.269185, 200), (4096, 3.0, 200),
                                   (16384, 2.269185, 50)])
def test_full_workloads_last_sweep_by_oracle(sw, orc, L, T, n):
    """The full configured runs (200 sweeps at L=4096, 50 at L=16384) in the
    benchmark's launch configuration (autotuned tile height): the last sweep
    is recomputed by the oracle from the spins before it."""
    thr = orc.threshold_T(1.0, T)
    with sw.Lattice(L, T=T, seed=1, tile_h=sw.sw_autotune(L, T)) as lat:
        lat.sweep(n - 1)
        prev = lat.spins()
        lat.sweep(1)
        obs = lat.observables()
        assert len(obs) == n and (obs["threshold"] == thr).all()
        _check_last_sweep_with_oracle(orc, L, 1, n - 1, thr, prev, lat.spins(), lat.labels(), lat.bonds(),
                                      obs[-1])


def test_L32768_first_sweep_bit_exact(sw, orc):
    """The largest lattice the GPU path admits: N = 2^30 sites, so the corner
    site's index 2^30 - 1 is the largest 30-bit root and key.  The first sweep
    from the hot start equals the oracle's."""
    L, T = 32768, 2.269185
    ref = orc.sw_chain(L, 1.0, T, 1)
    ref_obs = ref.run(1)
    with sw.Lattice(L, T=T, seed=1) as lat:
        lat.sweep(1)
        assert_obs_equal(lat.observables(), ref_obs)
        np.testing.assert_array_equal(lat.spins(), ref.spin)
        np.testing.assert_array_equal(lat.labels(), ref.label)
        np.testing.assert_array_equal(lat.bonds(), ref.bond)

