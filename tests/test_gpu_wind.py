"""The topological rule (SW_FLAG_WIND; Sec. III) on the GPU against the
oracle, bit for bit: per-sweep windings (spans_x / spans_y) of plain
lattices, topological PCC (whose feedback makes the whole chain depend on
every flag), every tile height, lattices narrower than a tile (which wrap
onto themselves), open boundaries (no winding possible) and batches mixing
both rules."""
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


def _compare(sw, orc, L, T=None, pcc=False, open_bc=False, seed=1, calls=(4,), tile_h=0, csize=False):
    if pcc:
        ref = orc.pcc_chain(L, seed, open=open_bc, wind=True, csize=csize)
        kw = dict(pcc=True)
    else:
        ref = orc.sw_chain(L, 1.0, T, seed, open=open_bc, wind=True, csize=csize)
        kw = dict(T=T)
    with sw.Lattice(L, seed=seed, tile_h=tile_h, open=open_bc, wind=True, csize=csize, **kw) as lat:
        for n in calls:
            lat.sweep(n)
            obs, want = lat.observables(), ref.run(n)
            assert_obs_equal(obs, want)
            if csize:
                np.testing.assert_array_equal(obs["csize2"], want["csize2"])
            np.testing.assert_array_equal(lat.spins(), ref.spin)
            np.testing.assert_array_equal(lat.labels(), ref.label)
        return ref


@pytest.mark.parametrize("L", [2, 3, 5, 17, 64, 100, 128, 129, 200, 300])
def test_windings_bit_exact(sw, orc, L):
    seen = set()
    for T in (2.0, 2.269185, 2.5):
        ref = orc.sw_chain(L, 1.0, T, L, wind=True)
        with sw.Lattice(L, T=T, seed=L, wind=True) as lat:
            lat.sweep(6)
            obs, want = lat.observables(), ref.run(6)
            assert_obs_equal(obs, want)
            seen |= set(zip(want["spans_x"].tolist(), want["spans_y"].tolist()))
    if L >= 17:   # both outcomes occur, so the flags are not constant
        assert (0, 0) in seen and len(seen) > 1


@pytest.mark.parametrize("tile_h", [32, 64, 96, 128])
@pytest.mark.parametrize("L", [7, 130, 385])
def test_windings_every_tile_height(sw, orc, L, tile_h):
    _compare(sw, orc, L, T=2.269185, seed=L + tile_h, calls=(3, 3), tile_h=tile_h)


@pytest.mark.parametrize("L", [16, 64, 130, 257])
def test_topological_pcc_bit_exact(sw, orc, L):
    _compare(sw, orc, L, pcc=True, seed=5, calls=(10, 25))


def test_topological_pcc_L2048(sw, orc):
    _compare(sw, orc, 2048, pcc=True, seed=1, calls=(20,))


def test_windings_with_open_boundaries_and_cluster_sizes(sw, orc):
    ref = _compare(sw, orc, 130, T=2.269185, open_bc=True, seed=2, calls=(5,), csize=True)
    assert ref.spin.size == 130 * 130
    _compare(sw, orc, 200, pcc=True, seed=3, calls=(15,), csize=True)


def test_both_rules_in_one_batch(sw, orc):
    specs = []
    for r in range(12):
        sp = {"L": [9, 64, 128, 250][r % 4], "sweeps": 8 + r, "seed": 70 + r, "wind": r % 2 == 0}
        if r % 3 == 0:
            sp["pcc"] = True
        else:
            sp["T"] = 2.15 + 0.04 * r
        specs.append(sp)
    with sw.Server() as srv:
        ids = srv.submit(specs, want_spins=True)
        srv.wait_all(120.0)
        got = [srv.poll(i) for i in ids]
    for sp, (res, out) in zip(specs, got):
        assert res.status == 0
        if sp.get("pcc"):
            ch = orc.pcc_chain(sp["L"], sp["seed"], wind=sp["wind"])
        else:
            ch = orc.sw_chain(sp["L"], 1.0, sp["T"], sp["seed"], wind=sp["wind"])
        assert_obs_equal(out["obs"], ch.run(sp["sweeps"]))
        np.testing.assert_array_equal(out["spins"], ch.spin)
        assert res.threshold == ch.threshold
