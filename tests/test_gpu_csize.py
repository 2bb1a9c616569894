"""The cluster estimator sum_C |C|^2 (SW_FLAG_CSIZE) against the oracle, bit
for bit per sweep: interior clusters (sized inside their tile) and clusters
that cross tiles (piece sizes added at the root node by the merge), for
every tile height, periodic and open boundaries, PCC, and batched jobs."""
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


def _compare(sw, orc, L, T=None, p=None, pcc=False, open_bc=False, seed=1, calls=(3,), tile_h=0):
    if pcc:
        ref = orc.pcc_chain(L, seed, open=open_bc, csize=True)
        kw = dict(pcc=True)
    elif T is not None:
        ref = orc.sw_chain(L, 1.0, T, seed, open=open_bc, csize=True)
        kw = dict(T=T)
    else:
        ref = orc.sw_chain_p(L, p, seed, open=open_bc, csize=True)
        kw = dict(p=p)
    with sw.Lattice(L, seed=seed, tile_h=tile_h, open=open_bc, csize=True, **kw) as lat:
        for n in calls:
            lat.sweep(n)
            assert_obs_equal(lat.observables(), ref.run(n), FIELDS)
            np.testing.assert_array_equal(lat.labels(), ref.label)


@pytest.mark.parametrize("L", [2, 3, 5, 33, 100, 129, 257, 1000])
def test_csize2_bit_exact(sw, orc, L):
    for T in (2.0, 2.269185, 3.0):
        _compare(sw, orc, L, T=T, seed=L, calls=(2, 3))


@pytest.mark.parametrize("tile_h", [32, 64, 96, 128])
@pytest.mark.parametrize("L", [7, 130, 385])
def test_csize2_every_tile_height(sw, orc, L, tile_h):
    _compare(sw, orc, L, T=2.269185, seed=L + tile_h, calls=(2, 2), tile_h=tile_h)


@pytest.mark.parametrize("p", [0.0, 1.0])
def test_csize2_limits(sw, orc, p):
    _compare(sw, orc, 200, p=p, seed=2, calls=(2,))


def test_csize2_open_and_pcc(sw, orc):
    _compare(sw, orc, 130, T=2.269185, open_bc=True, seed=3, calls=(4,))
    _compare(sw, orc, 257, pcc=True, seed=4, calls=(12,))
    _compare(sw, orc, 100, pcc=True, open_bc=True, seed=5, calls=(12,))


def test_csize2_L4096(sw, orc):
    _compare(sw, orc, 4096, T=2.269185, seed=1, calls=(2,))


def test_csize2_is_zero_without_the_flag(sw):
    with sw.Lattice(64, T=2.3, seed=1) as lat:
        lat.sweep(3)
        assert (lat.observables()["csize2"] == 0).all()


def test_csize2_in_a_batch(sw, orc):
    specs = [{"L": L, "T": 2.1 + 0.1 * r, "sweeps": 5 + r, "seed": 60 + r, "csize": r % 2 == 0,
              "open": r % 3 == 0} for r, L in enumerate([9, 64, 128, 200, 256, 333])]
    with sw.Server() as srv:
        ids = srv.submit(specs)
        srv.wait_all(120.0)
        got = [srv.poll(i) for i in ids]
    for sp, (res, out) in zip(specs, got):
        assert res.status == 0
        ch = orc.sw_chain(sp["L"], 1.0, sp["T"], sp["seed"], open=sp["open"], csize=sp["csize"])
        assert_obs_equal(out["obs"], ch.run(sp["sweeps"]), FIELDS)
