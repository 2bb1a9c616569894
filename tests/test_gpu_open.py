"""Open boundaries (SW_FLAG_OPEN; Sec. III treats open and periodic
boundaries): the GPU path against the oracle's open chain, bit for bit --
spins, labels, bonds and every per-sweep integer, including the
open-boundary PCC span test and feedback -- alone and in a batch."""
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


def _compare(sw, orc, L, T=None, p=None, pcc=False, seed=1, calls=(4,), tile_h=0):
    if pcc:
        ref = orc.pcc_chain(L, seed, open=True)
        kw = dict(pcc=True)
    elif T is not None:
        ref = orc.sw_chain(L, 1.0, T, seed, open=True)
        kw = dict(T=T)
    else:
        ref = orc.sw_chain_p(L, p, seed, open=True)
        kw = dict(p=p)
    with sw.Lattice(L, seed=seed, tile_h=tile_h, open=True, **kw) as lat:
        assert lat.state()["open"]
        for n in calls:
            lat.sweep(n)
            assert_obs_equal(lat.observables(), ref.run(n))
            np.testing.assert_array_equal(lat.spins(), ref.spin, err_msg="spins")
            np.testing.assert_array_equal(lat.labels(), ref.label, err_msg="labels")
            np.testing.assert_array_equal(lat.bonds(), ref.bond, err_msg="bonds")
        assert lat.state()["threshold"] == ref.threshold


@pytest.mark.parametrize("L", [2, 3, 5, 31, 33, 64, 100, 128, 129, 200, 257])
def test_open_lattices_bit_exact(sw, orc, L):
    for T in (2.0, 2.269185, 3.0):
        _compare(sw, orc, L, T=T, seed=L + 1, calls=(3, 2))


@pytest.mark.parametrize("tile_h", [32, 64, 96, 128])
@pytest.mark.parametrize("L", [5, 97, 130, 385])
def test_open_every_tile_height(sw, orc, L, tile_h):
    _compare(sw, orc, L, T=2.269185, seed=L + tile_h, calls=(2, 2), tile_h=tile_h)


@pytest.mark.parametrize("L", [2, 33, 130])
@pytest.mark.parametrize("p", [0.0, 1.0, 2 - math.sqrt(2)])
def test_open_bond_probability_limits(sw, orc, L, p):
    _compare(sw, orc, L, p=p, seed=9, calls=(3,))


def test_open_no_bond_leaves_the_lattice(sw):
    L = 300
    with sw.Lattice(L, p=1.0, seed=4, open=True) as lat:
        lat.sweep(1)
        b = lat.bonds().reshape(L, L)
        assert not (b[:, L - 1] & 1).any() and not (b[L - 1, :] & 2).any()


@pytest.mark.parametrize("L", [16, 64, 130, 257])
def test_open_pcc_bit_exact(sw, orc, L):
    _compare(sw, orc, L, pcc=True, seed=3, calls=(10, 20))


def test_open_pcc_L2048_first_sweeps(sw, orc):
    _compare(sw, orc, 2048, pcc=True, seed=1, calls=(15,))


def test_open_and_periodic_jobs_in_one_batch(sw, orc):
    specs = []
    for r in range(16):
        L = [7, 64, 130, 256][r % 4]
        sp = {"L": L, "sweeps": 6 + r, "seed": 40 + r, "open": r % 2 == 0}
        if r % 3 == 0:
            sp["pcc"] = True
        else:
            sp["T"] = 2.0 + 0.05 * r
        specs.append(sp)
    with sw.Server() as srv:
        ids = srv.submit(specs, want_spins=True, want_labels=True)
        srv.wait_all(120.0)
        got = [srv.poll(i) for i in ids]
    for sp, (res, out) in zip(specs, got):
        assert res.status == 0
        if sp.get("pcc"):
            ch = orc.pcc_chain(sp["L"], sp["seed"], open=sp["open"])
        else:
            ch = orc.sw_chain(sp["L"], 1.0, sp["T"], sp["seed"], open=sp["open"])
        assert_obs_equal(out["obs"], ch.run(sp["sweeps"]))
        np.testing.assert_array_equal(out["spins"], ch.spin)
        np.testing.assert_array_equal(out["labels"], ch.label)
        assert res.threshold == ch.threshold
