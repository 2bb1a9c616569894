"""Batched and served runs: every job equals the oracle (and so the same
lattice run alone), whatever runs beside it, whenever it joins, and
whatever tile height it gets."""
import time

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


def _oracle(orc, sp):
    if sp.get("pcc"):
        ch = orc.pcc_chain(sp["L"], sp["seed"])
    elif sp.get("p") is not None:
        ch = orc.sw_chain_p(sp["L"], sp["p"], sp["seed"])
    else:
        ch = orc.sw_chain(sp["L"], 1.0, sp["T"], sp["seed"])
    obs = ch.run(sp["sweeps"])
    return ch, obs


def _check_job(orc, sp, res, out):
    ch, obs = _oracle(orc, sp)
    assert res.status == 0
    assert_obs_equal(out["obs"], obs)
    if out["spins"] is not None:
        np.testing.assert_array_equal(out["spins"], ch.spin)
    if out["labels"] is not None:
        np.testing.assert_array_equal(out["labels"], ch.label)
    assert res.threshold == ch.threshold
    assert res.sum_bond_sum == int(obs["bond_sum"].sum())
    assert res.sum_nclusters == int(obs["nclusters"].sum())


def _mixed_specs(n, rng):
    specs = []
    for r in range(n):
        L = int(rng.choice([2, 5, 16, 33, 64, 100, 128, 200, 256]))
        kind = r % 5
        sp = {"L": L, "sweeps": int(rng.integers(3, 40)), "seed": 100 + r}
        if kind == 3:
            sp["pcc"] = True
        elif kind == 4:
            sp["p"] = float(rng.choice([0.0, 0.3, 2 - 2 ** 0.5, 1.0]))
        else:
            sp["T"] = float(2.0 + 0.6 * (r % 32) / 31)
        specs.append(sp)
    return specs


def test_batch_equals_oracle(sw, orc):
    rng = np.random.default_rng(7)
    specs = _mixed_specs(40, rng)
    with sw.Server() as srv:
        ids = srv.submit(specs, want_spins=True, want_labels=True)
        srv.wait_all(120.0)
        for sp, i in zip(specs, ids):
            got = srv.poll(i)
            assert got is not None
            _check_job(orc, sp, *got)
        st = srv.stats()
        assert st["finished"] == len(specs) and st["pending"] == 0


def test_jobs_join_while_others_run(sw, orc):
    """Continuous batching: a second wave submitted while the first is on the
    GPU is admitted at a sweep boundary and finishes first; every job equals
    its solo run (the long ones) or the oracle (the short ones)."""
    long_specs = [{"L": 1024, "T": 2.269185, "sweeps": 2000, "seed": 1 + r} for r in range(2)]
    short_specs = [{"L": 64, "T": 3.0, "sweeps": 5, "seed": 50 + r} for r in range(4)]
    with sw.Server() as srv:
        long_ids = srv.submit(long_specs, want_spins=True)
        time.sleep(0.02)
        short_ids = srv.submit(short_specs, want_spins=True)
        done_short = {}
        deadline = time.time() + 120
        while len(done_short) < len(short_ids) and time.time() < deadline:
            for i in short_ids:
                if i not in done_short:
                    got = srv.poll(i)
                    if got is not None:
                        done_short[i] = got
            time.sleep(0.001)
        assert len(done_short) == len(short_ids)
        # the long jobs were still running when the short ones finished
        still = [srv.poll(i) for i in long_ids]
        assert any(g is None for g in still)
        srv.wait_all(300.0)
        long_got = [g if g is not None else srv.poll(i) for g, i in zip(still, long_ids)]
    for sp, (res, out) in zip(long_specs, long_got):
        assert res.status == 0
        with sw.Lattice(sp["L"], T=sp["T"], seed=sp["seed"]) as lat:
            lat.sweep(sp["sweeps"])
            assert_obs_equal(out["obs"], lat.observables())
            np.testing.assert_array_equal(out["spins"], lat.spins())
    for sp, i in zip(short_specs, short_ids):
        _check_job(orc, sp, *done_short[i])


def test_admission_by_device_memory(sw, orc):
    """With room for about one L=1024 lattice, three of them queue and run
    one after another; a job larger than the budget and a malformed job are
    refused at submission."""
    budget = 12 << 20   # one L=1024 lattice needs about 7.7 MiB
    specs = [{"L": 1024, "T": 2.5, "sweeps": 3, "seed": 9 + r, "tile_h": 128} for r in range(3)]
    with sw.Server(device_bytes=budget) as srv:
        ids = srv.submit(specs, want_spins=True)
        peak_active = 0
        deadline = time.time() + 120
        while srv.stats()["finished"] < 3 and time.time() < deadline:
            peak_active = max(peak_active, srv.stats()["active"])
            time.sleep(0.001)
        assert peak_active <= 1
        for sp, i in zip(specs, ids):
            _check_job(orc, sp, *srv.poll(i))
        with pytest.raises(sw.SwError) as e:
            srv.submit([{"L": 4096, "T": 2.0, "sweeps": 1, "seed": 1}])
        assert e.value.code == sw.SW_ERR_NOMEM
        with pytest.raises(sw.SwError) as e:
            srv.submit([{"L": 1, "T": 2.0, "sweeps": 1, "seed": 1}])
        assert e.value.code == sw.SW_ERR_ARG
        with pytest.raises(sw.SwError):
            srv.submit([{"L": 64, "T": 2.0, "sweeps": 0, "seed": 1}])
        with pytest.raises(sw.SwError):
            srv.poll(123456789)   # unknown id


def test_tile_height_does_not_change_results(sw, orc):
    sp = {"L": 300, "T": 2.269185, "sweeps": 12, "seed": 4}
    outs = []
    with sw.Server() as srv:
        for th in (32, 64, 96, 128):
            (i,) = srv.submit([dict(sp, tile_h=th)], want_spins=True, want_labels=True)
            srv.wait_all(60.0)
            res, out = srv.poll(i)
            assert res.tile_h == th
            outs.append(out)
    for o in outs[1:]:
        assert_obs_equal(o["obs"], outs[0]["obs"])
        np.testing.assert_array_equal(o["spins"], outs[0]["spins"])
        np.testing.assert_array_equal(o["labels"], outs[0]["labels"])
    assert sw.sw_autotune(300, 2.269185) in (32, 64, 96, 128)
    assert sw.sw_autotune(20, 3.0) == 32


def test_batch_manifest_replicas_equal_solo_runs(sw):
    """A slice of the uneven replica mix: batched results equal the same
    lattices run one at a time through sw_create/sw_sweep."""
    from paper_0808_2109_gb300 import workloads
    jobs = workloads.batch_manifest(n=24, sweeps=30)
    specs = [{"L": j.L, "T": j.T, "sweeps": j.sweeps, "seed": j.seed} for j in jobs]
    with sw.Server() as srv:
        ids = srv.submit(specs, want_spins=True)
        srv.wait_all(120.0)
        got = [srv.poll(i) for i in ids]
    for sp, (res, out) in zip(specs, got):
        with sw.Lattice(sp["L"], T=sp["T"], seed=sp["seed"]) as lat:
            lat.sweep(sp["sweeps"])
            assert_obs_equal(out["obs"], lat.observables())
            np.testing.assert_array_equal(out["spins"], lat.spins())
