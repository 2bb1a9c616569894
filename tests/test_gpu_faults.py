"""Failure handling, injected on the host (no GPU fault): device allocations
that fail give SW_ERR_NOMEM from sw_create and a SW_ERR_NOMEM job result from
a server, with nothing left half-made; a server destroyed while its jobs run
(the client going away) stops cleanly; the library keeps working after."""
import time

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


def test_every_allocation_of_create_can_fail(sw):
    failed = 0
    try:
        for k in range(40):
            sw.sw_debug_fail_allocations(1, skip=k)   # the (k+1)-th allocation fails
            try:
                lat = sw.Lattice(200, T=2.3, seed=1, tile_h=64, csize=True, wind=True)
            except sw.SwError as e:
                assert e.code == sw.SW_ERR_NOMEM
                failed += 1
                continue
            lat.close()                               # past the last allocation
            break
    finally:
        sw.sw_debug_fail_allocations(0)
    assert failed >= 10
    with sw.Lattice(200, T=2.3, seed=1) as lat:   # nothing was left behind
        lat.sweep(3)
        assert len(lat.observables()) == 3


def test_potts_create_reports_nomem(sw):
    sw.sw_debug_fail_allocations(1)
    try:
        with pytest.raises(sw.SwError) as e:
            sw.PottsLattice(3, 16, 3, T=1.0)
        assert e.value.code == sw.SW_ERR_NOMEM
    finally:
        sw.sw_debug_fail_allocations(0)


def test_server_job_allocation_failure(sw):
    with sw.Server() as srv:
        sw.sw_debug_fail_allocations(1)
        try:
            (bad,) = srv.submit([{"L": 64, "T": 2.3, "sweeps": 3, "seed": 1, "tile_h": 64}])
            srv.wait_all(60.0)
        finally:
            sw.sw_debug_fail_allocations(0)
        res, _ = srv.poll(bad)
        assert res.status == sw.SW_ERR_NOMEM
        (good,) = srv.submit([{"L": 64, "T": 2.3, "sweeps": 3, "seed": 1, "tile_h": 64}])
        srv.wait_all(60.0)
        res, out = srv.poll(good)
        assert res.status == 0 and len(out["obs"]) == 3
        st = srv.stats()
        assert st["bytes_in_use"] == 0


def test_server_destroyed_while_jobs_run(sw):
    import torch
    free0, _ = torch.cuda.mem_get_info()
    srv = sw.Server()
    srv.submit([{"L": 1024, "T": 2.269185, "sweeps": 100000, "seed": r, "tile_h": 96} for r in range(4)])
    time.sleep(0.2)
    t0 = time.time()
    srv.close()                     # the client goes away mid-run
    assert time.time() - t0 < 30
    with sw.Server() as again:
        (i,) = again.submit([{"L": 32, "T": 2.0, "sweeps": 2, "seed": 3, "tile_h": 32}])
        again.wait_all(60.0)
        assert again.poll(i)[0].status == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 > free0 - (256 << 20)   # the dropped jobs' memory came back (pool slack aside)
