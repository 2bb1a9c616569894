"""sw_sweep_static: one sweep with no device allocation (for callers that
may not call cudaMalloc, e.g. under a framework or memory pool that owns all
device memory, or in a loop where cudaMalloc's implicit synchronisation is not
acceptable), checked against sw_sweep.

Two calls in a row -- the second in place on the first one's output -- must
give exactly the spins, labels and observables of two sweeps of a lattice
made with sw_create_p and run with sw_sweep.  This file sorts last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_0808_2109_gb300 import swgpu
    swgpu.lib()
    return swgpu, torch


@pytest.mark.parametrize("L,T,seed", [(300, 2.269185, 5), (1024, 2.0, 7), (33, 3.0, 2)])
def test_static_sweep_equals_sw_sweep_twice(env, L, T, seed):
    sw, torch = env
    thr = sw.sw_threshold(1.0, T)
    p = thr / 2.0 ** 32   # exactly representable: gives the same threshold back
    with sw.Lattice(L, p=p, seed=seed) as ref:
        spins0 = ref.spins()
        dev = torch.device("cuda", torch.cuda.current_device())
        s_in = torch.from_numpy(spins0).to(dev)
        s_out = torch.empty_like(s_in)
        labels = torch.empty(L * L, dtype=torch.int32, device=dev)
        obs = torch.full((sw.OBS_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device=dev)   # zeroed by the call
        stream = torch.cuda.current_stream()
        for k in range(2):
            src = s_in if k == 0 else s_out   # second call in place
            sw.sw_sweep_static(src.data_ptr(), s_out.data_ptr(), labels.data_ptr(), obs.data_ptr(),
                               L, thr, seed, k, stream)
            torch.cuda.synchronize()
            ref.sweep(1)
            want = ref.observables()
            got = np.frombuffer(obs.cpu().numpy().tobytes(), dtype=sw.OBS_DTYPE)
            for f in ("bond_sum", "mag", "nclusters", "nbonds", "threshold"):
                assert int(got[f][0]) == int(want[f][0]), (k, f)
            np.testing.assert_array_equal(s_out.cpu().numpy(), ref.spins())
            np.testing.assert_array_equal(labels.cpu().numpy(), ref.labels())


def test_static_sweep_rejects_sizes_beyond_its_array(env):
    sw, torch = env
    big = 1025   # above SW_STATIC_MAX_L
    with pytest.raises(sw.SwError) as e:
        sw.sw_sweep_static(1, 1, 1, 1, big, 1 << 31, 1, 0)
    assert e.value.code == sw.SW_ERR_ARG
    with pytest.raises(sw.SwError):
        sw.sw_sweep_static(1, 1, 1, 1, 64, (1 << 32) + 1, 1, 0)
    with pytest.raises(sw.SwError):
        sw.sw_sweep_static(0, 1, 1, 1, 64, 1 << 31, 1, 0)
