"""The measurement probes behind the benchmark's two ceilings do the work
they are timed for: the Philox probe draws exactly the BOND-stream blocks
(checked against the oracle's Philox), the L2 probe copies every word."""
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


@pytest.mark.parametrize("nblocks", [1, 1000, 100003])
def test_philox_rate_probe_draws_the_bond_stream(sw, orc, nblocks):
    import torch
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    seed = 0x123456789
    sw.sw_bench_philox(nblocks, seed, out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    ctr = np.zeros((nblocks, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(nblocks, dtype=np.uint32)
    ctr[:, 3] = orc.STREAM_BOND
    w = orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    assert int(out.cpu().numpy().view(np.uint32)[0]) == int(np.bitwise_xor.reduce(w.ravel()))


@pytest.mark.parametrize("nbytes,reps", [(16, 1), (4096, 3), (1 << 22, 5)])
def test_l2_probe_copies_every_word(sw, nbytes, reps):
    import torch
    g = torch.Generator().manual_seed(nbytes)
    src = torch.randint(0, 1 << 31, (nbytes // 4,), generator=g, dtype=torch.int32).cuda()
    dst = torch.zeros_like(src)
    sw.sw_bench_l2(src.data_ptr(), dst.data_ptr(), nbytes, reps, torch.cuda.current_stream())
    torch.cuda.synchronize()
    want = src.cpu().numpy().view(np.uint32).reshape(-1, 4).copy()
    want[:, 0] ^= np.uint32(reps - 1)
    np.testing.assert_array_equal(dst.cpu().numpy().view(np.uint32).reshape(-1, 4), want)
    with pytest.raises(sw.SwError):
        sw.sw_bench_l2(src.data_ptr(), src.data_ptr() + 16, 32, 1)   # overlapping
