"""Pin the oracle's Philox4x32-10 to a library implementation.

triton ships Philox4x32 as ``tl.philox(seed, c0, c1, c2, c3, n_rounds)`` with
key = (seed mod 2^32, seed >> 32); its interpreter runs it on the CPU.  The
oracle must agree with it word for word on random counters and keys.
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def philox_kernel(seed_ptr, c_ptr, out_ptr, BLOCK: tl.constexpr):
    offs = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    seed = tl.load(seed_ptr + offs)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)

d = np.load(sys.argv[1])
seeds = torch.from_numpy(d["seed"].view(np.int64).copy())
ctr = torch.from_numpy(d["ctr"].view(np.int32).copy())
out = torch.zeros_like(ctr)
BLOCK = 256
philox_kernel[(seeds.numel() // BLOCK,)](seeds, ctr, out, BLOCK)
np.save(sys.argv[2], out.numpy().view(np.uint32))
"""


def _triton_philox(seeds: np.ndarray, ctr: np.ndarray) -> np.ndarray:
    pytest.importorskip("triton")
    with tempfile.TemporaryDirectory() as td:
        inp = os.path.join(td, "in.npz")
        outp = os.path.join(td, "out.npy")
        np.savez(inp, seed=seeds.astype(np.uint64), ctr=ctr.astype(np.uint32))
        script = os.path.join(td, "tp.py")
        with open(script, "w") as f:
            f.write(_TRITON_SCRIPT)
        env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
        subprocess.run([sys.executable, script, inp, outp], check=True, env=env, timeout=600)
        return np.load(outp).reshape(-1, 4)


def test_philox_matches_triton_library(orc):
    rng = np.random.default_rng(20260101)
    n = 4096
    seeds = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    # a few structured counters and keys: zeros, all-ones, the method's layouts
    ctr[0] = 0
    seeds[0] = 0
    ctr[1] = 0xFFFFFFFF
    seeds[1] = np.uint64(2**64 - 1)
    ctr[2] = [7, 3, 0, 1]   # (index word, sweep lo, sweep hi, BOND)
    seeds[2] = 1
    ctr[3] = [5, 3, 0, 2]   # SPIN stream
    seeds[3] = 1
    key = np.stack([(seeds & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                    (seeds >> np.uint64(32)).astype(np.uint32)], axis=1)
    ours = orc.philox(ctr, key)
    ref = _triton_philox(seeds, ctr)
    np.testing.assert_array_equal(ours, ref)


def test_philox_is_a_bijection_of_the_counter_and_mixes(orc):
    """Distinct counters give distinct blocks, and output bits are unbiased."""
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    out = orc.philox(ctr, [1, 0])
    # injective on this set (Philox is a bijection of the counter for a fixed key)
    assert np.unique(out.view(np.dtype((np.void, 16)))).size == n
    bits = np.unpackbits(out.view(np.uint8))
    frac = bits.mean()
    # 2^22 fair bits: standard deviation 2.4e-4
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(bits.size)
    # flipping one counter bit changes about half of the output bits
    ctr2 = ctr.copy()
    ctr2[:, 1] ^= 1
    out2 = orc.philox(ctr2, [1, 0])
    flips = np.unpackbits((out ^ out2).view(np.uint8)).mean()
    assert abs(flips - 0.5) < 0.01
