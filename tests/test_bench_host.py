"""Host-side arithmetic behind the benchmark line (no GPU): the Philox block
count a tile launch draws, the roofline's DRAM traffic taken from the
committed ncu summary only while the kernel source matches it, and the
golden writer's inputs coming from the seeded generators alone."""
import hashlib
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _brute_blocks(L):
    """Philox blocks of one sweep's start, counted block by block: BOND blocks
    of every row (a row that starts on an odd site draws a block per site),
    SPIN blocks of every 128-wide tile row (one if the row's first site starts
    a block of 128, else two)."""
    tiles_x = (L + 127) // 128
    n = 0
    for y in range(L):
        for tx in range(tiles_x):
            g0 = y * L + 128 * tx
            n += 128 if (L % 2 and g0 % 2) else 64
            n += 1 if g0 % 128 == 0 else 2
    return n


@pytest.mark.parametrize("L", [64, 129, 300, 1024, 1025, 2048])
def test_philox_blocks_per_start(L):
    assert bench.philox_calls_per_start(L) == _brute_blocks(L)


def test_blocks_per_site_at_the_benchmark_lattice():
    L = 16384   # every tile row starts a block of 128 SPIN bits
    assert bench.philox_calls_per_start(L) / (L * L) == pytest.approx(0.5 + 1 / 128)


def test_profile_traffic_follows_the_kernel_source():
    """The committed summary names the source hash it was taken on; the bench
    reports its DRAM bytes only for that source."""
    txt = open(bench.PROFILE_FILE).read()
    m = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    assert m, "the summary states the source it was captured on"
    heights = [int(h) for h in re.findall(r"dram bytes per launch, tile height (\d+):", txt)]
    assert heights
    th = heights[0]
    assert bench.profile_traffic("0" * 64, th) is None
    got = bench.profile_traffic(m.group(1), th)
    assert isinstance(got, int) and got > 0
    assert bench.profile_traffic(m.group(1), 999) is None


def test_kernel_source_hash_is_the_two_files():
    h = hashlib.sha256()
    for f in ("sw_device.cuh", "sw_engine.cu"):
        h.update(open(os.path.join(ROOT, "paper_0808_2109_gb300", "csrc", f), "rb").read())
    assert bench.kernel_source_sha() == h.hexdigest()


def test_golden_writer_imports_no_cuda_binding():
    """The stored expected values are written from oracle/ alone: the writer
    loads the input generators by path and never imports the package that
    holds the CUDA binding."""
    src = open(os.path.join(ROOT, "tests", "golden", "make_goldens.py")).read()
    assert "import oracle" in src
    assert "paper_0808_2109_gb300 import" not in src and "import paper_0808_2109_gb300" not in src
    assert "swgpu" not in src


def test_potts_profile_traffic_follows_the_sources():
    """The Potts summary names the sources it was captured on (the tile
    kernels' file and the shared device header); its DRAM bytes are reported
    only for those sources and the named lattice."""
    txt = open(bench.POTTS_PROFILE_FILE).read()
    m = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    assert m, "the summary states the sources it was captured on"
    lat = re.findall(r"dram bytes per launch, (\d)D L=(\d+) q=(\d+):", txt)
    assert lat
    d, L, q = (int(v) for v in lat[0])
    assert bench.potts_profile_traffic("0" * 64, d, L, q) is None
    got = bench.potts_profile_traffic(m.group(1), d, L, q)
    assert isinstance(got, int) and got > 0
    assert bench.potts_profile_traffic(m.group(1), d, L + 1, q) is None


def test_potts_source_hash_is_the_two_files():
    h = hashlib.sha256()
    for f in ("sw_device.cuh", "sw_potts.cu"):
        h.update(open(os.path.join(ROOT, "paper_0808_2109_gb300", "csrc", f), "rb").read())
    assert bench.potts_source_sha() == h.hexdigest()
