"""The C-ABI library loads and exports every function that include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof", "defined"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def cuda_lib():
    from paper_0808_2109_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sw_create", "sw_create_p", "sw_destroy", "sw_sweep", "sw_observables",
              "sw_get_spins", "sw_get_labels", "pcc_create", "pcc_step", "sw_sync", "sw_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(cuda_lib):
    missing = [n for n in sorted(_declared()) if not hasattr(cuda_lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_0808_2109_gb300 import swgpu
    missing = [n for n in sorted(_declared()) if n not in swgpu.SIGNATURES]
    assert not missing, missing


def test_host_only_calls(cuda_lib):
    """Calls that need no device: status names and the host threshold."""
    from paper_0808_2109_gb300 import swgpu
    assert swgpu.strerror(0) == "ok"
    assert swgpu.strerror(-1) == "invalid argument"
    import oracle
    for T in (2.0, 2.269185, 3.0, 1e-300):
        assert swgpu.sw_threshold(1.0, T) == oracle.threshold_T(1.0, T)
    with pytest.raises(swgpu.SwError):
        swgpu.sw_threshold(1.0, 0.0)
    with pytest.raises(swgpu.SwError):
        swgpu.sw_threshold(-1.0, 2.0)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_0808_2109_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "sw_oracle" not in src, f


def test_static_sweep_rejects_misaligned_or_overlapping_buffers(cuda_lib):
    """sw_sweep_static checks its caller-owned buffers on the host before it
    enqueues anything: the kernels store spins 8, labels 16 and observables
    8 bytes at a time, and the input spins are copied to the output first.
    The addresses below are never dereferenced (the call returns first), so
    this runs without a GPU."""
    from paper_0808_2109_gb300 import swgpu
    L, thr = 64, 1 << 31
    base = 1 << 20        # 256-byte aligned stand-in addresses
    spin_in, spin_out, labels, obs = base, base + 0x10000, base + 0x20000, base + 0x40000
    bad = [
        (spin_in, spin_out + 4, labels, obs),      # spins out not 8-byte aligned
        (spin_in, spin_out, labels + 8, obs),      # labels not 16-byte aligned
        (spin_in, spin_out, labels, obs + 4),      # observables not 8-byte aligned
        (spin_in, spin_in + 64, labels, obs),      # spin buffers overlap, not equal
        (spin_in + 64, spin_in, labels, obs),
    ]
    for args in bad:
        with pytest.raises(swgpu.SwError) as e:
            swgpu.sw_sweep_static(*args, L, thr, 1, 0)
        assert e.value.code == swgpu.SW_ERR_ARG, args
