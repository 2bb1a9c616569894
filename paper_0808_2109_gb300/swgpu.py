"""Python binding of the C ABI in ``include/swgpu.h`` (argument marshalling only).

Every step of a sweep runs in the CUDA library ``_build/libswgpu.so``; this
module only loads it with ctypes and converts arguments.  There is no CPU
fallback: if the library is missing or cannot be loaded, ``lib()`` raises.

The functions keep the C names (``sw_create``, ``sw_sweep``,
``sw_observables``, ``pcc_create``, ``pcc_step`` ...).  ``Lattice`` wraps a
context for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

SW_OK, SW_PENDING = 0, 1
SW_ERR_ARG, SW_ERR_NOMEM, SW_ERR_CUDA, SW_ERR_TIMEOUT, SW_ERR_STATE = -1, -2, -3, -4, -5

OBS_DTYPE = np.dtype(
    [
        ("bond_sum", "<i8"),
        ("mag", "<i8"),
        ("nclusters", "<i8"),
        ("nbonds", "<i8"),
        ("spans_x", "<i4"),
        ("spans_y", "<i4"),
        ("threshold", "<u8"),
        ("csize2", "<i8"),
    ]
)


class SwState(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("pcc", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("sweep", ctypes.c_uint64),
        ("threshold", ctypes.c_uint64),
        ("open", ctypes.c_int32),
        ("tile_h", ctypes.c_int32),
        ("dim", ctypes.c_int32),
        ("q", ctypes.c_int32),
    ]


class SwKernelStats(ctypes.Structure):
    _fields_ = [
        ("tile_launches", ctypes.c_int64),
        ("tile_ms", ctypes.c_double),
        ("merge_groups", ctypes.c_int64),
        ("merge_ms", ctypes.c_double),
        ("tile_sites", ctypes.c_int64),
        ("tile_height", ctypes.c_int32),
    ]


SW_JOB_SW, SW_JOB_SWP, SW_JOB_PCC = 0, 1, 2
SW_FLAG_TILE = {32: 1 << 8, 64: 1 << 9, 96: 1 << 11, 128: 1 << 10}
SW_FLAG_OPEN = 1 << 12
SW_FLAG_CSIZE = 1 << 13
SW_FLAG_WIND = 1 << 14


class SwJob(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("J", ctypes.c_double),
        ("T", ctypes.c_double),
        ("p", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("nsweeps", ctypes.c_int32),
        ("tile_h", ctypes.c_int32),
        ("obs_out", ctypes.c_void_p),
        ("spins_out", ctypes.c_void_p),
        ("labels_out", ctypes.c_void_p),
        ("flags", ctypes.c_uint32),
    ]


class SwResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("nsweeps", ctypes.c_int32),
        ("tile_h", ctypes.c_int32),
        ("threshold", ctypes.c_uint64),
        ("sum_bond_sum", ctypes.c_int64),
        ("sum_abs_mag", ctypes.c_int64),
        ("sum_nclusters", ctypes.c_int64),
        ("queued_s", ctypes.c_double),
        ("run_s", ctypes.c_double),
    ]


class SwServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("admitted", ctypes.c_int64),
        ("finished", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("active", ctypes.c_int64),
        ("site_updates", ctypes.c_int64),
        ("bytes_in_use", ctypes.c_size_t),
        ("bytes_budget", ctypes.c_size_t),
        ("launches", ctypes.c_int64),
    ]


class SwError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code in (SW_ERR_CUDA, SW_ERR_NOMEM):
            try:
                detail = lib().sw_last_error_detail().decode()
            except Exception:
                detail = ""
        super().__init__(f"{where}: {strerror(code)} ({code})" + (f": {detail}" if detail else ""))


_lock = threading.Lock()
_lib = None

# exported symbol -> (argtypes, restype)
_P = ctypes.c_void_p
_i32, _u32, _i64, _u64, _dbl = ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
SIGNATURES = {
    "sw_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "sw_last_error_detail": ([], ctypes.c_char_p),
    "sw_threshold": ([_dbl, _dbl, _P], ctypes.c_int),
    "sw_create": ([_P, _i32, _dbl, _dbl, _u64, _u32], ctypes.c_int),
    "sw_create_p": ([_P, _i32, _dbl, _u64, _u32], ctypes.c_int),
    "pcc_create": ([_P, _i32, _u64, _u32], ctypes.c_int),
    "sw_create_potts": ([_P, _i32, _i32, _i32, _dbl, _dbl, _u64, _u32], ctypes.c_int),
    "pcc_create_potts": ([_P, _i32, _i32, _i32, _u64, _u32], ctypes.c_int),
    "sw_checkpoint_bytes": ([_P, _P], ctypes.c_int),
    "sw_save": ([_P, _P, _u64], ctypes.c_int),
    "sw_load": ([_P, _P, _u64], ctypes.c_int),
    "sw_debug_fail_allocations": ([_i32, _i32], ctypes.c_int),
    "sw_destroy": ([_P], ctypes.c_int),
    "sw_set_stream": ([_P, _P], ctypes.c_int),
    "sw_sweep": ([_P, _i32], ctypes.c_int),
    "pcc_step": ([_P, _i32], ctypes.c_int),
    "sw_observables": ([_P, _P, _i32, _P], ctypes.c_int),
    "sw_get_spins": ([_P, _P], ctypes.c_int),
    "sw_set_spins": ([_P, _P], ctypes.c_int),
    "sw_get_labels": ([_P, _P], ctypes.c_int),
    "sw_get_bonds": ([_P, _P], ctypes.c_int),
    "sw_get_state": ([_P, _P], ctypes.c_int),
    "sw_sync": ([_P], ctypes.c_int),
    "sw_profile": ([_P, _i32], ctypes.c_int),
    "sw_profile_read": ([_P, _P], ctypes.c_int),
    "sw_server_create": ([_P, ctypes.c_size_t, _u32], ctypes.c_int),
    "sw_server_destroy": ([_P], ctypes.c_int),
    "sw_batch_submit": ([_P, _P, _i32, _P], ctypes.c_int),
    "sw_batch_poll": ([_P, _u64, _P], ctypes.c_int),
    "sw_batch_wait_all": ([_P, _dbl], ctypes.c_int),
    "sw_server_get_stats": ([_P, _P], ctypes.c_int),
    "sw_autotune": ([_i32, _dbl, _P], ctypes.c_int),
    "sw_sweep_static": ([_P, _P, _P, _P, _i32, _u64, _u64, _u64, _P], ctypes.c_int),
    "sw_bench_philox": ([_i64, _u64, _P, _P], ctypes.c_int),
    "sw_bench_l2": ([_P, _P, _i64, _i32, _P], ctypes.c_int),
}


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """Load the CUDA library (raises if it is not built or does not load)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().sw_strerror(code).decode()
    except Exception:  # the library itself failed to load
        return f"status {code}"


def _check(rc: int, where: str):
    if rc != SW_OK:
        raise SwError(rc, where)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------- C-named calls

def sw_threshold(J: float, T: float) -> int:
    out = ctypes.c_uint64()
    _check(lib().sw_threshold(J, T, ctypes.byref(out)), "sw_threshold")
    return int(out.value)


def sw_create(L: int, J: float, T: float, seed: int, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sw_create(ctypes.byref(h), L, J, T, seed, flags), "sw_create")
    return h


def sw_create_p(L: int, p: float, seed: int, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sw_create_p(ctypes.byref(h), L, p, seed, flags), "sw_create_p")
    return h


def pcc_create(L: int, seed: int, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().pcc_create(ctypes.byref(h), L, seed, flags), "pcc_create")
    return h


def sw_create_potts(dim: int, L: int, q: int, J: float, T: float, seed: int, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sw_create_potts(ctypes.byref(h), dim, L, q, J, T, seed, flags), "sw_create_potts")
    return h


def pcc_create_potts(dim: int, L: int, q: int, seed: int, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().pcc_create_potts(ctypes.byref(h), dim, L, q, seed, flags), "pcc_create_potts")
    return h


def sw_save(h) -> bytes:
    n = ctypes.c_uint64()
    _check(lib().sw_checkpoint_bytes(h, ctypes.byref(n)), "sw_checkpoint_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().sw_save(h, buf, n.value), "sw_save")
    return buf.raw


def sw_load(h, data: bytes) -> None:
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib().sw_load(h, buf, len(data)), "sw_load")


def sw_debug_fail_allocations(n: int, skip: int = 0) -> None:
    _check(lib().sw_debug_fail_allocations(skip, n), "sw_debug_fail_allocations")


def sw_destroy(h) -> None:
    _check(lib().sw_destroy(h), "sw_destroy")


def sw_set_stream(h, stream) -> None:
    """``stream``: a ``torch.cuda.Stream``, a raw cudaStream_t integer, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().sw_set_stream(h, ctypes.c_void_p(raw) if raw else None), "sw_set_stream")


def sw_sweep(h, nsweeps: int) -> None:
    _check(lib().sw_sweep(h, nsweeps), "sw_sweep")


def pcc_step(h, nsweeps: int) -> None:
    _check(lib().pcc_step(h, nsweeps), "pcc_step")


def sw_observables(h, max_entries: int) -> np.ndarray:
    out = np.zeros(max(int(max_entries), 0), dtype=OBS_DTYPE)
    n = ctypes.c_int32()
    _check(lib().sw_observables(h, _ptr(out) if out.size else None, out.size, ctypes.byref(n)),
           "sw_observables")
    return out[: n.value]


def sw_get_spins(h, L: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(L * L, dtype=np.uint8) if out is None else out
    _check(lib().sw_get_spins(h, _ptr(out)), "sw_get_spins")
    return out


def sw_set_spins(h, spins: np.ndarray) -> None:
    spins = np.ascontiguousarray(spins, dtype=np.uint8)
    _check(lib().sw_set_spins(h, _ptr(spins)), "sw_set_spins")


def sw_get_labels(h, L: int) -> np.ndarray:
    out = np.empty(L * L, dtype=np.int32)
    _check(lib().sw_get_labels(h, _ptr(out)), "sw_get_labels")
    return out


def sw_get_bonds(h, L: int) -> np.ndarray:
    out = np.empty(L * L, dtype=np.uint8)
    _check(lib().sw_get_bonds(h, _ptr(out)), "sw_get_bonds")
    return out


def sw_get_state(h) -> dict:
    st = SwState()
    _check(lib().sw_get_state(h, ctypes.byref(st)), "sw_get_state")
    return {"L": st.L, "pcc": bool(st.pcc), "seed": st.seed, "sweep": st.sweep,
            "threshold": st.threshold, "open": bool(st.open), "tile_h": st.tile_h,
            "dim": st.dim, "q": st.q}


def sw_sync(h) -> None:
    _check(lib().sw_sync(h), "sw_sync")


def sw_profile(h, enable: bool) -> None:
    _check(lib().sw_profile(h, 1 if enable else 0), "sw_profile")


def sw_profile_read(h) -> dict:
    st = SwKernelStats()
    _check(lib().sw_profile_read(h, ctypes.byref(st)), "sw_profile_read")
    return {f: getattr(st, f) for f, _ in SwKernelStats._fields_}


def sw_server_create(device_bytes: int = 0, flags: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sw_server_create(ctypes.byref(h), device_bytes, flags), "sw_server_create")
    return h


def sw_server_destroy(h) -> None:
    _check(lib().sw_server_destroy(h), "sw_server_destroy")


def sw_batch_submit(h, jobs) -> list[int]:
    arr = (SwJob * len(jobs))(*jobs)
    ids = (ctypes.c_uint64 * max(len(jobs), 1))()
    _check(lib().sw_batch_submit(h, arr, len(jobs), ids), "sw_batch_submit")
    return [int(ids[i]) for i in range(len(jobs))]


def sw_batch_poll(h, job_id: int):
    """None while the job waits or runs, else its SwResult."""
    res = SwResult()
    rc = lib().sw_batch_poll(h, job_id, ctypes.byref(res))
    if rc == SW_PENDING:
        return None
    _check(rc, "sw_batch_poll")
    return res


def sw_batch_wait_all(h, timeout_s: float = 0.0) -> None:
    _check(lib().sw_batch_wait_all(h, timeout_s), "sw_batch_wait_all")


def sw_server_get_stats(h) -> dict:
    st = SwServerStats()
    _check(lib().sw_server_get_stats(h, ctypes.byref(st)), "sw_server_get_stats")
    return {f: getattr(st, f) for f, _ in SwServerStats._fields_}


def sw_sweep_static(spin_in: int, spin_out: int, labels_out: int, obs_out: int, L: int,
                    threshold: int, seed: int, sweep: int, stream=None) -> None:
    """One sweep on caller-owned device buffers (raw device addresses, e.g.
    ``tensor.data_ptr()``) with no device allocation; see include/swgpu.h."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().sw_sweep_static(ctypes.c_void_p(spin_in), ctypes.c_void_p(spin_out),
                                 ctypes.c_void_p(labels_out), ctypes.c_void_p(obs_out), L,
                                 threshold, seed, sweep, ctypes.c_void_p(raw) if raw else None),
           "sw_sweep_static")


def sw_bench_philox(nblocks: int, seed: int, out_dev: int, stream=None) -> None:
    """Draw nblocks BOND-stream Philox blocks on the device, xored into the
    device word at out_dev (e.g. ``tensor.data_ptr()``); asynchronous on
    stream.  Times the integer ceiling of the bond step."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().sw_bench_philox(nblocks, seed, ctypes.c_void_p(out_dev), ctypes.c_void_p(raw) if raw else None),
           "sw_bench_philox")


def sw_bench_l2(src_dev: int, dst_dev: int, nbytes: int, reps: int, stream=None) -> None:
    """reps passes of dst = src ^ pass over nbytes of device memory, cached in
    L2 only; asynchronous on stream.  Times the L2 copy ceiling."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().sw_bench_l2(ctypes.c_void_p(src_dev), ctypes.c_void_p(dst_dev), nbytes, reps,
                             ctypes.c_void_p(raw) if raw else None), "sw_bench_l2")


def sw_autotune(L: int, T: float) -> int:
    out = ctypes.c_int32()
    _check(lib().sw_autotune(L, T, ctypes.byref(out)), "sw_autotune")
    return int(out.value)


# -------------------------------------------------------------- convenience

class Lattice:
    """One L x L lattice on the GPU (plain SW at J, T or p; or PCC), with
    periodic or (open=True) open boundaries; csize=True also reports
    sum |C|^2 per sweep (obs["csize2"]); wind=True reports the topological
    rule in spans_x/spans_y (and PCC feeds back on it)."""

    def __init__(self, L: int, *, J: float = 1.0, T: float | None = None, p: float | None = None,
                 seed: int = 1, pcc: bool = False, tile_h: int = 0, open: bool = False,
                 csize: bool = False, wind: bool = False):
        self.L = int(L)
        flags = (SW_FLAG_TILE.get(int(tile_h), 0) | (SW_FLAG_OPEN if open else 0)
                 | (SW_FLAG_CSIZE if csize else 0) | (SW_FLAG_WIND if wind else 0))
        if pcc:
            self.h = pcc_create(self.L, seed, flags)
        elif p is not None:
            self.h = sw_create_p(self.L, p, seed, flags)
        else:
            if T is None:
                raise ValueError("give T, p or pcc=True")
            self.h = sw_create(self.L, J, T, seed, flags)
        self.pcc = bool(pcc)

    def close(self):
        if getattr(self, "h", None):
            sw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, n: int):
        (pcc_step if self.pcc else sw_sweep)(self.h, n)

    def observables(self, max_entries: int = 1 << 20) -> np.ndarray:
        return sw_observables(self.h, max_entries)

    def spins(self) -> np.ndarray:
        return sw_get_spins(self.h, self.L)

    def set_spins(self, spins: np.ndarray):
        sw_set_spins(self.h, spins)

    def labels(self) -> np.ndarray:
        return sw_get_labels(self.h, self.L)

    def bonds(self) -> np.ndarray:
        return sw_get_bonds(self.h, self.L)

    def state(self) -> dict:
        return sw_get_state(self.h)

    def save(self) -> bytes:
        return sw_save(self.h)

    def load(self, data: bytes):
        sw_load(self.h, data)

    def set_stream(self, stream):
        sw_set_stream(self.h, stream)

    def sync(self):
        sw_sync(self.h)

    def profile(self, enable: bool = True):
        sw_profile(self.h, enable)

    def profile_read(self) -> dict:
        return sw_profile_read(self.h)


class PottsLattice:
    """A q-state Potts lattice on the d-dimensional torus (d = 2, 3), with
    open=True on the open d-dimensional box; pcc=True runs the PCC feedback
    (the threshold starts at 2^31; T is then ignored); wind=True reports the
    topological rule (and feeds it back under PCC)."""

    def __init__(self, dim: int, L: int, q: int, *, J: float = 1.0, T: float = 1.0, seed: int = 1,
                 csize: bool = False, open: bool = False, pcc: bool = False, wind: bool = False):
        self.dim, self.L, self.q = int(dim), int(L), int(q)
        self.N = self.L ** self.dim
        self.pcc = bool(pcc)
        flags = ((SW_FLAG_CSIZE if csize else 0) | (SW_FLAG_OPEN if open else 0)
                 | (SW_FLAG_WIND if wind else 0))
        if pcc:
            self.h = pcc_create_potts(self.dim, self.L, self.q, seed, flags)
        else:
            self.h = sw_create_potts(self.dim, self.L, self.q, J, T, seed, flags)

    def close(self):
        if getattr(self, "h", None):
            sw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, n: int):
        sw_sweep(self.h, n)

    def observables(self, max_entries: int = 1 << 20) -> np.ndarray:
        return sw_observables(self.h, max_entries)

    def _get(self, fn, dtype):
        out = np.empty(self.N, dtype=dtype)
        _check(getattr(lib(), fn)(self.h, _ptr(out)), fn)
        return out

    def sync(self):
        sw_sync(self.h)

    def profile(self, enable: bool = True):
        sw_profile(self.h, enable)

    def profile_read(self) -> dict:
        return sw_profile_read(self.h)

    def spins(self) -> np.ndarray:
        return self._get("sw_get_spins", np.uint8)

    def labels(self) -> np.ndarray:
        return self._get("sw_get_labels", np.int32)

    def bonds(self) -> np.ndarray:
        return self._get("sw_get_bonds", np.uint8)

    def set_spins(self, spins: np.ndarray):
        sw_set_spins(self.h, spins)

    def state(self) -> dict:
        return sw_get_state(self.h)

    def save(self) -> bytes:
        return sw_save(self.h)

    def load(self, data: bytes):
        sw_load(self.h, data)

    def set_stream(self, stream):
        sw_set_stream(self.h, stream)

    def sync(self):
        sw_sync(self.h)


class Server:
    """A batch/serve server; jobs keep their output arrays alive until polled."""

    def __init__(self, device_bytes: int = 0):
        self.h = sw_server_create(device_bytes)
        self._outputs = {}

    def close(self):
        if getattr(self, "h", None):
            sw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, specs, want_obs=True, want_spins=False, want_labels=False) -> list[int]:
        """specs: dicts with L, sweeps, seed and T (plain), p, or pcc=True;
        optional tile_h, open=True (open boundaries), csize=True and wind=True."""
        jobs, outs = [], []
        for sp in specs:
            L, n = int(sp["L"]), int(sp["sweeps"])
            o = {"obs": np.zeros(n, dtype=OBS_DTYPE) if want_obs else None,
                 "spins": np.zeros(L * L, dtype=np.uint8) if want_spins else None,
                 "labels": np.zeros(L * L, dtype=np.int32) if want_labels else None}
            j = SwJob()
            j.L, j.nsweeps, j.seed = L, n, int(sp["seed"])
            j.J = float(sp.get("J", 1.0))
            if sp.get("pcc"):
                j.kind = SW_JOB_PCC
            elif sp.get("p") is not None:
                j.kind, j.p = SW_JOB_SWP, float(sp["p"])
            else:
                j.kind, j.T = SW_JOB_SW, float(sp["T"])
            j.tile_h = int(sp.get("tile_h", 0))
            j.flags = ((SW_FLAG_OPEN if sp.get("open") else 0) | (SW_FLAG_CSIZE if sp.get("csize") else 0)
                       | (SW_FLAG_WIND if sp.get("wind") else 0))
            j.obs_out = o["obs"].ctypes.data if want_obs else None
            j.spins_out = o["spins"].ctypes.data if want_spins else None
            j.labels_out = o["labels"].ctypes.data if want_labels else None
            jobs.append(j)
            outs.append(o)
        ids = sw_batch_submit(self.h, jobs)
        for i, o in zip(ids, outs):
            self._outputs[i] = o
        return ids

    def poll(self, job_id: int):
        """None while pending, else (SwResult, outputs dict)."""
        res = sw_batch_poll(self.h, job_id)
        if res is None:
            return None
        return res, self._outputs.pop(job_id)

    def wait_all(self, timeout_s: float = 0.0):
        sw_batch_wait_all(self.h, timeout_s)

    def stats(self) -> dict:
        return sw_server_get_stats(self.h)
