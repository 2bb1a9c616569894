"""CPU oracle of the Swendsen-Wang / PCC hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_0808_2109_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``sw_oracle.c`` (plain single-threaded C, one
function per step of the method, each citing the paper's section); this module
only builds it with gcc and marshals numpy arrays through ctypes.

Pins (what ties this oracle to something other than itself) are in
``tests/test_oracle_*.py``: Philox against triton's library routine, the
threshold against the exact identity 1 - exp(-2/T_c) = 2 - sqrt(2), labels
against scipy's connected components, the exact 3x3 Swendsen-Wang transition
matrix, brute-force 4x4 enumeration, Kaufman's finite-L energy at L=64, and
the paper's worked example of the range operator (Sec. III).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libswo.so")
_SRC = os.path.join(_HERE, "sw_oracle.c")
_HDR = os.path.join(_HERE, "sw_oracle.h")

STREAM_INIT, STREAM_BOND, STREAM_SPIN = 0, 1, 2

_lock = threading.Lock()
_lib = None


class Obs(ctypes.Structure):
    """Per-sweep observables (mirrors ``swo_obs``)."""

    _fields_ = [
        ("bond_sum", ctypes.c_int64),
        ("mag", ctypes.c_int64),
        ("nclusters", ctypes.c_int64),
        ("nbonds", ctypes.c_int64),
        ("spans_x", ctypes.c_int32),
        ("spans_y", ctypes.c_int32),
        ("threshold", ctypes.c_uint64),
        ("csize2", ctypes.c_int64),
    ]


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
assert OBS_DTYPE.itemsize == ctypes.sizeof(Obs) == 56


def build(force: bool = False) -> str:
    """Compile ``sw_oracle.c`` into ``_build/libswo.so`` (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest_src:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.swo_philox_batch.argtypes = [i64, P, P, P]
            L.swo_philox_batch.restype = None
            L.swo_threshold_T.argtypes = [dbl, dbl]
            L.swo_threshold_T.restype = u64
            L.swo_threshold_p.argtypes = [dbl]
            L.swo_threshold_p.restype = u64
            L.swo_hot_start.argtypes = [i32, u64, P]
            L.swo_hot_start.restype = None
            L.swo_bonds.argtypes = [i32, u64, u64, u64, P, P, i32]
            L.swo_bonds.restype = i64
            L.swo_label.argtypes = [i32, P, P]
            L.swo_label.restype = i64
            L.swo_count_clusters_batch.argtypes = [i32, i64, P, P]
            L.swo_count_clusters_batch.restype = None
            L.swo_assign.argtypes = [i32, u64, u64, P, P]
            L.swo_assign.restype = None
            L.swo_measure.argtypes = [i32, P, i32, P, P]
            L.swo_measure.restype = None
            L.swo_spans.argtypes = [i32, P, P, P]
            L.swo_spans.restype = ctypes.c_int
            L.swo_spans_open.argtypes = [i32, P, P, P]
            L.swo_spans_open.restype = ctypes.c_int
            L.swo_windings.argtypes = [i32, P, P, P]
            L.swo_windings.restype = ctypes.c_int
            L.swo_threshold_potts.argtypes = [ctypes.c_double, ctypes.c_double]
            L.swo_threshold_potts.restype = u64
            L.swo_potts_hot_start.argtypes = [i32, i32, i32, u64, P]
            L.swo_potts_hot_start.restype = None
            L.swo_potts_bonds.argtypes = [i32, i32, u64, u64, u64, P, P]
            L.swo_potts_bonds.restype = i64
            L.swo_label_nd.argtypes = [i32, i32, P, P]
            L.swo_label_nd.restype = i64
            L.swo_count_clusters_nd.argtypes = [i32, i32, i64, P, P]
            L.swo_count_clusters_nd.restype = None
            L.swo_potts_assign.argtypes = [i32, i32, i32, u64, u64, P, P]
            L.swo_potts_assign.restype = None
            L.swo_potts_measure.argtypes = [i32, i32, i32, P, P, P]
            L.swo_potts_measure.restype = None
            L.swo_potts_run.argtypes = [i32, i32, i32, u64, u64, i32, i32, u64, P, P, P, P]
            L.swo_potts_run.restype = ctypes.c_int
            L.swo_potts_bonds_open.argtypes = [i32, i32, u64, u64, u64, P, P, i32]
            L.swo_potts_bonds_open.restype = i64
            L.swo_potts_measure_open.argtypes = [i32, i32, i32, P, i32, P, P]
            L.swo_potts_measure_open.restype = None
            L.swo_spans_nd.argtypes = [i32, i32, P, P]
            L.swo_spans_nd.restype = ctypes.c_int
            L.swo_potts_run_pcc.argtypes = [i32, i32, i32, u64, u64, i32, i32, i32, i32, P, P, P, P, P]
            L.swo_potts_run_pcc.restype = ctypes.c_int
            L.swo_potts_run_rules.argtypes = [i32, i32, i32, u64, u64, i32, i32, i32, i32, i32, P, P, P, P, P]
            L.swo_potts_run_rules.restype = ctypes.c_int
            L.swo_windings_nd.argtypes = [i32, i32, P, P]
            L.swo_windings_nd.restype = ctypes.c_int
            L.swo_csize2.argtypes = [i32, P]
            L.swo_csize2.restype = i64
            L.swo_pcc_delta.argtypes = [u64]
            L.swo_pcc_delta.restype = u64
            L.swo_pcc_update.argtypes = [u64, u64, i32]
            L.swo_pcc_update.restype = u64
            L.swo_run.argtypes = [i32, u64, u64, i32, i32, i32, i32, i32, P, P, P, P, P]
            L.swo_run.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------- API

def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of blocks ``ctr[..., 4]`` (uint32) under ``key[..., 2]``."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32),
                                               (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().swo_philox_batch(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
    return out


def threshold_T(J: float, T: float) -> int:
    return int(lib().swo_threshold_T(float(J), float(T)))


def threshold_p(p: float) -> int:
    return int(lib().swo_threshold_p(float(p)))


def hot_start(L: int, seed: int) -> np.ndarray:
    spin = np.empty(L * L, dtype=np.uint8)
    lib().swo_hot_start(L, seed, _ptr(spin))
    return spin


def bonds(L: int, seed: int, sweep: int, thr: int, spin: np.ndarray, open: bool = False):
    spin = np.ascontiguousarray(spin, dtype=np.uint8)
    bond = np.empty(L * L, dtype=np.uint8)
    nb = lib().swo_bonds(L, seed, sweep, thr, _ptr(spin), _ptr(bond), 1 if open else 0)
    return bond, int(nb)


def label(L: int, bond: np.ndarray):
    bond = np.ascontiguousarray(bond, dtype=np.uint8)
    lab = np.empty(L * L, dtype=np.int32)
    nc = lib().swo_label(L, _ptr(bond), _ptr(lab))
    return lab, int(nc)


def count_clusters_batch(L: int, bond_sets: np.ndarray) -> np.ndarray:
    bond_sets = np.ascontiguousarray(bond_sets, dtype=np.uint8).reshape(-1, L * L)
    counts = np.empty(bond_sets.shape[0], dtype=np.int64)
    lib().swo_count_clusters_batch(L, bond_sets.shape[0], _ptr(bond_sets), _ptr(counts))
    return counts


def assign(L: int, seed: int, sweep: int, lab: np.ndarray) -> np.ndarray:
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    spin = np.empty(L * L, dtype=np.uint8)
    lib().swo_assign(L, seed, sweep, _ptr(lab), _ptr(spin))
    return spin


def measure(L: int, spin: np.ndarray, open: bool = False):
    spin = np.ascontiguousarray(spin, dtype=np.uint8)
    bs = np.zeros(1, dtype=np.int64)
    m = np.zeros(1, dtype=np.int64)
    lib().swo_measure(L, _ptr(spin), 1 if open else 0, _ptr(bs), _ptr(m))
    return int(bs[0]), int(m[0])


def spans(L: int, lab: np.ndarray):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    sx = np.zeros(1, dtype=np.int32)
    sy = np.zeros(1, dtype=np.int32)
    if lib().swo_spans(L, _ptr(lab), _ptr(sx), _ptr(sy)) != 0:
        raise MemoryError("swo_spans")
    return int(sx[0]), int(sy[0])


def csize2(L: int, lab: np.ndarray) -> int:
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    v = int(lib().swo_csize2(L, _ptr(lab)))
    if v < 0:
        raise MemoryError("swo_csize2")
    return v


def windings(L: int, bond: np.ndarray):
    bond = np.ascontiguousarray(bond, dtype=np.uint8)
    wx = np.zeros(1, dtype=np.int32)
    wy = np.zeros(1, dtype=np.int32)
    if lib().swo_windings(L, _ptr(bond), _ptr(wx), _ptr(wy)) != 0:
        raise MemoryError("swo_windings")
    return int(wx[0]), int(wy[0])


def spans_open(L: int, lab: np.ndarray):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    sx = np.zeros(1, dtype=np.int32)
    sy = np.zeros(1, dtype=np.int32)
    if lib().swo_spans_open(L, _ptr(lab), _ptr(sx), _ptr(sy)) != 0:
        raise MemoryError("swo_spans_open")
    return int(sx[0]), int(sy[0])


def pcc_delta(sweep: int) -> int:
    return int(lib().swo_pcc_delta(sweep))


def pcc_update(thr: int, sweep: int, flag: bool) -> int:
    return int(lib().swo_pcc_update(thr, sweep, 1 if flag else 0))


class Chain:
    """A lattice state advanced by the oracle: (spins, seed, sweep, threshold);
    open=True gives open boundaries, csize=True fills obs["csize2"], wind=True
    reports (and, for PCC, feeds back on) the topological rule in spans_x/y."""

    def __init__(self, L: int, seed: int, thr: int, pcc: bool = False,
                 spin: np.ndarray | None = None, sweep: int = 0, open: bool = False,
                 csize: bool = False, wind: bool = False):
        if L < 2:
            raise ValueError("L must be >= 2")
        self.L, self.seed, self.pcc, self.open = int(L), int(seed), bool(pcc), bool(open)
        self.csize, self.wind = bool(csize), bool(wind)
        self.thr = np.array([thr], dtype=np.uint64)
        self.sweep = int(sweep)
        self.spin = hot_start(L, seed) if spin is None else np.array(spin, dtype=np.uint8).ravel()
        self.label = np.arange(L * L, dtype=np.int32)
        self.bond = np.zeros(L * L, dtype=np.uint8)

    @property
    def threshold(self) -> int:
        return int(self.thr[0])

    def run(self, nsweeps: int) -> np.ndarray:
        obs = np.zeros(nsweeps, dtype=OBS_DTYPE)
        if nsweeps <= 0:
            return obs
        rc = lib().swo_run(self.L, self.seed, self.sweep, nsweeps, 1 if self.pcc else 0,
                           1 if self.open else 0, 1 if self.csize else 0, 1 if self.wind else 0,
                           _ptr(self.thr), _ptr(self.spin), _ptr(self.label), _ptr(self.bond),
                           _ptr(obs))
        if rc != 0:
            raise MemoryError("swo_run")
        self.sweep += nsweeps
        return obs


def sw_chain(L: int, J: float, T: float, seed: int, open: bool = False, csize: bool = False,
             wind: bool = False) -> Chain:
    return Chain(L, seed, threshold_T(J, T), open=open, csize=csize, wind=wind)


def sw_chain_p(L: int, p: float, seed: int, open: bool = False, csize: bool = False,
               wind: bool = False) -> Chain:
    return Chain(L, seed, threshold_p(p), open=open, csize=csize, wind=wind)


def pcc_chain(L: int, seed: int, open: bool = False, csize: bool = False, wind: bool = False) -> Chain:
    return Chain(L, seed, 1 << 31, pcc=True, open=open, csize=csize, wind=wind)


def energy_per_site(obs: np.ndarray, L: int, J: float = 1.0) -> np.ndarray:
    """E/N = -J * bond_sum / N per sweep, in float64."""
    return -J * obs["bond_sum"].astype(np.float64) / float(L * L)


# ------------------------------------------------- q-state Potts, d = 2 or 3

def threshold_potts(J: float, T: float) -> int:
    return int(lib().swo_threshold_potts(float(J), float(T)))


def potts_hot_start(dim: int, L: int, q: int, seed: int) -> np.ndarray:
    spin = np.empty(L ** dim, dtype=np.uint8)
    lib().swo_potts_hot_start(dim, L, q, seed, _ptr(spin))
    return spin


def potts_bonds(dim: int, L: int, seed: int, sweep: int, thr: int, spin: np.ndarray, open: bool = False):
    spin = np.ascontiguousarray(spin, dtype=np.uint8)
    bond = np.empty(L ** dim, dtype=np.uint8)
    nb = lib().swo_potts_bonds_open(dim, L, seed, sweep, thr, _ptr(spin), _ptr(bond), 1 if open else 0)
    return bond, int(nb)


def spans_nd(dim: int, L: int, lab: np.ndarray):
    """Extension rule per axis: (spans x, spans y[, spans z])."""
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    out = np.zeros(3, dtype=np.int32)
    if lib().swo_spans_nd(dim, L, _ptr(lab), _ptr(out)) != 0:
        raise MemoryError("swo_spans_nd")
    return tuple(int(v) for v in out[:dim])


def windings_nd(dim: int, L: int, bond: np.ndarray):
    """Topological rule per axis: (winds x, winds y[, winds z])."""
    bond = np.ascontiguousarray(bond, dtype=np.uint8)
    out = np.zeros(3, dtype=np.int32)
    if lib().swo_windings_nd(dim, L, _ptr(bond), _ptr(out)) != 0:
        raise MemoryError("swo_windings_nd")
    return tuple(int(v) for v in out[:dim])


def label_nd(dim: int, L: int, bond: np.ndarray):
    bond = np.ascontiguousarray(bond, dtype=np.uint8)
    lab = np.empty(L ** dim, dtype=np.int32)
    nc = lib().swo_label_nd(dim, L, _ptr(bond), _ptr(lab))
    return lab, int(nc)


def count_clusters_nd(dim: int, L: int, bond_sets: np.ndarray) -> np.ndarray:
    bond_sets = np.ascontiguousarray(bond_sets, dtype=np.uint8).reshape(-1, L ** dim)
    counts = np.empty(bond_sets.shape[0], dtype=np.int64)
    lib().swo_count_clusters_nd(dim, L, bond_sets.shape[0], _ptr(bond_sets), _ptr(counts))
    return counts


def potts_assign(dim: int, L: int, q: int, seed: int, sweep: int, lab: np.ndarray) -> np.ndarray:
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    spin = np.empty(L ** dim, dtype=np.uint8)
    lib().swo_potts_assign(dim, L, q, seed, sweep, _ptr(lab), _ptr(spin))
    return spin


def potts_measure(dim: int, L: int, q: int, spin: np.ndarray, open: bool = False):
    spin = np.ascontiguousarray(spin, dtype=np.uint8)
    bs = np.zeros(1, dtype=np.int64)
    m = np.zeros(1, dtype=np.int64)
    lib().swo_potts_measure_open(dim, L, q, _ptr(spin), 1 if open else 0, _ptr(bs), _ptr(m))
    return int(bs[0]), int(m[0])


class PottsChain:
    """A q-state Potts lattice (d = 2 or 3) advanced by the oracle; open=True
    gives open boundaries, pcc=True the PCC feedback (the threshold starts at
    2^31 and J, T are ignored), wind=True the topological rule for the span
    flags (reported every sweep, and the feedback's criterion under PCC)."""

    def __init__(self, dim: int, L: int, q: int, J: float, T: float, seed: int, csize: bool = False,
                 open: bool = False, pcc: bool = False, wind: bool = False):
        if dim not in (2, 3) or L < 2 or not 2 <= q <= 256:
            raise ValueError("dim in {2, 3}, L >= 2, 2 <= q <= 256")
        self.dim, self.L, self.q, self.seed, self.csize = int(dim), int(L), int(q), int(seed), bool(csize)
        self.open, self.pcc, self.wind = bool(open), bool(pcc), bool(wind)
        self.threshold = (1 << 31) if pcc else threshold_potts(J, T)
        self.sweep = 0
        self.spin = potts_hot_start(dim, L, q, seed)
        self.label = np.arange(L ** dim, dtype=np.int32)
        self.bond = np.zeros(L ** dim, dtype=np.uint8)

    def run(self, nsweeps: int) -> np.ndarray:
        obs = np.zeros(nsweeps, dtype=OBS_DTYPE)
        if nsweeps <= 0:
            return obs
        thr = np.array([self.threshold], dtype=np.uint64)
        rc = lib().swo_potts_run_rules(self.dim, self.L, self.q, self.seed, self.sweep, nsweeps,
                                       1 if self.pcc else 0, 1 if self.open else 0, 1 if self.csize else 0,
                                       1 if self.wind else 0, _ptr(thr), _ptr(self.spin), _ptr(self.label),
                                       _ptr(self.bond), _ptr(obs))
        if rc != 0:
            raise MemoryError("swo_potts_run_rules")
        self.threshold = int(thr[0])
        self.sweep += nsweeps
        return obs
