#!/usr/bin/env python3
"""Writes the stored expected values of the configured runs, from the CPU
oracle alone.

Every value written here comes from ``oracle/`` (plain single-threaded C, one
function per step of Sec. I and Sec. III) run on the seeded workloads of
``paper_0808_2109_gb300/workloads.py``.  That module holds input generators
only and is loaded by file path, so the CUDA package (and its binding) is
never imported.  The GPU tests compare their runs with these files field by
field and hash by hash.

Runs (each: hot start, seed as listed, sweeps counted from 0):

  sw_L64_T2.269185_1000     plain SW, L=64, T=2.269185, 1000 sweeps
  sw_L4096_T2.0_200         plain SW, L=4096, T=2.0, 200 sweeps (giant cluster)
  sw_L4096_T2.269185_200    plain SW, L=4096, T=2.269185, 200 sweeps (critical)
  sw_L4096_T3.0_200         plain SW, L=4096, T=3.0, 200 sweeps (small clusters)
  sw_L16384_T2.269185_50    plain SW, L=16384, T=2.269185, 50 sweeps
  pcc_L2048_10000           PCC, L=2048, t0 = 2^31, 10000 sweeps
  batch_512x500             the 512-replica uneven mix, 500 sweeps each

Per run: ``<name>.npz`` holds the per-sweep observables (bond_sum, mag,
nclusters, nbonds, spans_x, spans_y, threshold; int64), and ``runs.json``
the SHA-256 of the final spins (uint8), labels (int32 little-endian) and the
last sweep's bond bytes (uint8).  The batch stores, per replica, the SHA-256
of its observables (the seven fields as an int64 little-endian array of shape
[sweeps, 7]), of its final spins and labels, and its last sweep's
observables, in ``batch_512x500.json``.

  python tests/golden/make_goldens.py [--jobs N] [name ...]

The PCC run is one chain of 10^4 sweeps and takes about 1.5 h on one core;
the whole set takes that long with 8 cores.
"""
from __future__ import annotations

import argparse
import hashlib
import importlib.util
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FIELDS = ("bond_sum", "mag", "nclusters", "nbonds", "spans_x", "spans_y", "threshold")
T_C = 2.269185

PLAIN_RUNS = {
    "sw_L64_T2.269185_1000": (64, T_C, 1000),
    "sw_L4096_T2.0_200": (4096, 2.0, 200),
    "sw_L4096_T2.269185_200": (4096, T_C, 200),
    "sw_L4096_T3.0_200": (4096, 3.0, 200),
    "sw_L16384_T2.269185_50": (16384, T_C, 50),
}
PCC_RUN = ("pcc_L2048_10000", 2048, 10000)
BATCH = "batch_512x500"
CITE = {"plain": "Sec. I steps 1-4 (bonds, clusters, flip, observables after the flip)",
        "pcc": "Sec. I and Sec. III (extension rule under periodic boundaries, threshold feedback)"}


def load_workloads():
    """The seeded input generators, without importing the CUDA package."""
    path = os.path.join(ROOT, "paper_0808_2109_gb300", "workloads.py")
    spec = importlib.util.spec_from_file_location("sw_workloads_inputs", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def sha256(a, dtype) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def obs_matrix(obs):
    """The seven per-sweep fields as int64 [sweeps, 7] (the hashed form)."""
    import numpy as np
    return np.stack([np.asarray(obs[f]).astype("<i8") for f in FIELDS], axis=1)


def _plain(name):
    import numpy as np
    import oracle
    L, T, n = PLAIN_RUNS[name]
    t0 = time.time()
    ch = oracle.sw_chain(L, 1.0, T, 1)
    obs = ch.run(n)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), **{f: obs[f].astype(np.int64) for f in FIELDS})
    return name, {"kind": "plain", "L": L, "T": T, "J": 1.0, "seed": 1, "sweeps": n,
                  "threshold": ch.threshold, "spins_sha256": sha256(ch.spin, "u1"),
                  "labels_sha256": sha256(ch.label, "<i4"), "bonds_sha256": sha256(ch.bond, "u1"),
                  "cite": CITE["plain"], "oracle_seconds": round(time.time() - t0, 1)}


def _pcc(name):
    import numpy as np
    import oracle
    _, L, n = PCC_RUN
    t0 = time.time()
    ch = oracle.pcc_chain(L, 1)
    obs = ch.run(n)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), **{f: obs[f].astype(np.int64) for f in FIELDS})
    return name, {"kind": "pcc", "L": L, "seed": 1, "sweeps": n, "threshold0": 1 << 31,
                  "threshold_final": ch.threshold, "spins_sha256": sha256(ch.spin, "u1"),
                  "labels_sha256": sha256(ch.label, "<i4"), "bonds_sha256": sha256(ch.bond, "u1"),
                  "cite": CITE["pcc"], "oracle_seconds": round(time.time() - t0, 1)}


def _replica(arg):
    r, L, T, seed, n = arg
    import oracle
    ch = oracle.sw_chain(L, 1.0, T, seed)
    obs = ch.run(n)
    last = {f: int(obs[f][-1]) for f in FIELDS}
    return r, {"replica": r, "L": L, "T": T, "seed": seed, "sweeps": n,
               "obs_sha256": sha256(obs_matrix(obs), "<i8"), "spins_sha256": sha256(ch.spin, "u1"),
               "labels_sha256": sha256(ch.label, "<i4"), "last_obs": last}


def _run(task):
    kind, name = task
    return _pcc(name) if kind == "pcc" else _plain(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("names", nargs="*")
    args = ap.parse_args()
    names = args.names or [PCC_RUN[0], "sw_L16384_T2.269185_50", *[k for k in PLAIN_RUNS if "16384" not in k], BATCH]
    import oracle
    oracle.build()
    wl = load_workloads()
    ctx = mp.get_context("spawn")
    index_path = os.path.join(HERE, "runs.json")
    index = json.load(open(index_path)) if os.path.exists(index_path) else {}
    tasks = [("pcc" if n == PCC_RUN[0] else "plain", n) for n in names if n != BATCH]
    batch_args = []
    if BATCH in names:
        batch_args = [(r, j.L, j.T, j.seed, j.sweeps) for r, j in enumerate(wl.batch_manifest())]
        batch_args.sort(key=lambda a: -a[1])   # largest lattices first
    import threading
    lock = threading.Lock()

    def save_index():
        with open(index_path, "w") as f:
            json.dump(dict(sorted(index.items())), f, indent=1)

    def done(res):   # runs in the pool's result thread: record each run as it ends
        name, rec = res
        with lock:
            index[name] = rec
            save_index()
        print(f"{name}: {rec['oracle_seconds']} s", flush=True)

    with ctx.Pool(args.jobs) as pool:
        pending = [pool.apply_async(_run, (t,), callback=done) for t in tasks]
        reps = pool.map_async(_replica, batch_args, chunksize=1) if batch_args else None
        if reps is not None:
            recs = sorted(reps.get(), key=lambda x: x[0])
            out = {"kind": "batch", "manifest": "512 replicas: L from {64,128,256,512,1024} with weights "
                                                "{.4,.25,.2,.1,.05} (numpy default_rng(20260)), T_r = "
                                                "2.0 + 0.6 (r mod 32)/31, seed 1000 + r, 500 sweeps, hot start",
                   "fields": list(FIELDS), "cite": CITE["plain"], "replicas": [x[1] for x in recs]}
            with open(os.path.join(HERE, BATCH + ".json"), "w") as f:
                json.dump(out, f, indent=0)
            print(f"{BATCH}: {len(recs)} replicas", flush=True)
        for p in pending:
            p.get()

if __name__ == "__main__":
    main()
