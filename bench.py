#!/usr/bin/env python3
"""Benchmark of the Swendsen-Wang hot path on GB300: prints one JSON line.

Workload: plain SW on the 2D periodic Ising lattice, L = 16384 (268M sites),
J = 1, T = 2.269185 (critical), hot start; one step = 50 sweeps, the
configured run length of that lattice.  Metric: site updates per ns over the
whole job (all ranks), with the lattice resident on the device, beside the
achieved HBM GB/s of the dominant kernel.  The same line carries the batched
512-replica mix (against the same replicas run one at a time) and the served
Poisson trace (p50/p99 latency beside throughput).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
  python bench.py --workload configs   # every configured run, oracle timed beside it

N > 1 runs under torchrun, one independent lattice per GPU (replicas: the
single-lattice path has no exchange step), timed between barriers, max over
ranks.  ``--impl reference`` times the CPU oracle (the only reference that
exists: the paper publishes no code) on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SW site updates/ns at T_c (L=16384)"
L2_BYTES = 129 << 20     # GB300 L2
UNIT = "site-updates/ns"
ALG_BYTES_PER_SITE = 10            # old spin in, label out, label in, new spin out
PROFILE_FILE = os.path.join(ROOT, "profiles", "k_tile_L16384_Tc.md")
LAUNCHES_PER_SWEEP = 4             # tile kernel, merge union, pointer jumping, resolve


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-solo comparison")
    ap.add_argument("--workload", default="plain", choices=["plain", "serve", "potts", "configs", "batch64"])
    ap.add_argument("--no-serve", action="store_true", help="skip the served trace")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="--workload serve: arrivals per second")
    ap.add_argument("--lattice", type=int, default=0, help="profiling only: another L")
    ap.add_argument("--sweeps", type=int, default=0, help="profiling only: sweeps per step")
    ap.add_argument("--temperature", type=float, default=0.0, help="profiling only: another T")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--potts-case", default="",
                    help="profiling only: --workload potts on one lattice, DIM,L,Q,T (e.g. 3,320,3,1.8164)")
    ap.add_argument("--tile-h", type=int, default=0, choices=[0, 32, 64, 96, 128],
                    help="rows per tile (0: the autotuner's choice for this L and T)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_jobs(jobs, rank: int, world: int):
    """Independent jobs split over ranks with no exchange: largest first, each
    to the least-loaded rank (cost = sites x sweeps); every rank computes the
    same assignment and keeps its own share."""
    load = [0] * world
    mine = []
    order = sorted(range(len(jobs)), key=lambda i: (-jobs[i].L * jobs[i].L * jobs[i].sweeps, i))
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += jobs[i].L * jobs[i].L * jobs[i].sweeps
        if r == rank:
            mine.append(jobs[i])
    return mine


def workload_config(w, extra=None):
    cfg = {"workload": f"plain SW, 2D Ising periodic L={w.L}, J=1, T={w.T}, hot start, "
                       f"{w.sweeps} sweeps per step",
           "L": w.L, "T": w.T, "J": 1.0, "sweeps_per_step": w.sweeps,
           "l2": (f"inputs larger than L2 ({w.L * w.L >> 20} MiB spins, {2 * w.L * w.L >> 20} MiB site "
                  f"codes per lattice)" if 3 * w.L * w.L > L2_BYTES else
                  f"state L2-resident ({3 * w.L * w.L >> 10} KiB of spins and site codes)")}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- roofline
def philox_calls_per_start(L: int) -> int:
    """Philox blocks the tile kernel draws to start one sweep: per 128-wide
    tile row, 64 BOND blocks (one per two sites; 128 on rows that begin on an
    odd site, which odd L gives every other row) and the SPIN blocks for the
    clusters that end inside the tile: one when the row's first site is a
    multiple of 128 (its 128 bits are one block), else the two it straddles."""
    tiles_x = (L + 127) // 128
    odd_rows = L // 2 if L % 2 else 0
    bond = tiles_x * (64 * (L - odd_rows) + 128 * odd_rows)
    spin = tiles_x * sum(1 if (y * L) % 128 == 0 else 2 for y in range(L))   # tile rows start at y L + 128 tx
    return bond + spin


def profile_traffic(kernel_src_sha: str, tile_h: int):
    """DRAM bytes per launch of the tile kernel at this tile height from the
    committed ncu summary, or None when that summary was taken on a different
    kernel source (or lacks the height)."""
    try:
        txt = open(PROFILE_FILE).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(rf"dram bytes per launch, tile height {int(tile_h)}:\s*([0-9]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != kernel_src_sha:
        return None
    return int(m_tr.group(1))


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("sw_device.cuh", "sw_engine.cu"):
        h.update(open(os.path.join(ROOT, "paper_0808_2109_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def hbm_peak_gbs():
    """The measured HBM copy bandwidth (driver-written), else the fallback."""
    pk = measured_peaks()
    if "hbm_gbs" in pk:
        return float(pk["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    return 6800.0, "of fallback (6.8 TB/s, an earlier GB300 copy measurement)"


def time_on_stream(torch, stream, fn, reps: int, warm: int = 2) -> float:
    """Average ms of fn() over reps calls, CUDA events on stream."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_philox_peak(torch, swgpu, stream) -> float:
    """Philox4x32-10 blocks/s of the library's probe (sw_bench_philox): 2^32
    BOND blocks per launch on a grid that fills the GPU."""
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = (1 << 32)
    ms = time_on_stream(torch, stream, lambda: swgpu.sw_bench_philox(n, 1, out.data_ptr(), stream), 5)
    return n / (ms * 1e-3)


def measure_l2_peak(torch, swgpu, stream, nbytes: int = 16 << 20, reps: int = 400) -> float:
    """L2 copy bandwidth (GB/s, read + write) of the library's probe
    (sw_bench_l2) on two 16 MiB buffers: 32 MiB in all, resident in L2."""
    src = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda")
    dst = torch.empty_like(src)
    ms = time_on_stream(torch, stream,
                        lambda: swgpu.sw_bench_l2(src.data_ptr(), dst.data_ptr(), nbytes, reps, stream), 3)
    return 2.0 * nbytes * reps / (ms * 1e-3) / 1e9


# ------------------------------------------------------------ cpu baseline
def cpu_baseline_oracle(w):
    """The oracle as it stands, single-threaded, on one sweep of the lattice."""
    import oracle
    oracle.build()
    chain = oracle.sw_chain(w.L, 1.0, w.T, w.seed)
    t0 = time.perf_counter()
    chain.run(1)
    dt = time.perf_counter() - t0
    return {"value": w.L * w.L / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 sweep of the L={w.L} lattice from the hot start ({dt:.1f} s)"}


def _oracle_replicas(args):
    """Worker: run each (L, T, seed, sweeps) replica with the oracle; returns
    the site updates done (runs in a spawned process)."""
    import oracle
    n = 0
    for L, T, seed, sweeps in args:
        oracle.sw_chain(L, 1.0, T, seed).run(sweeps)
        n += L * L * sweeps
    return n


def cpu_baseline_batch(pool, jobs, sample_replicas: int = 64, sweeps: int = 20):
    """The oracle on a bounded sample of the batch mix: the first
    `sample_replicas` replicas of the manifest, `sweeps` sweeps each, on one
    core and on all host cores (one replica per process at a time, a pool
    started before the first GPU call)."""
    import oracle
    oracle.build()
    sample = [(j.L, j.T, j.seed, sweeps) for j in jobs[:sample_replicas]]
    t0 = time.perf_counter()
    n1 = _oracle_replicas(sample)
    t1 = time.perf_counter() - t0
    out = {"value": round(n1 / (t1 * 1e9), 6), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{len(sample)} replicas of the mix (first of the manifest), {sweeps} sweeps each, "
                     f"one core ({t1:.1f} s)"}
    if pool is not None:
        ncores = pool._processes
        pool.map(_oracle_replicas, [[]] * ncores)          # workers up before timing
        t0 = time.perf_counter()
        nall = sum(pool.map(_oracle_replicas, [[a] for a in sample], chunksize=1))
        tall = time.perf_counter() - t0
        out["all_cores"] = {"value": round(nall / (tall * 1e9), 6), "unit": UNIT, "cores": ncores,
                            "kind": "oracle", "sample": f"the same {len(sample)} replicas, one per process "
                                                         f"({tall:.1f} s)"}
    return out


def start_oracle_pool():
    """A spawn pool of one process per host core, for the all-cores oracle
    baseline (started before any GPU call).  Its workers are waited for here,
    so that their start-up does not load the host cores while the end-to-end
    step (host copies and the calls that issue them) is timed."""
    import multiprocessing as mp
    try:
        n = os.cpu_count() or 1
        pool = mp.get_context("spawn").Pool(n)
        pool.map(time.sleep, [0.05] * (4 * n), chunksize=1)   # every worker up and idle
        return pool
    except OSError:
        return None


# --------------------------------------------------------------- our arm
def run_gb300(args):
    import numpy as np
    import torch
    from paper_0808_2109_gb300 import _build, swgpu, workloads

    rank, world, local = dist_env()
    profiling = bool(args.lattice or args.sweeps or args.temperature)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_batch and not profiling:
        pool = start_oracle_pool()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    w = workloads.LARGE
    if profiling:
        w = workloads.Plain(args.lattice or w.L, args.temperature or w.T, args.sweeps or w.sweeps, w.seed)
    K, W = args.steps, args.warmup
    N = w.L * w.L
    stream = torch.cuda.Stream()
    tile_h = args.tile_h or swgpu.sw_autotune(w.L, w.T)
    lat = swgpu.Lattice(w.L, T=w.T, seed=w.seed + rank, tile_h=tile_h)
    lat.set_stream(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(W):
        lat.sweep(w.sweeps)
    lat.sync()
    lat.observables()

    # ---- timed region: K steps, lattice resident in HBM
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        lat.sweep(w.sweeps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    obs = lat.observables()
    assert len(obs) == K * w.sweeps
    value = world * N * w.sweeps * K / (ms * 1e6)

    # ---- per-kernel device times: the same steps, kernels bracketed by events
    prof_steps = max(1, min(K, 3))
    lat.profile(True)
    for _ in range(prof_steps):
        lat.sweep(w.sweeps)
    st = lat.profile_read()
    lat.profile(False)
    lat.observables()
    roofline = tile_roofline(torch, swgpu, stream, w, tile_h, st, ms / (K * w.sweeps))

    # ---- end to end through the public API with pinned host buffers
    e2e_steps = max(1, min(K, 5))
    h_in = torch.empty(N, dtype=torch.uint8, pin_memory=True).numpy()
    h_out = torch.empty(N, dtype=torch.uint8, pin_memory=True).numpy()
    h_in[:] = lat.spins()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    part = [0.0, 0.0, 0.0]   # host wall time: upload + state check, sweeps + observables, download
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        lat.set_spins(h_in)                  # host -> device: this step's input lattice (checked)
        tb = time.perf_counter()
        lat.sweep(w.sweeps)
        o = lat.observables()                # device -> host: per-sweep observables
        tc = time.perf_counter()
        swgpu.sw_get_spins(lat.h, w.L, h_out)  # device -> host: the resulting lattice
        td = time.perf_counter()
        part[0] += tb - ta
        part[1] += tc - tb
        part[2] += td - tc
        h_in, h_out = h_out, h_in
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * N * w.sweeps * e2e_steps / (e2e_s * 1e9), "unit": UNIT,
           "h2d_bytes_per_step": N, "d2h_bytes_per_step": N + w.sweeps * swgpu.OBS_DTYPE.itemsize,
           "steps": e2e_steps,
           "ms_per_step": {"upload_and_check": round(1e3 * part[0] / e2e_steps, 3),
                           "sweeps_and_observables": round(1e3 * part[1] / e2e_steps, 3),
                           "download": round(1e3 * part[2] / e2e_steps, 3)}}
    del o
    lat.close()

    batched = None
    if not args.no_batch and not profiling:
        batched = run_batch_vs_solo(swgpu, workloads, rank, world, barrier, pool)
    served = None
    if not args.no_serve and not profiling and rank == 0 and world == 1:
        served = run_served(swgpu, workloads, local, args.serve_seconds)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_oracle(w)
        out = {
            "metric": METRIC if not profiling else f"SW site updates/ns at T={w.T} (L={w.L})",
            "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": workload_config(w, {"parallelism": f"replicas x{world}",
                                          "seeds": f"{w.seed}..{w.seed + world - 1}"}),
            "tile_h": tile_h, "hbm_gbs_achieved": roofline["achieved"],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "batched": batched, "served": served,
            "gpu_launches": K * (LAUNCHES_PER_SWEEP * w.sweeps + 1),
            "clocks": clk, "impl": "gb300",
        }
    if pool is not None:
        pool.terminate()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def tile_roofline(torch, swgpu, stream, w, tile_h, st, ms_per_sweep):
    """Both ceilings of the dominant kernel (the tile kernel), each measured
    in this run: HBM (the algorithmic 10 B/site of a sweep against the
    measured copy bandwidth; the DRAM bytes ncu counted per launch beside it)
    and the integer pipe (the Philox blocks a launch draws against the
    library's Philox probe).  Neither is what binds the kernel: it issues
    instructions on about two thirds of its cycles and waits on dependent
    shared-memory loads and barriers in the union-find (the ncu summaries in
    profiles/)."""
    N = w.L * w.L
    tile_s = st["tile_ms"] / st["tile_launches"] * 1e-3
    peak, peak_src = hbm_peak_gbs()
    achieved = ALG_BYTES_PER_SITE * N / tile_s / 1e9
    traffic = profile_traffic(kernel_source_sha(), tile_h)
    blocks = philox_calls_per_start(w.L)
    philox_peak = measure_philox_peak(torch, swgpu, stream)
    l2_peak = measure_l2_peak(torch, swgpu, stream)
    alu_achieved = blocks / tile_s
    sweep_gbs = ALG_BYTES_PER_SITE * N / (ms_per_sweep * 1e-3) / 1e9
    return {
        "bound": "hbm", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": traffic,
        "peak_source": peak_src,
        "kernel": f"k_tile<{tile_h}> (fused finish/start of a sweep)",
        "bytes_per_site_algorithmic": ALG_BYTES_PER_SITE,
        "units_per_launch": N,
        "tile_kernel_avg_ms": round(tile_s * 1e3, 4),
        "merge_group_avg_ms": round(st["merge_ms"] / max(st["merge_groups"], 1), 4),
        "dram_gbs_measured": round(traffic / tile_s / 1e9, 1) if traffic is not None else None,
        "frac_dram_measured": round(traffic / tile_s / 1e9 / peak, 4) if traffic is not None else None,
        "sweep_frac_hbm": round(sweep_gbs / peak, 4),
        "alu": {"achieved": round(alu_achieved / 1e9, 2), "peak": round(philox_peak / 1e9, 2),
                "unit": "G Philox4x32-10 blocks/s", "frac": round(alu_achieved / philox_peak, 4),
                "blocks_per_site": round(blocks / N, 6),
                "site_updates_per_ns_ceiling": round(philox_peak / (blocks / N) / 1e9, 1),
                "peak_source": "measured in this run: sw_bench_philox, 2^32 BOND blocks per launch"},
        "l2_gbs_peak": round(l2_peak, 1),
        "l2_peak_source": "measured in this run: sw_bench_l2, 32 MiB copy resident in L2",
        "binding": "neither ceiling: instruction issue (about 2/3 of cycles) and dependent shared-memory "
                   "latency in the union-find, with phase barriers (profiles/k_tile_L4096_full.md)",
    }


# ------------------------------------------------------ batched vs solo
def run_batch_vs_solo(swgpu, workloads, rank, world, barrier, pool=None):
    """The uneven 512-replica mix (500 sweeps each) through the batch server,
    then the same replicas one at a time on the same GPU: once with each
    lattice created (and destroyed) inside the timed region, once with the
    lattices created and their sweep graphs captured beforehand (sweeps
    only).  Replicas shard over ranks with no exchange."""
    all_jobs = workloads.batch_manifest()
    jobs = shard_jobs(all_jobs, rank, world)
    specs = [{"L": j.L, "T": j.T, "sweeps": j.sweeps, "seed": j.seed} for j in jobs]
    updates = sum(j.L * j.L * j.sweeps for j in jobs)
    srv = swgpu.Server()
    for L in sorted({j.L for j in jobs}):            # autotune outside the timed region
        for T in (2.0, 2.3, 2.6):
            swgpu.sw_autotune(L, T)
    barrier()
    t0 = time.perf_counter()
    ids = srv.submit(specs, want_obs=True)
    srv.wait_all(0.0)
    t_batch = max_over_ranks(time.perf_counter() - t0)
    res = [srv.poll(i) for i in ids]
    assert all(r is not None and r[0].status == 0 for r in res)
    stats = srv.stats()
    srv.close()
    # solo, create + sweeps + observables + destroy per replica
    barrier()
    t0 = time.perf_counter()
    for sp in specs:
        lat = swgpu.Lattice(sp["L"], T=sp["T"], seed=sp["seed"])
        lat.sweep(sp["sweeps"])
        lat.observables()
        lat.close()
    t_solo = max_over_ranks(time.perf_counter() - t0)
    # solo, sweeps only: lattices made and their graphs captured beforehand
    lats = [swgpu.Lattice(sp["L"], T=sp["T"], seed=sp["seed"]) for sp in specs]
    for lat, sp in zip(lats, specs):
        lat.sweep(sp["sweeps"])   # captures the graph of this run length
        lat.sync()
        lat.observables()
    barrier()
    t0 = time.perf_counter()
    for lat, sp in zip(lats, specs):
        lat.sweep(sp["sweeps"])
        lat.observables()         # waits for the lattice's sweeps
    t_solo_sweeps = max_over_ranks(time.perf_counter() - t0)
    for lat in lats:
        lat.close()
    total = updates * world   # equal shares by construction, up to one job
    out = {"replicas": 512, "sweeps": 500, "site_updates": int(total),
           "value": round(total / (t_batch * 1e9), 3), "unit": UNIT,
           "solo_value": round(total / (t_solo * 1e9), 3),
           "solo_sweep_only_value": round(total / (t_solo_sweeps * 1e9), 3),
           "speedup_vs_solo": round(t_solo / t_batch, 3),
           "speedup_vs_solo_sweep_only": round(t_solo_sweeps / t_batch, 3),
           "batch_s": round(t_batch, 3), "solo_s": round(t_solo, 3), "solo_sweep_only_s": round(t_solo_sweeps, 3),
           "launch_groups": int(stats["launches"]),
           "timing": "wall clock from submit to last completion (host), max over ranks; solo: the same "
                     "replicas one at a time through sw_create/sw_sweep/sw_observables, with and without "
                     "creation, graph capture and destruction in the timed region"}
    if rank == 0 and world == 1 and pool is not None:
        out["cpu_baseline"] = cpu_baseline_batch(pool, all_jobs)
    return out


# ------------------------------------------------------------------- serve
def serve_trace_run(swgpu, jobs, duration_s):
    """Replays jobs in real time against a fresh server: each is submitted at
    its arrival time; latency = submit -> finished (server clocks)."""
    import numpy as np
    srv = swgpu.Server()
    ids = []
    t0 = time.perf_counter()
    for job in jobs:
        delay = job.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        sp = {"L": job.L, "sweeps": job.sweeps, "seed": job.seed}
        if job.pcc:
            sp["pcc"] = True
        else:
            sp["T"] = job.T
        ids += srv.submit([sp], want_obs=False)
    srv.wait_all(0.0)
    wall = time.perf_counter() - t0
    lat, upd = [], 0
    for i, job in zip(ids, jobs):
        r, _ = srv.poll(i)
        assert r.status == 0
        lat.append(r.queued_s + r.run_s)
        upd += job.L * job.L * job.sweeps
    srv.close()
    lat = np.array(lat)
    return {"jobs": len(jobs), "value": round(upd / (wall * 1e9), 3), "unit": UNIT,
            "offered_site_updates_per_ns": round(upd / (duration_s * 1e9), 3),
            "latency_s": {"p50": round(float(np.percentile(lat, 50)), 4),
                          "p99": round(float(np.percentile(lat, 99)), 4),
                          "max": round(float(lat.max()), 4)},
            "wall_s": round(wall, 2), "arrival_window_s": duration_s,
            "drain_s": round(wall - duration_s, 2)}


def run_served(swgpu, workloads, local, duration_s, rate=200.0, probe_s=20.0):
    """The configured Poisson trace (200 jobs/s), then a probe of the rate
    the server keeps up with: the trace's job mix at 85% of the rate its
    measured capacity can absorb (capacity / mean work per job), for
    probe_s seconds.  While the first trace's queue never empties, its
    aggregate throughput is the server's capacity."""
    for L in (32, 64, 128, 256, 512, 1024, 2048, 4096):
        for T in (2.0, 2.3, 2.6):
            swgpu.sw_autotune(L, T)
    clocks = ClockSampler(local)
    clocks.start()
    trace = workloads.serve_trace(rate_hz=rate, duration_s=duration_s)
    main = serve_trace_run(swgpu, trace, duration_s)
    mean_work = sum(j.L * j.L * j.sweeps for j in trace) / len(trace)
    capacity = main["value"] * 1e9   # site updates/s while the queue is never empty
    keep_rate = 0.85 * capacity / mean_work
    probe = serve_trace_run(swgpu, workloads.serve_trace(rate_hz=keep_rate, duration_s=probe_s, rng_seed=20262),
                            probe_s)
    probe["rate_jobs_per_s"] = round(keep_rate, 1)
    main.update({"rate_jobs_per_s": rate, "clocks": clocks.stop(),
                 "workload": "Poisson arrivals, L log-uniform [32,4096], sweeps U[10,1000], 80% SW T~U[1.8,3.2], "
                             "20% PCC; lattice state resident on the device, admission by device memory",
                 "served_jobs_per_s": round(capacity / mean_work, 1),
                 "keep_up_probe": probe})
    return main


def run_serve(args):
    """--workload serve: the trace at --serve-rate for --serve-seconds."""
    import torch
    from paper_0808_2109_gb300 import _build, swgpu, workloads

    rank, world, local = dist_env()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    _build.build()
    for L in (32, 64, 128, 256, 512, 1024, 2048, 4096):
        for T in (2.0, 2.3, 2.6):
            swgpu.sw_autotune(L, T)
    clocks = ClockSampler(local)
    clocks.start()
    trace = workloads.serve_trace(rate_hz=args.serve_rate, duration_s=args.serve_seconds)
    out = serve_trace_run(swgpu, trace, args.serve_seconds)
    out.update({"metric": f"served SW/PCC site updates/ns (Poisson {args.serve_rate:g} jobs/s)", "n_gpus": 1,
                "higher_is_better": True, "clocks": clocks.stop(), "data": "synthetic", "impl": "gb300"})
    return out


# ------------------------------------------------------- configured runs
def run_configs(args):
    """Every configured run once on the GPU (CUDA events around one whole
    run, after one untimed run) with its roofline fraction -- HBM, or L2 when
    the lattice's state fits L2 -- and the oracle timed beside it on a
    bounded sample (one core)."""
    import torch
    import oracle
    from paper_0808_2109_gb300 import _build, swgpu, workloads

    rank, world, local = dist_env()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    _build.build()
    oracle.build()
    stream = torch.cuda.Stream()
    hbm, _ = hbm_peak_gbs()
    l2 = measure_l2_peak(torch, swgpu, stream)
    cases = [("plain", workloads.SMALL, 1000)] + [("plain", r, 2) for r in workloads.REGIMES] + \
            [("plain", workloads.LARGE, 1), ("pcc", workloads.PCC_RUN, 20)]
    clocks = ClockSampler(local)
    clocks.start()
    rows = []
    for kind, w, osweeps in cases:
        L = w.L
        n = w.sweeps
        if kind == "pcc":   # the tile height the autotuner picks for the critical plain lattice
            th = swgpu.sw_autotune(L, workloads.T_CRITICAL_ROUNDED)
            mk = lambda: swgpu.Lattice(L, seed=w.seed, pcc=True, tile_h=th)
            ork = lambda: oracle.pcc_chain(L, w.seed)
        else:
            th = swgpu.sw_autotune(L, w.T)
            mk = lambda: swgpu.Lattice(L, T=w.T, seed=w.seed, tile_h=th)
            ork = lambda: oracle.sw_chain(L, 1.0, w.T, w.seed)
        with mk() as lat:
            lat.set_stream(stream)
            lat.sweep(n)
            lat.sync()
            lat.observables()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.sweep(n)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            lat.observables()
        rate = L * L * n / (ms * 1e6)
        state_bytes = L * L * 3 + (L * L) // 4   # spins, site codes, bond bits: the per-site state
        resident = state_bytes < (96 << 20)
        peak = l2 if resident else hbm
        ch = ork()
        t0 = time.perf_counter()
        ch.run(osweeps)
        ot = time.perf_counter() - t0
        rows.append({"config": (f"PCC L={L} {n} sweeps" if kind == "pcc" else f"SW L={L} T={w.T} {n} sweeps"),
                     "gpu_site_updates_per_ns": round(rate, 3), "gpu_ms": round(ms, 3),
                     "roofline": {"bound": "l2" if resident else "hbm",
                                  "achieved_gbs": round(rate * ALG_BYTES_PER_SITE, 1), "peak_gbs": round(peak, 1),
                                  "frac": round(rate * ALG_BYTES_PER_SITE / peak, 4)},
                     "cpu_oracle_1core": {"value": round(L * L * osweeps / (ot * 1e9), 6), "unit": UNIT,
                                          "sample": f"{osweeps} sweeps from the hot start ({ot:.1f} s)"}})
    return {"metric": "configured runs: site updates/ns, roofline fraction, oracle beside", "rows": rows,
            "l2_gbs_peak": round(l2, 1), "hbm_gbs_peak": round(hbm, 1), "clocks": clocks.stop(),
            "n_gpus": 1, "data": "synthetic", "impl": "gb300"}


def run_batch64(args):
    """Launch gaps of the batched form on small lattices: 512 L=64 replicas
    through the server, wall clock against the device time of the launches
    (the sum of kernel times comes from a separate ncu launch list)."""
    import torch
    from paper_0808_2109_gb300 import _build, swgpu, workloads

    rank, world, local = dist_env()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    _build.build()
    swgpu.sw_autotune(64, 2.3)
    specs = [{"L": 64, "T": 2.0 + 0.6 * (r % 32) / 31.0, "sweeps": args.sweeps or 500, "seed": 1000 + r}
             for r in range(512)]
    res = {}
    for rep in range(args.warmup + args.steps):
        with swgpu.Server() as srv:
            t0 = time.perf_counter()
            ids = srv.submit(specs, want_obs=True)
            srv.wait_all(0.0)
            dt = time.perf_counter() - t0
            st = srv.stats()
        if rep >= args.warmup:
            res.setdefault("wall_s", []).append(round(dt, 4))
            res["launch_groups"] = int(st["launches"])
    upd = 512 * 64 * 64 * (args.sweeps or 500)
    return {"metric": "batched SW, 512 x L=64 (launch-bound)", "wall_s": res["wall_s"],
            "value": round(upd / (min(res["wall_s"]) * 1e9), 3), "unit": UNIT,
            "launch_groups": res["launch_groups"], "n_gpus": 1, "impl": "gb300"}


# ------------------------------------------------------------- Potts / 3D
POTTS_BYTES_PER_SITE = 10   # the stated minimum of a sweep: old state in, label out, label in, new state out
POTTS_PROFILE_FILE = os.path.join(ROOT, "profiles", "k_potts_tiles_critical.md")


def potts_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("sw_device.cuh", "sw_potts.cu"):
        h.update(open(os.path.join(ROOT, "paper_0808_2109_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def potts_profile_traffic(sha: str, dim: int, L: int, q: int):
    """DRAM bytes per launch of the Potts tile kernel on this lattice from the
    committed ncu summary, or None when it was taken on other sources."""
    try:
        txt = open(POTTS_PROFILE_FILE).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(rf"dram bytes per launch, {int(dim)}D L={int(L)} q={int(q)}:\s*([0-9]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != sha:
        return None
    return int(m_tr.group(1))


def potts_philox_per_site(dim: int, L: int) -> float:
    """Philox blocks the Potts tile kernel draws per site to start a sweep
    when 4 divides L: 2D, two BOND blocks and one QSPIN block per lane for a
    128-site row; 3D, 24 BOND and 8 QSPIN blocks per 32-site row."""
    return 0.75 if dim == 2 else 1.0


def run_potts(args):
    """The q-state Potts / 3D path at four critical points (2D: exact T_c;
    3D: the published estimates), each lattice larger than L2: W warm-up
    steps of 10 sweeps, then K steps timed with CUDA events on its stream,
    then one step in profiling mode (events around every tile kernel and
    merge) for the per-kernel times behind the roofline."""
    import math
    import torch
    from paper_0808_2109_gb300 import _build, swgpu

    rank, world, local = dist_env()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    _build.build()
    cases = [(2, 8192, 2, 1.0 / math.log(1.0 + math.sqrt(2.0))),
             (2, 8192, 3, 1.0 / math.log(1.0 + math.sqrt(3.0))),
             (3, 512, 2, 2.2557),     # q=2 is Ising at J/2: 4.5115 / 2
             (3, 512, 3, 1.8164)]
    if args.potts_case:
        d, l, qq, tt = args.potts_case.split(",")
        cases = [(int(d), int(l), int(qq), float(tt))]
    SW = 10
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local)
    clocks.start()
    rows, upd, ms_tot = [], 0, 0.0
    for dim, L, q, T in cases:
        with swgpu.PottsLattice(dim, L, q, T=T, seed=1) as lat:
            lat.set_stream(stream)
            for _ in range(args.warmup):
                lat.sweep(SW)
            lat.sync()
            lat.observables()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                lat.sweep(SW)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            assert len(lat.observables()) == args.steps * SW
            lat.profile(True)
            lat.sweep(SW)
            st = lat.profile_read()
            lat.profile(False)
            lat.observables()
            n = L ** dim * SW * args.steps
            upd += n
            ms_tot += ms
            rows.append({"dim": dim, "L": L, "q": q, "T": round(T, 6),
                         "value": round(n / (ms * 1e6), 3), "ms_per_sweep": round(ms / (SW * args.steps), 4),
                         "tile_kernel_avg_ms": round(st["tile_ms"] / st["tile_launches"], 4),
                         "merge_group_avg_ms": round(st["merge_ms"] / st["merge_groups"], 4)})
    clk = clocks.stop()
    value = upd / (ms_tot * 1e6)
    hbm, src = hbm_peak_gbs()
    philox_peak = measure_philox_peak(torch, swgpu, stream)
    # the dominant kernel: the tile kernel of the case with the most tile time
    # (3D L=512 q=3 in the default set); one launch finishes a sweep and
    # starts the next over L^d sites
    dom = max(rows, key=lambda r: r["tile_kernel_avg_ms"] * (r["L"] ** r["dim"]))
    sites = dom["L"] ** dom["dim"]
    tile_s = dom["tile_kernel_avg_ms"] * 1e-3
    achieved = POTTS_BYTES_PER_SITE * sites / tile_s / 1e9
    traffic = potts_profile_traffic(potts_source_sha(), dom["dim"], dom["L"], dom["q"])
    blocks = potts_philox_per_site(dom["dim"], dom["L"]) * sites
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": round(hbm, 1), "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_source": src,
                "kernel": f"k_ptile<{dom['dim']}> ({dom['dim']}D L={dom['L']} q={dom['q']}: fused finish/start "
                          "of a sweep, the largest share of the workload's device time)",
                "bytes_per_site_algorithmic": POTTS_BYTES_PER_SITE, "units_per_launch": sites,
                "tile_kernel_avg_ms": dom["tile_kernel_avg_ms"], "merge_group_avg_ms": dom["merge_group_avg_ms"],
                "whole_workload_frac_hbm": round(value * POTTS_BYTES_PER_SITE / hbm, 4),
                "alu": {"philox_blocks_per_site": potts_philox_per_site(dom["dim"], dom["L"]),
                        "achieved_blocks_per_s": round(blocks / tile_s, 1),
                        "peak_blocks_per_s": round(philox_peak, 1),
                        "frac": round(blocks / tile_s / philox_peak, 4),
                        "peak_source": "measured in this run: sw_bench_philox, 2^32 BOND blocks per launch"},
                "binding": "neither ceiling: instruction issue (70-76% of cycles) and the union-find's "
                           "dependent shared-memory latency (profiles/k_potts_tiles_critical.md)"}
    if traffic is not None:
        roofline["dram_gbs_measured"] = round(traffic / tile_s / 1e9, 1)
        roofline["frac_dram_measured"] = round(traffic / tile_s / 1e9 / hbm, 4)
    return {"metric": "Potts/3D SW site updates/ns (four critical lattices)", "value": round(value, 3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "q-state Potts, hot start, 10 sweeps per step", "cases": rows,
                       "l2": "every lattice larger than L2 (states, labels and site codes >= 400 MB)"},
            "roofline": roofline, "clocks": clk, "impl": "gb300"}


# ---------------------------------------------------------- reference arm
REF_SAMPLE_L = 4096


def run_reference(args):
    """The CPU oracle, single-threaded, as it stands.  Each step is a bounded
    sample of the benchmark workload: one sweep of an L=4096 lattice with the
    workload's J, T, seed and hot start (an L=16384 sweep takes ~17 s on one
    core, too long for K steps).  The line names the same workload, metric
    and unit as the GPU arm; its `sample` says what each step timed."""
    from paper_0808_2109_gb300 import workloads
    import oracle

    rank, world, _ = dist_env()
    if rank != 0:
        return None
    oracle.build()
    w = workloads.LARGE
    Ls = REF_SAMPLE_L
    chain = oracle.sw_chain(Ls, 1.0, w.T, w.seed)
    for _ in range(args.warmup):
        chain.run(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        chain.run(1)
    dt = time.perf_counter() - t0
    value = Ls * Ls * args.steps / (dt * 1e9)
    sample = (f"each step: one sweep of an L={Ls} lattice at T={w.T}, J=1, seed {w.seed}, hot start "
              f"(a bounded sample of the L={w.L} workload), single-threaded oracle")
    return {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload_config(w, {"parallelism": f"replicas x{world}",
                                                          "seeds": f"{w.seed}..{w.seed + world - 1}"}),
        "sample": sample, "site_updates_per_step": Ls * Ls, "impl": "reference",
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "serve":
        out = run_serve(args)
    elif args.workload == "potts":
        out = run_potts(args)
    elif args.workload == "configs":
        out = run_configs(args)
    elif args.workload == "batch64":
        out = run_batch64(args)
    else:
        out = run_gb300(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
