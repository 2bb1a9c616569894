"""The seeded workload generators: shapes and distributions as configured."""
import math

import numpy as np

from paper_0808_2109_gb300 import workloads


def test_batch_manifest_mix():
    jobs = workloads.batch_manifest()
    assert len(jobs) == 512
    Ls = np.array([j.L for j in jobs])
    for L, w in zip([64, 128, 256, 512, 1024], [0.4, 0.25, 0.2, 0.1, 0.05]):
        assert abs((Ls == L).mean() - w) < 4 * math.sqrt(w * (1 - w) / 512)
    Ts = sorted({round(j.T, 9) for j in jobs})
    assert len(Ts) == 32 and Ts[0] == 2.0 and abs(Ts[-1] - 2.6) < 1e-12
    assert [j.seed for j in jobs] == list(range(1000, 1512))
    assert all(j.sweeps == 500 for j in jobs)
    assert workloads.batch_manifest() == jobs   # deterministic


def test_serve_trace_shape():
    jobs = workloads.serve_trace()
    n = len(jobs)
    assert abs(n - 12000) < 5 * math.sqrt(12000)
    t = np.array([j.arrival_s for j in jobs])
    assert (np.diff(t) > 0).all() and t[-1] < 60.0
    Ls = np.array([j.L for j in jobs])
    assert Ls.min() >= 32 and Ls.max() <= 4096
    assert abs(np.log(Ls).mean() - 0.5 * (math.log(32) + math.log(4096))) < 0.05
    pcc = np.array([j.pcc for j in jobs])
    assert abs(pcc.mean() - 0.2) < 0.02
    Ts = np.array([j.T for j in jobs if not j.pcc])
    assert Ts.min() >= 1.8 and Ts.max() <= 3.2
    sw = np.array([j.sweeps for j in jobs])
    assert sw.min() >= 10 and sw.max() <= 1000


def test_configured_lattices():
    assert workloads.SMALL.L == 64 and workloads.SMALL.sweeps == 1000
    assert workloads.LARGE.L == 16384 and workloads.LARGE.sweeps == 50
    assert [w.T for w in workloads.REGIMES] == [2.0, 2.269185, 3.0]
    assert workloads.PCC_RUN.L == 2048 and workloads.PCC_RUN.sweeps == 10000
