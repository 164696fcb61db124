"""The seeded input tables (replicas, request trace) are deterministic and
follow their stated distributions."""
import math

import numpy as np

from paper_1110_0899_gb300 import workloads


def test_batched_replicas_table():
    a = workloads.batched_replicas(512)
    b = workloads.batched_replicas(512)
    assert a == b and len(a) == 512
    Ls = np.array([r["L"] for r in a])
    Ts = np.array([r["T"] for r in a])
    assert set(Ls.tolist()) == {64, 128, 256, 512, 1024}
    assert Ts.min() >= 2.0 and Ts.max() <= 2.6
    assert [r["seed"] for r in a] == list(range(1000, 1512))
    for L in (64, 128, 256, 512, 1024):   # uniform over five sizes
        assert abs((Ls == L).mean() - 0.2) < 0.06


def test_serving_trace():
    tr = workloads.serving_trace(1000)
    assert tr == workloads.serving_trace(1000)
    arr = np.array([r["arrival_s"] for r in tr])
    assert np.all(np.diff(arr) > 0)
    assert abs(arr[-1] / 1000 - 1 / 200) < 0.15 / 200 * 10   # mean gap 5 ms
    d2 = np.array([r["dim"] == 2 for r in tr])
    assert abs(d2.mean() - 0.7) < 0.05
    for r in tr:
        lo, hi = ((32, 2048) if r["dim"] == 2 else (16, 128))
        assert lo <= r["L"] <= hi
        tc = workloads.TC_2D if r["dim"] == 2 else workloads.TC_3D
        assert 0.9 * tc - 1e-9 <= r["T"] <= 1.1 * tc + 1e-9
        assert 1000 <= r["n_updates"] <= 100_000
    logn = np.log([r["n_updates"] for r in tr])
    assert abs(logn.mean() - 0.5 * (math.log(1e3) + math.log(1e5))) < 0.2
