"""Seeded synthetic inputs shared by the tests, the benchmark and the server.

Only input generation lives here -- lattice shapes, temperatures, seeds,
update counts and arrival times -- drawn from numpy's Philox bit generator;
none of the update's arithmetic.  Every table is a pure function of its key,
so the GPU path and the CPU oracle see the same inputs.
"""
import math

import numpy as np

TC_2D = 2.0 / math.log(1.0 + math.sqrt(2.0))   # Onsager, J = 1
TC_3D = 4.5115                                  # simple cubic, J = 1


def _rng(key):
    return np.random.Generator(np.random.Philox(key=key))


def batched_replicas(n=512, key=0xBA7C4, sizes=(64, 128, 256, 512, 1024), t_range=(2.0, 2.6),
                     seed_base=1000):
    """Independent 2D replicas: L uniform over `sizes`, T uniform in t_range,
    seed seed_base + i.  Returns a list of dicts (dim, L, T, seed)."""
    g = _rng(key)
    Ls = g.integers(0, len(sizes), size=n)
    Ts = g.uniform(t_range[0], t_range[1], size=n)
    return [dict(dim=2, L=int(sizes[Ls[i]]), T=float(Ts[i]), seed=seed_base + i)
            for i in range(n)]


def _log_uniform_int(g, lo, hi, size):
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def serving_trace(n=1000, rate=200.0, key=0x5E4F3, frac_2d=0.7, l2d=(32, 2048), l3d=(16, 128),
                  t_scale=(0.9, 1.1), updates=(1_000, 100_000), seed_base=50_000):
    """Poisson stream of Wolff-run requests.

    Arrival gaps are exponential with mean 1/rate seconds; 70% of requests are
    2D with L log-uniform in l2d, the rest 3D with L log-uniform in l3d; T is
    uniform in t_scale * T_c(D); the number of updates is log-uniform in
    `updates`.  Returns a list of dicts (id, arrival_s, dim, L, T, seed,
    n_updates), arrival times increasing."""
    g = _rng(key)
    gaps = g.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps)
    is2d = g.uniform(size=n) < frac_2d
    L2 = _log_uniform_int(g, *l2d, size=n)
    L3 = _log_uniform_int(g, *l3d, size=n)
    ts = g.uniform(t_scale[0], t_scale[1], size=n)
    nu = _log_uniform_int(g, *updates, size=n)
    out = []
    for i in range(n):
        dim = 2 if is2d[i] else 3
        L = int(L2[i] if dim == 2 else L3[i])
        out.append(dict(id=i, arrival_s=float(arrivals[i]), dim=dim, L=L,
                        T=float(ts[i] * (TC_2D if dim == 2 else TC_3D)), seed=seed_base + i,
                        n_updates=int(nu[i])))
    return out
