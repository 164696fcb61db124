"""Temperature sweep and Binder ratio on the batched engine.

Section 5 of the paper illustrates the method with the Binder ratio
U(T) = 1 - <M^4> / (3 <M^2>^2) of the 2D and 3D Ising model (its Fig. 2: 2D
L = 512..4096 with 5000 discarded and 50000 measured single-cluster updates,
3D L = 64..256 with 10000 + 100000).  Here every (L, T) point is one replica
of the batched form, so a whole sweep runs in shared launches; the
magnetisation comes from the per-update records (M after each update), and
the error bars from a jackknife over blocks of the time series.
"""
import itertools

import numpy as np

from . import WolffLattice
from .batched import BatchedRunner, Plan


def binder_from_series(M, n_blocks=32):
    """U = 1 - <M^4>/(3<M^2>^2) of a magnetisation series, with its jackknife
    error over n_blocks contiguous blocks."""
    m = np.asarray(M, dtype=np.float64)
    m2, m4 = m ** 2, m ** 4

    def u(a2, a4):
        return 1.0 - a4 / (3.0 * a2 * a2)

    full = u(m2.mean(), m4.mean())
    nb = max(2, min(n_blocks, len(m) // 4))
    size = len(m) // nb
    b2 = m2[:nb * size].reshape(nb, size).mean(axis=1)
    b4 = m4[:nb * size].reshape(nb, size).mean(axis=1)
    s2, s4 = b2.sum(), b4.sum()
    jk = np.array([u((s2 - b2[k]) / (nb - 1), (s4 - b4[k]) / (nb - 1)) for k in range(nb)])
    err = float(np.sqrt((nb - 1) / nb * ((jk - jk.mean()) ** 2).sum()))
    return float(full), err


def sweep(dim, Ls, Ts, discard, measure, seed_base=70_000, chunk=2000, cluster_size=1,
          block_threads=256, start="random"):
    """One replica per (L, T); returns a list of dicts with L, T, U, U_err,
    <|m|>, <E_bond>/N, mean cluster size, and the number of measured updates."""
    import torch
    points = list(itertools.product(Ls, Ts))
    lats = [WolffLattice(dim, L, T, seed=seed_base + k) for k, (L, T) in enumerate(points)]
    if start == "ordered":
        for lat in lats:
            lat.set_state(np.ones(lat.N, np.int8), 0)
    runner = BatchedRunner(lats, Plan([(list(range(len(lats))), cluster_size, block_threads)],
                                      "sweep"))
    done = 0
    while done < discard:
        k = min(chunk, discard - done)
        runner.run(k, records=False)
        done += k
    series = [[] for _ in lats]
    done = 0
    while done < measure:
        k = min(chunk, measure - done)
        bufs = runner.run(k, records=True)
        torch.cuda.synchronize()
        for i, rec in enumerate(runner.records_numpy(bufs, k)):
            series[i].append(rec)
        done += k
    runner.close()
    out = []
    for (L, T), lat, parts in zip(points, lats, series):
        rec = np.concatenate(parts)
        N = L ** dim
        U, err = binder_from_series(rec["M"])
        out.append({"L": L, "T": T, "U": U, "U_err": err,
                    "abs_m": float(np.abs(rec["M"]).mean() / N),
                    "e_bond_per_site": float(rec["E"].mean() / N),
                    "mean_cluster": float(rec["C"].mean()), "updates": int(len(rec))})
        lat.close()
    return out


def crossing(points, L_small, L_large):
    """Temperature where U(L_small) and U(L_large) cross (linear interpolation
    between the bracketing sweep temperatures), or None."""
    a = sorted((p["T"], p["U"]) for p in points if p["L"] == L_small)
    b = sorted((p["T"], p["U"]) for p in points if p["L"] == L_large)
    diff = [(ta, ua - ub) for (ta, ua), (tb, ub) in zip(a, b)]
    for (t0, d0), (t1, d1) in zip(diff, diff[1:]):
        if d0 == 0:
            return t0
        if d0 * d1 < 0:
            return t0 + (t1 - t0) * d0 / (d0 - d1)
    return None
