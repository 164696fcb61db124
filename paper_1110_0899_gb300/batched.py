"""Batched form: many independent lattices per launch, with an autotuner.

A plan splits the lattices into groups; each group is launched through one
wolff_batch (one thread-block cluster per lattice, the C ABI's batched entry
point) on its own CUDA stream, so groups with different team shapes run
concurrently.  The autotuner times candidate plans on throw-away copies of
the workload (same shapes and temperatures, other seeds) and caches the
winner per GPU and workload signature.  No plan changes any result: each
lattice follows the chain it would follow alone.
"""
import hashlib
import json
import os
import time

import numpy as np

from . import (RECORD_BYTES, WolffBatch, WolffLattice, _build, records_to_numpy)


class Plan:
    """groups: list of (indices, cluster_size, block_threads)."""

    def __init__(self, groups, label=""):
        self.groups = [(list(ix), int(cs), int(th)) for ix, cs, th in groups]
        self.label = label

    def to_json(self):
        return {"label": self.label,
                "groups": [{"n": len(ix), "cluster_size": cs, "block_threads": th}
                           for ix, cs, th in self.groups]}


class BatchedRunner:
    """Executes a plan over a list of lattices created on the caller's device."""

    def __init__(self, lattices, plan):
        import torch
        self.lattices = lattices
        self.plan = plan
        self.streams = [torch.cuda.Stream() for _ in plan.groups]
        self.batches = [WolffBatch(max(1, len(ix)), stream=st)
                        for (ix, _, _), st in zip(plan.groups, self.streams)]
        self._records = None
        self._rec_n = 0

    def record_buffers(self, n):
        import torch
        if self._records is None or self._rec_n < n:
            flat = torch.empty(len(self.lattices) * n * RECORD_BYTES, dtype=torch.uint8,
                               device="cuda")
            self._records = [flat[i * n * RECORD_BYTES:(i + 1) * n * RECORD_BYTES]
                             for i in range(len(self.lattices))]
            self._rec_n = n
        return self._records

    def run(self, n_updates, records=True):
        """Enqueues n_updates updates of every lattice; returns the per-lattice
        device record buffers (or None).  The caller synchronises."""
        import torch
        bufs = self.record_buffers(n_updates) if records else None
        cur = torch.cuda.current_stream()
        for (ix, cs, th), st, b in zip(self.plan.groups, self.streams, self.batches):
            if not ix:
                continue
            st.wait_stream(cur)
            b.run([self.lattices[i] for i in ix], n_updates,
                  None if bufs is None else [bufs[i] for i in ix], cluster_size=cs,
                  block_threads=th)
        for st in self.streams:
            cur.wait_stream(st)
        return bufs

    def records_numpy(self, bufs, n_updates):
        return [records_to_numpy(b, n_updates) for b in bufs]

    def close(self):
        for b in self.batches:
            b.close()


def candidate_plans(specs):
    """Single-launch plans over all lattices and size-split plans (large
    lattices with bigger teams, concurrently with the small ones)."""
    n = len(specs)
    allix = list(range(n))
    plans = []
    for cs in (1, 2, 4):
        for th in (128, 256, 512):
            plans.append(Plan([(allix, cs, th)], "all cs=%d th=%d" % (cs, th)))
    sizes = np.array([s["L"] ** s["dim"] for s in specs])
    cut = np.quantile(sizes, 0.75) if n else 0
    big = [i for i in allix if sizes[i] >= cut and sizes[i] > 100_000]
    small = [i for i in allix if i not in set(big)]
    if big and small:
        for cs in (2, 4, 8):
            for th in (256, 512):
                plans.append(Plan([(big, cs, th), (small, 1, 256)],
                                  "split big cs=%d th=%d / small cs=1 th=256" % (cs, th)))
    return plans


def _signature(specs, probe_updates):
    import torch
    h = hashlib.sha1(json.dumps([(s["dim"], s["L"], round(s["T"], 6)) for s in specs]).encode())
    return "%s|%s|%d" % (torch.cuda.get_device_name(), h.hexdigest()[:16], probe_updates)


def _cache_path():
    return os.path.join(_build.OUT_DIR, "autotune.json")


def autotune(specs, probe_updates=40, seed_offset=10_000_000, use_cache=True, verbose=False):
    """Times every candidate plan on fresh lattices of the same shapes (other
    seeds) for probe_updates updates each; returns (best Plan, table)."""
    import torch
    sig = _signature(specs, probe_updates)
    cache = {}
    if use_cache and os.path.exists(_cache_path()):
        try:
            with open(_cache_path()) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    plans = candidate_plans(specs)
    if use_cache and sig in cache:
        label = cache[sig]["best"]
        for p in plans:
            if p.label == label:
                return p, cache[sig]["table"]
    table = []
    for k, p in enumerate(plans):
        # every candidate runs the same updates from the same fresh lattices
        lats = [WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"] + seed_offset)
                for s in specs]
        r = BatchedRunner(lats, p)
        # first launches of a team shape (kernel attributes, shared-memory
        # carve-out) happen outside the timing, on two throwaway lattices
        warm = [WolffLattice(2, 8, 2.0, seed=1) for _ in range(2)]
        for _, cs, th in p.groups:
            BatchedRunner(warm, Plan([([0, 1], cs, th)])).run(2, records=False)
        torch.cuda.synchronize()
        for x in warm:
            x.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bufs = r.run(probe_updates, records=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        flips = sum(int(x["C"].astype(np.int64).sum())
                    for x in r.records_numpy(bufs, probe_updates))
        r.close()
        for lat in lats:
            lat.close()
        table.append({"plan": p.label, "seconds": dt, "flips_per_s": flips / dt})
        if verbose:
            print("autotune %-45s %.4g flips/s" % (p.label, flips / dt))
    best = min(range(len(plans)), key=lambda i: table[i]["seconds"])
    if use_cache:
        cache[sig] = {"best": plans[best].label, "table": table}
        os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
        with open(_cache_path(), "w") as f:
            json.dump(cache, f, indent=1)
    return plans[best], table
