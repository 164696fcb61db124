"""Batched form: many independent lattices per launch, with an autotuner.

A plan splits the lattices into groups.  A group runs on one of three
schedules:
  - "batched": one persistent launch through a wolff_batch (one
    thread-block cluster per lattice, the C ABI's batched entry point) on the
    group's own CUDA stream, with the group's team shape (cluster size,
    threads per CTA) and window-mode queue (window slots per CTA, growth
    levels per commit round);
  - "tiny": a wolff_batch on the tiny engine (one CTA per lattice of at most
    TINY_MAX_SITES sites, the lattice in shared memory as bit planes) on the
    group's own stream; lattices of at most 64 words and larger ones form
    separate groups, so that each launch has the CTA size its lattices want;
  - "launches": one wolff_step launch per lattice with the library's default
    schedule (the largest thread-block cluster, window mode), on the stream
    the lattices were created on, concurrently with the batched groups.
The autotuner times candidate plans on throw-away copies of the workload
(same shapes and temperatures, other seeds): first the team shapes and the
size split, then, around the best of those, the window slots, the levels
per round, the schedule of the large lattices and the tiny engine for the
lattices it takes.  It caches the winner per
GPU and workload signature.  No plan changes any result: each lattice
follows the chain it would follow alone.
"""
import hashlib
import json
import os
import time

import numpy as np

from . import (RECORD_BYTES, SCHED_TINY, TINY_MAX_SITES, WolffBatch, WolffLattice, _build,
               records_to_numpy, wolff_step)


BATCHED, LAUNCHES, TINY = "batched", "launches", "tiny"
DEFAULT_SLOTS = 64


def tiny_words(dim, L):
    """32-bit words of a lattice's bit planes: (N / L) ceil(L / 32)."""
    return L ** (dim - 1) * ((L + 31) // 32)


def tiny_split(specs, ix):
    """The lattices of ix the tiny engine takes, as (at most 64 words, more),
    and the rest."""
    small, large, rest = [], [], []
    for i in ix:
        s = specs[i]
        if s["L"] ** s["dim"] > TINY_MAX_SITES:
            rest.append(i)
        elif tiny_words(s["dim"], s["L"]) <= 64:
            small.append(i)
        else:
            large.append(i)
    return small, large, rest


class Group:
    """Lattices `ix` on one schedule: BATCHED with team shape (cs, th),
    `slots` window slots per CTA and `levels` growth levels per round (1 =
    the library's default), LAUNCHES (one default launch per lattice), or
    TINY (one CTA per lattice, th threads, 0 = the engine's default)."""

    def __init__(self, ix, cs=1, th=256, slots=DEFAULT_SLOTS, levels=1, kind=BATCHED):
        self.ix, self.cs, self.th = list(ix), int(cs), int(th)
        self.slots, self.levels, self.kind = int(slots), int(levels), kind

    def replace(self, **kw):
        d = dict(ix=self.ix, cs=self.cs, th=self.th, slots=self.slots, levels=self.levels,
                 kind=self.kind)
        d.update(kw)
        return Group(**d)

    def to_json(self):
        if self.kind == LAUNCHES:
            return {"n": len(self.ix), "schedule": LAUNCHES}
        if self.kind == TINY:
            return {"n": len(self.ix), "schedule": TINY,
                    "block_threads": self.th if self.th else "default"}
        return {"n": len(self.ix), "schedule": BATCHED, "cluster_size": self.cs,
                "block_threads": self.th, "window_slots": self.slots,
                "levels_per_round": self.levels if self.levels > 1 else "default"}


class Plan:
    """groups: list of Group (or of (indices, cluster_size, block_threads))."""

    def __init__(self, groups, label=""):
        self.groups = [g if isinstance(g, Group) else Group(*g) for g in groups]
        self.label = label

    def to_json(self):
        return {"label": self.label, "groups": [g.to_json() for g in self.groups]}


class BatchedRunner:
    """Executes a plan over a list of lattices created on the caller's device
    (the lattices of a LAUNCHES group on the stream that is current when
    run() is called)."""

    def __init__(self, lattices, plan):
        import torch
        self.lattices = lattices
        self.plan = plan
        self.streams, self.batches = [], []
        for g in plan.groups:
            if g.kind == BATCHED:
                st = torch.cuda.Stream()
                b = WolffBatch(max(1, len(g.ix)), stream=st)
                b.set_window(g.slots)
                self.streams.append(st)
                self.batches.append(b)
            elif g.kind == TINY:
                st = torch.cuda.Stream()
                self.streams.append(st)
                self.batches.append(WolffBatch(max(1, len(g.ix)), stream=st, schedule=SCHED_TINY))
            else:
                self.streams.append(None)
                self.batches.append(None)
            for i in g.ix:
                lattices[i].set_burst(g.levels if g.kind == BATCHED else 1)
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
        # the batched groups first, each on its stream once the current
        # stream's earlier work is done ...
        for g, st, b in zip(self.plan.groups, self.streams, self.batches):
            if g.kind == LAUNCHES or not g.ix:
                continue
            st.wait_stream(cur)
            b.run([self.lattices[i] for i in g.ix], n_updates,
                  None if bufs is None else [bufs[i] for i in g.ix],
                  cluster_size=1 if g.kind == TINY else g.cs, block_threads=g.th)
        # ... then the per-lattice launches on the current stream, concurrently
        for g in self.plan.groups:
            if g.kind != LAUNCHES:
                continue
            for i in g.ix:
                lat = self.lattices[i]
                if (lat.stream or 0) != (cur.cuda_stream or 0):
                    raise ValueError("a LAUNCHES group needs lattices made on the current stream")
                wolff_step(lat.handle, n_updates, None if bufs is None else bufs[i])
        for st in self.streams:
            if st is not None:
                cur.wait_stream(st)
        return bufs

    def records_numpy(self, bufs, n_updates):
        return [records_to_numpy(b, n_updates) for b in bufs]

    def close(self):
        for b in self.batches:
            if b is not None:
                b.close()


def _size_split(specs):
    n = len(specs)
    allix = list(range(n))
    sizes = np.array([s["L"] ** s["dim"] for s in specs])
    cut = np.quantile(sizes, 0.75) if n else 0
    big = [i for i in allix if sizes[i] >= cut and sizes[i] > 100_000]
    small = [i for i in allix if i not in set(big)]
    return big, small


def candidate_plans(specs):
    """First stage: single-launch plans over all lattices and size-split plans
    (large lattices with bigger teams, concurrently with the small ones)."""
    allix = list(range(len(specs)))
    plans = []
    for cs in (1, 2, 4):
        for th in (128, 256, 512):
            plans.append(Plan([Group(allix, cs, th)], "all cs=%d th=%d" % (cs, th)))
    big, small = _size_split(specs)
    if big and small:
        for cs in (2, 4, 8):
            for th in (256, 512):
                plans.append(Plan([Group(big, cs, th), Group(small, 1, 256)],
                                  "split big cs=%d th=%d / small cs=1 th=256" % (cs, th)))
    return plans


def refine_plans(best, specs):
    """Second stage, around the best first-stage plan: the window-mode queue
    (slots per CTA 32 or 128 instead of 64; 12 or 32 growth levels per round
    instead of the default) and the schedule of the large lattices (one
    default launch each instead of a batched launch)."""
    out = []
    for slots in (32, 128):
        out.append(Plan([g.replace(slots=slots) for g in best.groups],
                        best.label + " / slots=%d" % slots))
    for levels in (12, 32):
        out.append(Plan([g.replace(levels=levels) for g in best.groups],
                        best.label + " / levels=%d" % levels))
    big, small = _size_split(specs)
    if big and small:
        small_g = [g for g in best.groups if set(g.ix) == set(small)]
        small_g = small_g[0] if small_g else Group(small, 1, 256)
        out.append(Plan([Group(big, kind=LAUNCHES), small_g],
                        "big: one default launch each / small: %s" % (
                            "cs=%d th=%d" % (small_g.cs, small_g.th))))
    # the tiny engine for the lattices it takes, the rest as in the best plan
    tw, tl, _ = tiny_split(specs, range(len(specs)))
    if tw or tl:
        taken = set(tw) | set(tl)
        groups = [Group(x, th=0, kind=TINY) for x in (tw, tl) if x]
        for g in best.groups:
            keep = [i for i in g.ix if i not in taken]
            if keep:
                groups.append(g.replace(ix=keep))
        out.append(Plan(groups, best.label + " / tiny engine for %d lattices" % len(taken)))
    return out


def _signature(specs, probe_updates):
    import torch
    h = hashlib.sha1(json.dumps([(s["dim"], s["L"], round(s["T"], 6)) for s in specs]).encode())
    return "%s|%s|%d" % (torch.cuda.get_device_name(), h.hexdigest()[:16], probe_updates)


def _cache_path():
    return os.path.join(_build.OUT_DIR, "autotune.json")


def _time_plan(p, specs, probe_updates, seed_offset):
    import torch
    # every candidate runs the same updates from the same fresh lattices
    lats = [WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"] + seed_offset)
            for s in specs]
    r = None
    try:
        r = BatchedRunner(lats, p)
        # first launches of a team shape (kernel attributes, shared-memory
        # carve-out) happen outside the timing, on two throwaway lattices
        warm = [WolffLattice(2, 8, 2.0, seed=1) for _ in range(2)]
        for g in p.groups:
            if g.kind in (BATCHED, TINY):
                w = BatchedRunner(warm, Plan([g.replace(ix=[0, 1])]))
                w.run(2, records=False)
                torch.cuda.synchronize()
                w.close()
        for x in warm:
            x.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bufs = r.run(probe_updates, records=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        flips = sum(int(x["C"].astype(np.int64).sum())
                    for x in r.records_numpy(bufs, probe_updates))
        return {"plan": p.label, "groups": [g.to_json() for g in p.groups], "seconds": dt,
                "flips_per_s": flips / dt}
    except Exception as e:   # a window that does not fit a team shape, etc.
        torch.cuda.synchronize()
        return {"plan": p.label, "groups": [g.to_json() for g in p.groups], "seconds": None,
                "error": str(e)[:200]}
    finally:
        if r is not None:
            r.close()
        for lat in lats:
            lat.close()


def autotune(specs, probe_updates=40, seed_offset=10_000_000, use_cache=True, verbose=False):
    """Times the candidate plans on fresh lattices of the same shapes (other
    seeds) for probe_updates updates each, in two stages (team shapes and
    size split; then window queue, levels per round and the large lattices'
    schedule around the best); returns (best Plan, table)."""
    sig = _signature(specs, probe_updates)
    cache = {}
    if use_cache and os.path.exists(_cache_path()):
        try:
            with open(_cache_path()) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache and "plan" in cache[sig]:
        return _plan_from_json(cache[sig]["plan"], specs), cache[sig]["table"]
    table, plans = [], []

    def run_stage(cands):
        for p in cands:
            row = _time_plan(p, specs, probe_updates, seed_offset)
            table.append(row)
            plans.append(p)
            if verbose:
                print("autotune %-60s %s" % (p.label, row.get("flips_per_s", row.get("error"))))

    def best_index():
        ok = [i for i in range(len(plans)) if table[i]["seconds"] is not None]
        return min(ok, key=lambda i: table[i]["seconds"])
    run_stage(candidate_plans(specs))
    run_stage(refine_plans(plans[best_index()], specs))
    best = plans[best_index()]
    if use_cache:
        cache[sig] = {"best": best.label, "plan": _plan_to_cache(best), "table": table}
        os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
        with open(_cache_path(), "w") as f:
            json.dump(cache, f, indent=1)
    return best, table


def _plan_to_cache(p):
    return {"label": p.label,
            "groups": [{"ix": g.ix, "cs": g.cs, "th": g.th, "slots": g.slots,
                        "levels": g.levels, "kind": g.kind} for g in p.groups]}


def _plan_from_json(d, specs):
    return Plan([Group(g["ix"], g["cs"], g["th"], g["slots"], g["levels"], g["kind"])
                 for g in d["groups"]], d["label"])
