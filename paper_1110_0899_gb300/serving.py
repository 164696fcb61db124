"""Serving loop: continuous batching of Wolff-run requests on one GPU.

A request asks for n updates of a fresh lattice (dim, L, T, seed) and gets
back its per-update records (|C|, levels, E_bond, M) and final E, M.  The
server keeps every admitted lattice resident on the device and works in
epochs: at each epoch boundary it admits the requests that have arrived, as
long as their memory (workspace + record buffer) fits the budget, then runs
updates of every active request in shared batched launches -- each request's
share sized from its measured cost per update and capped on the device by a
time budget -- and retires the requests that are done.
Engines: a lattice of at most 64 words runs on the tiny engine (one CTA,
always the faster there); one of up to TINY_MAX_SITES sites runs on whichever
of the tiny and the team engine its own measured cost per update favours
(the team engine first: a fresh lattice's clusters are small; the other one
is timed again every few epochs, since a lattice's clusters grow as it
orders); the rest on the team engine, one thread-block cluster per lattice,
large lattices with larger teams.  Each engine group has its own stream.
Requests that arrive while others are on the GPU therefore join at the next
epoch and their work overlaps on the device.  A request's chain does not
depend on what it shares the GPU with: its records equal those of the same
request run alone.
"""
import collections
import time

import numpy as np

from . import (RECORD_BYTES, SCHED_CLUSTER, SCHED_TINY, TINY_MAX_SITES, WolffBatch, WolffLattice,
               records_to_numpy, wolff_workspace_bytes)


def _tiny_words(dim, L):
    return L ** (dim - 1) * ((L + 31) // 32)


TINY, TEAM = "tiny", "team"


class Request:
    __slots__ = ("spec", "lattice", "records", "done", "admitted_s", "finished_s", "result",
                 "ns_per_update", "quota", "updates_seen", "first_update_s", "engine", "ns_by",
                 "same_engine_epochs")

    def __init__(self, spec):
        self.spec = spec
        self.lattice = None
        self.records = None
        self.done = 0
        self.admitted_s = None
        self.finished_s = None
        self.result = None
        self.ns_per_update = None
        self.quota = 0
        self.updates_seen = 0
        self.first_update_s = None
        self.engine = TEAM
        self.ns_by = {TINY: None, TEAM: None}   # measured ns per update on each engine
        self.same_engine_epochs = 0

    @property
    def remaining(self):
        return self.spec["n_updates"] - self.done

    def memory_bytes(self):
        s = self.spec
        return wolff_workspace_bytes(s["dim"], s["L"]) + s["n_updates"] * RECORD_BYTES


class WolffServer:
    def __init__(self, memory_budget=None, epoch_updates=1 << 20, big_sites=1 << 18,
                 small_team=(1, 256), big_team=(4, 256), max_active=4096, keep_records=True,
                 epoch_seconds=0.02, first_quota=16, tiny=True, reprobe_epochs=8):
        import torch
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget = int(free * 0.6)
        self.memory_budget = int(memory_budget)
        self.epoch_updates = int(epoch_updates)
        self.big_sites = int(big_sites)
        self.small_team = small_team
        self.big_team = big_team
        self.max_active = int(max_active)
        self.keep_records = keep_records
        # each request's share of an epoch is sized from its measured cost per
        # update so that one slow lattice does not hold the others back
        self.epoch_seconds = float(epoch_seconds)
        self.first_quota = int(first_quota)
        # groups: tiny engine (<= 64 words), tiny engine (larger), small
        # teams, large teams -- each on its own stream
        self.tiny = bool(tiny)
        self.reprobe_epochs = int(reprobe_epochs)
        self.engine_epochs = {TINY: 0, TEAM: 0}
        self.streams = [torch.cuda.Stream() for _ in range(4)]
        self.batches = [WolffBatch(max_active, stream=s,
                                   schedule=SCHED_TINY if k < 2 else SCHED_CLUSTER)
                        for k, s in enumerate(self.streams)]

    def _admit(self, req, now):
        import torch
        s = req.spec
        req.lattice = WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"])
        req.records = torch.empty(max(1, s["n_updates"]) * RECORD_BYTES, dtype=torch.uint8,
                                  device="cuda")
        req.admitted_s = now

    def _engine(self, r):
        """The engine for this epoch (see choose_engine)."""
        s = r.spec
        return choose_engine(s["dim"], s["L"], r.ns_by, r.engine, r.same_engine_epochs,
                             self.tiny, self.reprobe_epochs)

    def _quota(self, r):
        if r.ns_per_update is None:
            q = self.first_quota
        else:
            q = int(self.epoch_seconds * 1e9 / max(r.ns_per_update, 1.0))
            # grow at most 4x per epoch: a young lattice's updates get dearer
            # as it orders, faster than one epoch's estimate can follow
            q = min(q, 4 * max(r.quota, 1))
        return max(1, min(q, self.epoch_updates, r.remaining))

    def _epoch(self, active, t0=None):
        import torch
        cur = torch.cuda.current_stream()
        groups = [[], [], [], []]
        for r in active:
            s = r.spec
            eng = self._engine(r)
            r.same_engine_epochs = r.same_engine_epochs + 1 if eng == r.engine else 1
            r.engine = eng
            r.ns_per_update = r.ns_by[eng]
            self.engine_epochs[eng] += 1
            if eng == TINY:
                groups[0 if _tiny_words(s["dim"], s["L"]) <= 64 else 1].append(r)
            else:
                groups[3 if r.lattice.N >= self.big_sites else 2].append(r)
        shapes = ((1, 0), (1, 0), self.small_team, self.big_team)
        for g, (cs, th), st, b in zip(groups, shapes, self.streams, self.batches):
            if not g:
                continue
            st.wait_stream(cur)
            for r in g:
                r.quota = self._quota(r)
            recs = [r.records[r.done * RECORD_BYTES:] for r in g]
            # the device stops each lattice at the first update boundary past
            # twice the epoch target, whatever its quota said
            b.run([r.lattice for r in g], [r.quota for r in g], recs, cluster_size=cs,
                  block_threads=th, budget_ns=int(2 * self.epoch_seconds * 1e9))
        for st in self.streams:
            cur.wait_stream(st)
        torch.cuda.synchronize()
        for r in active:
            st = r.lattice.stats()
            ran = st["updates"] - r.updates_seen
            r.updates_seen = st["updates"]
            dt = max(1, st["end_ns"] - st["start_ns"])
            if ran > 0:
                per = dt / ran
                old = r.ns_by[r.engine]
                r.ns_by[r.engine] = per if old is None else 0.5 * (old + per)
                r.ns_per_update = r.ns_by[r.engine]
            r.quota = max(ran, 1)
            if ran > 0 and r.done == 0 and t0 is not None:
                r.first_update_s = time.perf_counter() - t0
            r.done += ran

    def _retire(self, req, now):
        E, M, C = req.lattice.measure()
        rec = records_to_numpy(req.records, req.spec["n_updates"]) if self.keep_records else None
        req.result = {"E_bond": E, "M": M, "last_C": C, "records": rec,
                      "flips": int(rec["C"].astype(np.int64).sum()) if rec is not None else None}
        req.finished_s = now
        req.lattice.close()
        req.lattice = None
        req.records = None

    def serve(self, trace, time_scale=1.0, max_seconds=None):
        """Runs the trace (arrival_s scaled by time_scale) in real time.
        Returns (requests, summary)."""
        pending = collections.deque(sorted((Request(s) for s in trace),
                                           key=lambda r: r.spec["arrival_s"]))
        everyone = list(pending)
        active = []
        mem_used = 0
        max_backlog = 0
        epochs = 0
        active_per_epoch = []
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            if max_seconds is not None and now > max_seconds:
                break
            while (pending and pending[0].spec["arrival_s"] * time_scale <= now
                   and len(active) < self.max_active
                   and mem_used + pending[0].memory_bytes() <= self.memory_budget):
                r = pending.popleft()
                self._admit(r, now)
                mem_used += r.memory_bytes()
                active.append(r)
            waiting = sum(1 for r in pending if r.spec["arrival_s"] * time_scale <= now)
            max_backlog = max(max_backlog, waiting)
            if not active:
                if pending:
                    delay = pending[0].spec["arrival_s"] * time_scale - now
                    if delay > 0:
                        time.sleep(min(delay, 0.01))
                continue
            active_per_epoch.append(len(active))
            self._epoch(active, t0)
            epochs += 1
            now = time.perf_counter() - t0
            still = []
            for r in active:
                if r.remaining == 0:
                    self._retire(r, now)
                    mem_used -= r.memory_bytes()
                else:
                    still.append(r)
            active = still
        wall = time.perf_counter() - t0
        partial_flips = 0
        for r in active:   # stopped early: count the updates already run
            if r.done:
                partial_flips += int(records_to_numpy(r.records, r.done)["C"].astype(np.int64).sum())
            r.lattice.close()
        done = [r for r in everyone if r.finished_s is not None]
        lat = np.array([r.finished_s - r.spec["arrival_s"] * time_scale for r in done])
        flips = sum(r.result["flips"] or 0 for r in done) + partial_flips
        updates = sum(r.spec["n_updates"] for r in done) + sum(r.done for r in active)
        last_arrival = max((r.spec["arrival_s"] for r in everyone), default=0.0) * time_scale
        # latency over every request: an unfinished one is censored at the end
        # of the window (its latency is at least wall - arrival)
        lat_all = censored_latencies(everyone, wall, time_scale)
        first = np.array([r.first_update_s - r.spec["arrival_s"] * time_scale for r in everyone
                          if r.first_update_s is not None])
        summary = {
            "requests": len(everyone), "completed": len(done), "epochs": epochs,
            "wall_s": wall, "flips": flips, "updates": updates,
            "flips_per_s": flips / wall if wall > 0 else 0.0,
            "updates_per_s": updates / wall if wall > 0 else 0.0,
            "latency_p50_s": None, "latency_p99_s": None,
            "latency_p50_exact": None, "latency_p99_exact": None,
            "completed_latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "completed_latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "first_update_p50_s": float(np.percentile(first, 50)) if len(first) else None,
            "first_update_p99_s": float(np.percentile(first, 99)) if len(first) else None,
            "started": int(len(first)),
            "active_per_epoch_median": (float(np.median(active_per_epoch))
                                        if active_per_epoch else 0.0),
            "active_per_epoch_max": int(max(active_per_epoch, default=0)),
            "max_backlog": max_backlog,
            "offered_span_s": last_arrival,
            "saturated": wall > 1.5 * last_arrival + 1.0,
            "engine_epochs": dict(self.engine_epochs),
        }
        for q in (50, 99):
            v, exact = censored_quantile(lat_all, q / 100.0)
            summary["latency_p%d_s" % q] = v
            summary["latency_p%d_exact" % q] = exact
        return everyone, summary

    def close(self):
        for b in self.batches:
            b.close()


def choose_engine(dim, L, ns_by, current, same_epochs, tiny=True, reprobe_epochs=8):
    """Engine of a request's next epoch: TEAM above TINY_MAX_SITES sites (or
    with the tiny engine off); TINY up to 64 words; otherwise TEAM until it
    has been timed, then TINY once, then the faster by the measured ns per
    update (ns_by), switching to the other for one epoch after
    reprobe_epochs epochs in a row on the same one."""
    if not tiny or L ** dim > TINY_MAX_SITES:
        return TEAM
    if _tiny_words(dim, L) <= 64:
        return TINY
    if ns_by[TEAM] is None:
        return TEAM
    if ns_by[TINY] is None:
        return TINY
    best = TINY if ns_by[TINY] < ns_by[TEAM] else TEAM
    if current == best and same_epochs >= reprobe_epochs:
        return TEAM if best == TINY else TINY
    return best


def censored_latencies(requests, wall, time_scale=1.0):
    """(latency, finished) per request: completion - arrival for a finished
    request, wall - arrival (a lower bound) for one still running or waiting
    when the window ended."""
    out = []
    for r in requests:
        arr = r.spec["arrival_s"] * time_scale
        if r.finished_s is not None:
            out.append((r.finished_s - arr, True))
        else:
            out.append((max(0.0, wall - arr), False))
    return out


def censored_quantile(values, q):
    """Nearest-rank q-quantile of latencies some of which are censored lower
    bounds.  Returns (value, exact): the quantile computed with the bounds in
    place of the unknown latencies; it is exact when the k = ceil(q n)
    smallest entries are all finished requests no larger than every bound
    (then no unknown latency can move below it), else the true quantile is at
    least the value returned."""
    if not values:
        return None, None
    n = len(values)
    k = max(1, int(np.ceil(q * n)))
    srt = sorted(values, key=lambda x: x[0])
    v = float(srt[k - 1][0])
    exact = all(fin for _, fin in srt[:k])
    bounds = [x for x, fin in values if not fin]
    if bounds and v > min(bounds):
        exact = False
    return v, exact
