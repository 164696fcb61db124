"""Benchmark: flipped spins per second of the Wolff single-cluster update.

Default run (N=1), one JSON line:
  - headline: 2D square lattice L = 4096 (16.8M spins), periodic, J = 1,
    T = T_c = 2/ln(1+sqrt 2), int8 spins, Philox random start from seed 2,
    equilibrated for 2000 updates (untimed); every step then runs the 10^4
    measured updates (t = 2000 .. 11999) in one launch (the plain form),
    records written every update (the "+ measurement" form of the paper's
    Tables 1-2).  Before each step the equilibrated lattice is restored
    (untimed), so every step repeats the same chain and must give the same
    records;
  - "3d": the same for the simple-cubic L = 256 lattice at T = 4.5115, seed 3;
  - "batched": 512 2D replicas (L in {64..1024}, T in [2.0, 2.6], seeds
    1000+i), 10^4 updates each through the autotuned batched plan, against
    the same replicas one lattice per launch, records compared;
  - "served": the 200-request Poisson trace through the continuous-batching
    server for a bounded window, latency percentiles over every request
    (unfinished ones censored at the window's end);
  - "small": 2D L=16, seed 1, the whole 10^4-update run on the GPU and by
    the oracle, records compared.

value = sum of cluster sizes over the timed updates / device time of the
timed steps (CUDA events on the lattice's stream, an L2 flush of 256 MB
between steps, outside the events).  With torchrun (N > 1) every rank runs its
own independent lattice (seed + rank): replicas only, no collective on the
data path; value = all ranks' flips / the slowest rank's time.

--impl reference times the CPU oracle (single-threaded C) on the host cores:
each step is the same 10^4 measured updates with their records.
"""
import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "flipped spins/s at Tc (2D L=4096, 3D L=256); batched/served vs plain, p50/p99"
UNIT = "flipped spins/s"
# algorithmic bytes per flipped spin of the int8 layout: frontier write+read
# (8 B), the 2D neighbour spin reads (4 B in 2D, 6 B in 3D), the claim's
# read-modify-write (2 B), and the energy/unmark pass (list re-read 4 B,
# neighbour re-read 2D B, mark write 1 B)
ALGO_BYTES_PER_FLIP = {2: 23.0, 3: 27.0}

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))
# Counters of one timed k_team launch of the specified workloads from the
# committed ncu captures (profiles/k_team_2d_L4096_random_start.md and
# profiles/k_team_3d_L256_random_start.md), valid only while the sources of
# k_team hash to the captured value: DRAM bytes (dram__bytes_read.sum +
# dram__bytes_write.sum), L2 bytes (lts__t_bytes.sum) and the fmaheavy pipe
# (IMAD) activity.
# imad: the fmaheavy pipe (integer multiply-add, the Philox arithmetic) busy
# cycles over its peak (4 per SM-cycle), on the SMs the launch kept active and
# over the whole GPU, and its warp instructions per launch.
TRAFFIC_CAPTURES = {
    ("2d", 10000): {"src": "8f06b8d9d2d9", "bytes_per_launch": 13881088 + 2304,
                    "l2_bytes_per_launch": 78064736,
                    "imad": {"pipe_frac_active_sms": 11261724 / (4 * 59805320),
                             "pipe_frac_gpu": 11261724 / (4 * 105197348),
                             "warp_insts": 4664428}},
    # 84 MB of the 3D launch's DRAM bytes are its first window's prefetch of
    # the lattice and the cluster list into L2
    ("3d", 10000): {"src": "8f06b8d9d2d9", "bytes_per_launch": 86614784 + 828416,
                    "l2_bytes_per_launch": 254802688,
                    "imad": {"pipe_frac_active_sms": 13794552 / (4 * 73513989),
                             "pipe_frac_gpu": 13794552 / (4 * 157390900),
                             "warp_insts": 5733166}},
}


# the sources the cluster-schedule kernel k_team is built from
TEAM_SOURCES = ("wolff_device.cuh", "wolff_internal.h", "wolff_team.cu")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    for name in TEAM_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1110_0899_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


WORKLOADS = {
    # the configurations as specified: random start, 2000 equilibration updates
    "2d": dict(dim=2, L=4096, T=TC2, seed=2, equil=2000, start="random", updates=10000),
    "3d": dict(dim=3, L=256, T=4.5115, seed=3, equil=2000, start="random", updates=10000),
    # the same lattices at equilibrium (ordered start, which the cluster
    # update equilibrates quickly at T_c), where clusters are large
    "2d-eq": dict(dim=2, L=4096, T=TC2, seed=2, equil=1000, start="ordered"),
    "3d-eq": dict(dim=3, L=256, T=4.5115, seed=3, equil=1000, start="ordered"),
    # q = 3 Potts (the extension named in section 6) at its exact 2D critical
    # point T_c = 1 / ln(1 + sqrt 3), J = 1
    "potts3-2d": dict(dim=2, L=2048, T=1.0 / math.log(1.0 + math.sqrt(3.0)), seed=4, equil=1000,
                      start="ordered", q=3),
    # XY embedded-cluster update (the other extension section 6 names): 15-bit
    # angles, 2D near the BKT temperature 0.8929, 3D near its critical 2.2017
    "xy-2d": dict(dim=2, L=1024, T=0.89, seed=6, equil=200, start="ordered", model="xy"),
    "xy-3d": dict(dim=3, L=128, T=2.2, seed=7, equil=200, start="ordered", model="xy"),
}
# algorithmic bytes per flipped XY site (32-bit words): own word 4, 2D
# neighbour words, claim read-modify-write 8, list write + read 8, boundary
# pass re-reading 2D neighbour words and the list entry 4, reflected word 4
XY_ALGO_BYTES_PER_FLIP = {2: 60.0, 3: 76.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="2d",
                    choices=sorted(WORKLOADS) + ["batched", "served", "binder", "small",
                                                "tiny-sizes"])
    ap.add_argument("--sizes", default=None,
                    help="tiny-sizes: dim:L pairs, comma separated (default: 2D L 16..181, "
                         "3D L 4..32)")
    ap.add_argument("--temps", default="0.9,1.0,1.1",
                    help="tiny-sizes: temperatures as fractions of T_c")
    ap.add_argument("--regimes", default="random,equil",
                    help="tiny-sizes: random (fresh lattice) and/or equil (after updates)")
    ap.add_argument("--updates-per-step", type=int, default=None,
                    help="updates per step (default: the workload's measured run, "
                         "10^4 for 2d and 3d, else 1000)")
    ap.add_argument("--equil", type=int, default=None)
    ap.add_argument("--schedule", default="auto",
                    choices=["auto", "persistent", "graph", "cluster"])
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--t-up", type=int, default=None,
                    help="leader hands wave fronts above this size to all CTAs")
    ap.add_argument("--t-down", type=int, default=None)
    ap.add_argument("--levels", type=int, default=None,
                    help="window mode: growth levels per commit round (0 = window mode off)")
    ap.add_argument("--helpers", type=int, default=None,
                    help="pre-growing helper teams of the cluster schedule (-1 = as many as "
                         "fit, 0 = none)")
    ap.add_argument("--cpu-seconds", type=float, default=5.0,
                    help="bound of the oracle's full-recount sample timed beside the GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=120.0)
    ap.add_argument("--no-3d", action="store_true",
                    help="skip the 3D L=256 object in the default line")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-plain comparison in the default line")
    ap.add_argument("--batched-updates", type=int, default=10000,
                    help="updates per replica of the batched comparison")
    ap.add_argument("--plain-every", type=int, default=8,
                    help="the default line's batched comparison runs its plain arm on every "
                         "k-th replica (--workload batched runs all)")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the serving run in the default line")
    ap.add_argument("--no-l2-probe", action="store_true")
    ap.add_argument("--epoch-ms", type=float, default=20.0,
                    help="served form: device time per epoch the server aims at")
    ap.add_argument("--no-tiny-engine", action="store_true",
                    help="served form: run every lattice on the team engine (no tiny engine)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small configuration (2D L=16) in the default line")
    ap.add_argument("--embed-serve-seconds", type=float, default=30.0)
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def cpu_description():
    """The host CPU: model name (lscpu) and the cores the OS reports."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(base_seed, rank):
    """Replicas only: every rank runs its own lattice, seeded base + rank."""
    return base_seed + rank


def aggregate_ranks(total_ms, flips, device):
    """Whole-job numbers over the ranks: the slowest rank's time and the sum
    of all ranks' flipped spins (the only collective, on the host path)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ff = torch.tensor([float(flips)], dtype=torch.float64, device=device)
    dist.all_reduce(ff, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ff.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_step_times(wl, steps, warmup):
    """The oracle on the workload's measured run: the lattice after its own
    equilibration (untimed), then every step replays the 10^4 measured
    updates with their records (the local-recount form, the records the GPU
    writes) from a restored copy; E_bond and M of the start are counted once,
    untimed, as the GPU's restore does."""
    import numpy as np

    import oracle
    dim, L, T, seed, equil = wl["dim"], wl["L"], wl["T"], wl["seed"], wl["equil"]
    U = wl["updates"]
    thr = oracle.bond_threshold(1.0, T)
    s0 = oracle.init_lattice(dim, L, seed)
    oracle.run(dim, L, thr, seed, 0, equil, s0, records=False)
    em0 = np.array([oracle.energy_bond(dim, L, s0), oracle.magnetisation(dim, L, s0)], np.int64)
    times, flips = [], []
    for k in range(warmup + steps):
        s, em = s0.copy(), em0.copy()
        t0 = time.perf_counter()
        rec = oracle.run_local(dim, L, thr, seed, equil, U, s, em)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
            flips.append(int(rec["C"].astype(np.int64).sum()))
    return times, flips


def run_reference(args):
    """CPU oracle on the host cores, the same workload as the GPU arm."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    if args.workload not in ("2d", "3d"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm times the specified 2d and 3d workloads"}))
        return

    def line_for(name):
        wl = WORKLOADS[name]
        times, flips = reference_step_times(wl, args.steps, args.warmup)
        value = sum(flips) / sum(times)
        cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d steps, each the %d measured updates (t = %d .. %d) with records, "
                         "from the oracle's own equilibrated lattice"
                         % (args.steps, wl["updates"], wl["equil"],
                            wl["equil"] + wl["updates"] - 1)}
        cpu.update(cpu_description())
        return {
            "value": value, "ms_per_step": 1000.0 * sum(times) / len(times),
            "config": {"workload": "%dD L=%d T=%.6g seed %d, oracle equilibrated %d updates, "
                                   "per step the %d measured updates with records"
                                   % (wl["dim"], wl["L"], wl["T"], wl["seed"], wl["equil"],
                                      wl["updates"]),
                       "dim": wl["dim"], "L": wl["L"], "T": wl["T"], "seed": wl["seed"]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
    main_part = line_for(args.workload)
    line = {
        "impl": "reference", "metric": METRIC, "value": main_part["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_part["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": main_part["config"], "cpu_baseline": main_part["cpu_baseline"],
        "e2e": main_part["e2e"],
    }
    if args.workload == "2d" and not args.no_3d:
        line["3d"] = line_for("3d")
    print(json.dumps(line), flush=True)


def l2_probe(sizes_mb=(16, 32, 64), passes=200):
    """L2 bandwidth, measured with the library's probe kernel: a buffer that
    fits in L2 streamed `passes` times in one launch (16-byte loads that skip
    L1), CUDA events around the launch after a warm-up launch; the best of
    three per size.  Returns GB/s figures."""
    import torch

    import paper_1110_0899_gb300 as w
    out = {"read_gbs_by_mb": {}, "rmw_gbs_by_mb": {}}
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for mode, key in ((0, "read_gbs_by_mb"), (1, "rmw_gbs_by_mb")):
        for mb in sizes_mb:
            buf = torch.zeros(mb << 20, dtype=torch.uint8, device="cuda")
            w.wolff_l2_probe(buf, 2, mode, sink, stream)
            best = None
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                w.wolff_l2_probe(buf, passes, mode, sink, stream)
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b)
                gbs = (2 if mode else 1) * passes * buf.numel() / (ms / 1000.0) / 1e9
                best = gbs if best is None else max(best, gbs)
            out[key][str(mb)] = best
            del buf
    out["read_gbs"] = max(out["read_gbs_by_mb"].values())
    out["rmw_gbs"] = max(out["rmw_gbs_by_mb"].values())
    out["how"] = ("library L2 probe: %s MB buffers streamed %d times per launch by a "
                  "full-occupancy grid, 16-byte ld.global.cg, best of 3 launches after a warm-up"
                  % ("/".join(str(m) for m in sizes_mb), passes))
    return out


def ising_cpu_baseline(wl, gpu_records, full_seconds):
    """The oracle (single-threaded C) on the workload, in the paper's two
    columns (section 5, Tables 1-2): "update" -- the 10^4 measured updates
    alone, no observables (the whole run, repeated for at least a second) --
    and "+ measurement" -- E_bond and M recounted from their definitions
    after every update, as the paper's CPU code does (a bounded sample of
    the same run).  Between them: the same updates with the records the GPU
    writes, kept by the oracle's local recount.  The oracle starts from its
    own equilibrated lattice; its records of the measured run are compared
    with the GPU's."""
    import numpy as np

    import oracle
    dim, L, T, seed, equil, U = wl["dim"], wl["L"], wl["T"], wl["seed"], wl["equil"], wl["updates"]
    thr = oracle.bond_threshold(1.0, T)
    s0 = oracle.init_lattice(dim, L, seed)
    oracle.run(dim, L, thr, seed, 0, equil, s0, records=False)
    em0 = np.array([oracle.energy_bond(dim, L, s0), oracle.magnetisation(dim, L, s0)], np.int64)
    s, em = s0.copy(), em0.copy()
    t0 = time.perf_counter()
    ref = oracle.run_local(dim, L, thr, seed, equil, U, s, em)
    t_rec = time.perf_counter() - t0
    flips = int(ref["C"].astype(np.int64).sum())
    reps, t_upd = 0, 0.0
    while reps < 3 or t_upd < 1.0:
        s = s0.copy()
        t0 = time.perf_counter()
        oracle.run(dim, L, thr, seed, equil, U, s, records=False)
        t_upd += time.perf_counter() - t0
        reps += 1
    s, n, f_full, t_full = s0.copy(), 0, 0, 0.0
    while t_full < full_seconds and n < U:
        t0 = time.perf_counter()
        r = oracle.run(dim, L, thr, seed, equil + n, 1, s)
        t_full += time.perf_counter() - t0
        f_full += int(r["C"][0])
        n += 1
    upd = reps * flips / t_upd
    out = {"value": upd, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "update only: the whole measured run (%d updates, t = %d .. %d) from the "
                     "oracle's own equilibrated lattice, %d times, %.2f s of one core"
                     % (U, equil, equil + U - 1, reps, t_upd),
           "update_only": upd,
           "update_and_records": flips / t_rec,
           "update_and_full_recount": f_full / t_full if t_full > 0 else None,
           "full_recount_sample": "%d updates from t = %d, %.1f s of one core" % (n, equil, t_full),
           "records_equal_gpu": (bool(np.array_equal(gpu_records, ref))
                                 if gpu_records is not None else None)}
    out.update(cpu_description())
    return out


def run_batched(args, n_replicas=512, updates=None, embed=False, plain_every=1):
    """512 independent 2D replicas (L in {64..1024}, T in [2.0, 2.6], seeds
    1000+i) through the autotuned batched plan, against the same replicas run
    one lattice per launch with the library's default settings.  Both arms
    run the same updates from the same random starts, so their records must
    agree bit for bit.  plain_every = k > 1 runs the plain arm on every k-th
    replica only (a stratified sample of the same table: one lattice per
    launch takes minutes at 10^4 updates per replica), its throughput the
    sample's flips over the sample's time."""
    import numpy as np
    import torch

    import paper_1110_0899_gb300 as w
    from paper_1110_0899_gb300 import batched, workloads
    torch.cuda.set_device(0)
    U = updates or args.updates_per_step or 1000
    specs = workloads.batched_replicas(n_replicas)
    t_tune = time.perf_counter()
    plan, table = batched.autotune(specs, probe_updates=max(10, U // 4))
    t_tune = time.perf_counter() - t_tune
    lat_b = [w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"]) for s in specs]
    runner = batched.BatchedRunner(lat_b, plan)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    recs_b, lat_ms = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record()
        bufs = runner.run(U)
        ev[k][1].record()
        torch.cuda.synchronize()
        recs_b.append([r for r in runner.records_numpy(bufs, U)])
        st = [x.stats() for x in lat_b]
        t_start = min(x["start_ns"] for x in st)
        lat_ms.extend((x["end_ns"] - t_start) / 1e6 for x in st)
    t_b = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    flips_b = sum(int(r["C"].astype(np.int64).sum()) for step in recs_b for r in step)
    runner.close()
    for x in lat_b:
        x.close()
    # plain: one lattice per launch (the library's default schedule), the same
    # updates; a sample takes every k-th replica in (L, T) order (strata of
    # size and temperature, which set a replica's cost)
    order = sorted(range(n_replicas), key=lambda i: (specs[i]["L"], specs[i]["T"]))
    k = max(1, plain_every)
    plain_ix = sorted(order[k // 2::k]) if k > 1 else list(range(n_replicas))
    lat_p = [w.WolffLattice(specs[i]["dim"], specs[i]["L"], specs[i]["T"], seed=specs[i]["seed"])
             for i in plain_ix]
    bufs_p = [x.record_buffer(U) for x in lat_p]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    same = True
    flips_p = 0
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record()
        for x, b in zip(lat_p, bufs_p):
            w.wolff_step(x.handle, U, b)
        ev[k][1].record()
        torch.cuda.synchronize()
        for i, x, b in zip(plain_ix, lat_p, bufs_p):
            r = w.records_to_numpy(b, U)
            flips_p += int(r["C"].astype(np.int64).sum())
            same = same and np.array_equal(r, recs_b[k][i])
    t_p = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    plain_scheds = {}
    for x in lat_p:
        inf = x.info()
        key = ("tiny (one CTA of %d threads)" % inf["block_threads"]
               if inf["schedule"] == w.SCHED_TINY else
               "cluster (%d CTAs x %d threads)" % (inf["grid_blocks"], inf["block_threads"]))
        plain_scheds[key] = plain_scheds.get(key, 0) + 1
    for x in lat_p:
        x.close()
    out = {
        "workload": "%d 2D replicas, L in {64..1024}, T in [2.0, 2.6], seeds 1000+i, "
                    "%d x %d updates each" % (n_replicas, args.steps, U),
        "updates_per_replica": U * args.steps,
        "batched_flips_per_s": flips_b / t_b, "plain_flips_per_s": flips_p / t_p,
        "speedup": (flips_b / t_b) / (flips_p / t_p),
        "batched_s": t_b, "plain_s": t_p, "records_identical": bool(same),
        "replica_latency_ms_p50": float(np.percentile(lat_ms, 50)),
        "replica_latency_ms_p99": float(np.percentile(lat_ms, 99)),
        "plan": plan.to_json(), "autotune_s": t_tune, "autotune": table,
        "plain_form": "one wolff_step launch per lattice, the library's default schedule: " +
                      ", ".join("%s for %d" % (k, v) for k, v in sorted(plain_scheds.items())),
        "plain_sample": ("all %d replicas" % n_replicas if len(plain_ix) == n_replicas else
                         "every %d-th replica in (L, T) order (%d of %d), the full %d updates "
                         "each; records compared with the batched arm's for those" % (
                             plain_every, len(plain_ix), n_replicas, U)),
    }
    if embed:
        return out
    print(json.dumps({"metric": METRIC, "value": out["batched_flips_per_s"], "unit": UNIT,
                      "n_gpus": 1, "steps": args.steps, "warmup": 0, "higher_is_better": True,
                      "config": {"workload": out["workload"]}, "batched": out}), flush=True)


def run_served(args, n_requests=200, embed=False):
    """Poisson stream of Wolff-run requests (the 200-request trace at 200
    req/s) through the continuous-batching server."""
    import torch

    from paper_1110_0899_gb300 import serving, workloads
    torch.cuda.set_device(0)
    trace = workloads.serving_trace(n_requests)
    srv = serving.WolffServer(keep_records=True, tiny=not getattr(args, "no_tiny_engine", False),
                              epoch_seconds=getattr(args, "epoch_ms", 20.0) / 1000.0)
    reqs, summary = srv.serve(trace, max_seconds=args.serve_seconds)
    srv.close()
    summary["workload"] = ("%d requests, Poisson 200 req/s, 70%% 2D L 32..2048, 30%% 3D L 16..128, "
                           "T in [0.9, 1.1] Tc, 1e3..1e5 updates; latency percentiles over every "
                           "request, unfinished ones censored at the window's end (exact=false "
                           "marks a lower bound)" % n_requests)
    if embed:
        return summary
    print(json.dumps({"metric": METRIC, "value": summary["flips_per_s"], "unit": UNIT,
                      "n_gpus": 1, "higher_is_better": True,
                      "config": {"workload": summary["workload"]}, "served": summary}), flush=True)


def run_binder(args):
    """Temperature sweep of the Binder ratio on the batched form (section 5,
    Fig. 2 of the paper): 2D L in {64, 128, 256} with 5000 discarded and 50000
    measured updates per point, 3D L in {16, 32} with 10000 + 100000."""
    import time as _time

    import torch

    from paper_1110_0899_gb300 import binder, workloads
    torch.cuda.set_device(0)
    out = {}
    for dim, Ls, tc, disc, meas in ((2, [64, 128, 256], workloads.TC_2D, 5000, 50_000),
                                    (3, [16, 32], workloads.TC_3D, 10_000, 100_000)):
        Ts = [tc * f for f in (0.97, 0.98, 0.99, 1.0, 1.01, 1.02, 1.03)]
        t0 = _time.perf_counter()
        pts = binder.sweep(dim, Ls, Ts, disc, meas, chunk=5000)
        wall = _time.perf_counter() - t0
        flips = sum(p["mean_cluster"] * p["updates"] for p in pts)
        out["%dd" % dim] = {
            "points": pts, "wall_s": wall, "flips_per_s": flips / wall,
            "crossings": {"%d-%d" % (a, b): binder.crossing(pts, a, b)
                          for a, b in zip(Ls, Ls[1:])},
            "tc": tc}
    print(json.dumps({"metric": "Binder ratio sweep", "binder": out}), flush=True)


def potts_cpu_baseline(dim, L, q, T, seed, spins, t, seconds):
    """The Potts oracle from the GPU's equilibrated lattice, one update at a
    time until `seconds` of CPU work have run."""
    import numpy as np

    import oracle
    thr = oracle.potts_threshold(1.0, T)
    s = np.array(spins, dtype=np.int8, copy=True)
    flips, spent, n = 0, 0.0, 0
    while spent < seconds and n < 1000:
        t0 = time.perf_counter()
        rec = oracle.potts_run(dim, L, q, thr, seed, t + n, 1, s)
        spent += time.perf_counter() - t0
        flips += int(rec["C"][0])
        n += 1
    out = {"value": flips / spent, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d updates from the GPU's equilibrated lattice (t=%d), %.1f s of one core"
                     % (n, t, spent)}
    out.update(cpu_description())
    return out


def run_xy(args):
    """One XY lattice per launch: the same timing contract as the Ising
    workloads (L2 flush between steps, CUDA events on the lattice's stream,
    clocks sampled, e2e through host buffers, the oracle as CPU baseline)."""
    import numpy as np
    import torch

    import paper_1110_0899_gb300 as w
    world, rank, local = dist_setup(args)
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    dim, L, T = wl["dim"], wl["L"], wl["T"]
    seed = rank_seed(wl["seed"], rank)
    equil = wl["equil"] if args.equil is None else args.equil
    U = args.updates_per_step or wl.get("updates", 1000)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = w.WolffXY(dim, L, T, seed=seed, stream=stream, grid_blocks=args.blocks,
                        block_threads=args.threads)
        info = lat.info()
        lat.set_state(np.zeros(lat.N, np.uint16), 0)
        done = 0
        while done < equil:
            k = min(100, equil - done)
            lat.step(k, records=False)
            done += k
        rec_buf = lat.record_buffer(U)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            w.wolff_step(lat.handle, U, rec_buf)
        torch.cuda.synchronize()
        # the e2e leg re-runs, from this snapshot, the updates of the first timed step
        snap, t_snap = lat.get_state()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        recs = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.5)   # the sampler's start-up stays out of the timed steps
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            w.wolff_step(lat.handle, U, rec_buf)
            ends[k].record(stream)
            recs.append(rec_buf[: U * w.XY_RECORD_BYTES].clone())
        torch.cuda.synchronize()
        clk = clocks.stop()
        if world > 1:
            torch.distributed.barrier()
        total_ms = float(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
        records = np.concatenate([r.cpu().numpy().view(w.XY_RECORD_DTYPE) for r in recs])
        flips = int(records["C"].astype(np.int64).sum())
        if world > 1:
            total_ms_all, flips_all = aggregate_ranks(total_ms, flips, "cuda")
        else:
            total_ms_all, flips_all = total_ms, float(flips)
        value = flips_all / (total_ms_all / 1000.0)
        e2e = None
        if not args.no_e2e:
            # the public API end to end: upload the snapshot, run U recorded
            # updates, read the records back
            pinned = torch.empty(lat.N, dtype=torch.int16, pin_memory=True)
            pinned.numpy().view(np.uint16)[:] = snap
            snap_in = pinned.numpy().view(np.uint16)
            e_flips, e_s = 0, 0.0
            lat.set_state(snap_in, t_snap)   # untimed warm-up call
            lat.step(U)
            for k in range(max(3, min(args.steps, 5))):
                t0 = time.perf_counter()
                lat.set_state(snap_in, t_snap)
                r = lat.step(U)
                e_s += time.perf_counter() - t0
                e_flips += int(r["C"].astype(np.int64).sum())
            e2e = {"value": e_flips / e_s, "unit": UNIT, "h2d_bytes_per_step": int(2 * lat.N),
                   "d2h_bytes_per_step": int(U * w.XY_RECORD_BYTES)}
    lat.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, peak_kind = measured_peaks()
    achieved = XY_ALGO_BYTES_PER_FLIP[dim] * (flips / args.steps) / (total_ms / args.steps / 1000.0) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_kind": peak_kind,
            "kernel": "k_xy_team<%d>" % dim}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = xy_cpu_baseline(dim, L, T, seed, snap, t_snap, args.cpu_seconds)
    warm = 1 if L ** dim >= (1 << 22) else 0   # the XY path's L2 warm-up kernel
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16 angles, i64 fixed point, f64 bond test", "data": "synthetic",
        "config": {"workload": "XY %dD L=%d T=%.6g J=1 seed %d, 15-bit angles, %s start, %d "
                               "equilibration + %d x %d recorded updates, one lattice per launch"
                               % (dim, L, T, seed, wl["start"], equil, args.steps, U),
                   "dim": dim, "L": L, "T": T, "seed": seed, "updates_per_step": U,
                   "schedule": "cluster", "grid_blocks": info["grid_blocks"],
                   "block_threads": info["block_threads"],
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": "replicas x%d" % world},
        "e2e": e2e, "gpu_launches": args.steps * (1 + warm), "roofline": roof,
        "cpu_baseline": cpu, "clocks": clk,
        "detail": {"mean_cluster": flips / len(records),
                   "mean_levels": float(records["levels"].mean()),
                   "max_levels": int(records["levels"].max()),
                   "ms_per_update": total_ms / len(records)},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def xy_cpu_baseline(dim, L, T, seed, theta, t, seconds):
    """The XY oracle from the GPU's equilibrated lattice, one update at a
    time until `seconds` of CPU work have run."""
    import numpy as np

    import oracle
    kk = oracle.xy_coupling(1.0, T)
    th = np.array(theta, dtype=np.uint16, copy=True)
    flips, spent, n = 0, 0.0, 0
    while spent < seconds and n < 1000:
        t0 = time.perf_counter()
        rec = oracle.xy_run(dim, L, oracle.XY_ANGLE_BITS, kk, seed, t + n, 1, th)
        spent += time.perf_counter() - t0
        flips += int(rec["C"][0])
        n += 1
    out = {"value": flips / spent, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d updates from the GPU's equilibrated lattice (t=%d), %.1f s of one core"
                     % (n, t, spent)}
    out.update(cpu_description())
    return out


def run_ising(args, name, stream_clocks=True):
    """One Ising (or Potts) lattice per launch on workload `name`; returns the
    bench line (not printed)."""
    import numpy as np
    import torch

    import paper_1110_0899_gb300 as w
    world, rank, local = dist_setup(args)
    wl = WORKLOADS[name]
    dim, L, T = wl["dim"], wl["L"], wl["T"]
    seed = rank_seed(wl["seed"], rank)
    equil = wl["equil"] if args.equil is None else args.equil
    U = args.updates_per_step or wl.get("updates", 1000)
    sched = {"auto": w.SCHED_AUTO, "persistent": w.SCHED_PERSISTENT, "graph": w.SCHED_GRAPH,
             "cluster": w.SCHED_CLUSTER}[args.schedule]

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = w.WolffLattice(dim, L, T, seed=seed, stream=stream, q=wl.get("q"))
        lat.set_schedule(sched, args.blocks, args.threads)
        if args.t_up is not None:
            lat.set_local_thresholds(args.t_up, args.t_down if args.t_down is not None
                                     else args.t_up // 2)
        if args.levels is not None:
            lat.set_burst(args.levels)
        if args.helpers is not None:
            lat.set_helpers(args.helpers)
        info = lat.info()
        if wl["start"] == "ordered":
            lat.set_state(np.zeros(lat.N, dtype=np.int8) if wl.get("q") else
                          np.ones(lat.N, dtype=np.int8), 0)
        rec_buf = lat.record_buffer(U)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        # equilibration (untimed)
        done = 0
        while done < equil:
            k = min(1000, equil - done)
            lat.step(k, records=False)
            done += k
        torch.cuda.synchronize()
        snap, t_snap = lat.get_state()
        if wl.get("q"):
            def restore():
                lat.set_state(snap, t_snap)
        else:
            snap_bits = w.pack_spins(snap)

            def restore():   # 2.1 MB upload of the equilibrated lattice, untimed
                lat.set_state_bits(snap_bits, t_snap)
        # warm-up steps
        for _ in range(args.warmup):
            restore()
            w.wolff_step(lat.handle, U, rec_buf)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        recs = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.5)   # the sampler's start-up stays out of the timed steps
        for k in range(args.steps):
            restore()
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            w.wolff_step(lat.handle, U, rec_buf)
            ends[k].record(stream)
            recs.append(rec_buf[: U * w.RECORD_BYTES].clone())
        torch.cuda.synchronize()
        clk = clocks.stop()
        # the kernel's counters over one more (untimed) step: restoring the
        # lattice resets them
        restore()
        stats0 = lat.stats()
        w.wolff_step(lat.handle, U, rec_buf)
        stats1 = lat.stats()
        if world > 1:
            torch.distributed.barrier()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        step_recs = [r.cpu().numpy().view(w.RECORD_DTYPE) for r in recs]
        # every step ran the same updates from the same lattice
        repeat_identical = all(np.array_equal(step_recs[0], r) for r in step_recs[1:])
        records = np.concatenate(step_recs)
        flips = int(records["C"].astype(np.int64).sum())
        total_ms = float(sum(step_ms))
        levels = records["levels"].astype(np.int64)
        if world > 1:
            total_ms_all, flips_all = aggregate_ranks(total_ms, flips, "cuda")
        else:
            total_ms_all, flips_all = total_ms, float(flips)
        value = flips_all / (total_ms_all / 1000.0)

        # end to end through the host-buffer entry point: upload the
        # equilibrated lattice, run U recorded updates, read the records back
        e2e = None
        if not args.no_e2e and not wl.get("q"):
            # the input lattice, bit-packed (one bit per site), in pinned host memory
            packed = w.pack_spins(snap)
            pinned = torch.empty(packed.size, dtype=torch.int32, pin_memory=True)
            pinned.numpy().view(np.uint32)[:] = packed
            snap_in = pinned.numpy().view(np.uint32)
            # the records land in a caller-owned pinned buffer (a direct copy)
            rec_pinned = torch.empty(U * w.RECORD_BYTES, dtype=torch.uint8, pin_memory=True)
            rec_out = rec_pinned.numpy().view(w.RECORD_DTYPE)
            e2e_flips, e2e_s = 0, 0.0
            # untimed warm-up calls, as for the device timing: the first call
            # allocates the device staging buffer of the records
            for k in range(max(1, min(args.warmup, 3))):
                lat.run_host_bits(U, bits_in=snap_in, t_in=t_snap, records=True, bits_out=False,
                                  records_out=rec_out)
            for k in range(max(3, min(args.steps, 10))):
                t0 = time.perf_counter()
                r, _ = lat.run_host_bits(U, bits_in=snap_in, t_in=t_snap, records=True,
                                         bits_out=False, records_out=rec_out)
                e2e_s += time.perf_counter() - t0
                e2e_flips += int(r["C"].astype(np.int64).sum())
                repeat_identical = repeat_identical and np.array_equal(r, step_recs[0])
            e2e = {"value": e2e_flips / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(snap_in.nbytes),
                   "d2h_bytes_per_step": int(U * w.RECORD_BYTES),
                   "returns": "the %d records (|C|, levels, E_bond, M); the lattice stays on "
                              "the device" % U}
    lat.close()
    peaks, peak_kind = measured_peaks()
    per_launch_flips = flips / args.steps
    avg_launch_s = total_ms / args.steps / 1000.0
    achieved = ALGO_BYTES_PER_FLIP[dim] * per_launch_flips / avg_launch_s / 1e9
    cap = TRAFFIC_CAPTURES.get((name, U))
    fresh = bool(cap and args.schedule in ("auto", "cluster") and not wl.get("q")
                 and kernel_source_hash() == cap["src"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "traffic": cap["bytes_per_launch"] if fresh else None,
            "peak_kind": peak_kind,
            "kernel": {"persistent": "k_persistent<%d>", "graph": "k_graph_level<%d>",
                       "cluster": "k_team<%d>", "auto": "k_team<%d>"}[args.schedule] % dim}
    if fresh and "l2_bytes_per_launch" in cap:
        roof["l2_traffic"] = cap["l2_bytes_per_launch"]
    if fresh and "imad" in cap:
        roof["imad"] = dict(cap["imad"])
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        if wl.get("q"):
            cpu = potts_cpu_baseline(dim, L, wl["q"], T, seed, snap, t_snap, args.cpu_seconds)
        elif name in ("2d", "3d") and U == wl["updates"] and equil == wl["equil"]:
            cpu = ising_cpu_baseline(wl, step_recs[0], args.cpu_seconds)
    # kernels per step: an L2 warm-up for lattices of 2^22 sites or more
    # (except on the Ising cluster path), the persistent schedule's pre-launch
    # reset, the update kernel (or, for the graph schedule, one call kernel and
    # levels + 3 nodes per update)
    warm = 1 if L ** dim >= (1 << 22) and (wl.get("q") or args.schedule in
                                            ("persistent", "graph")) else 0
    if args.schedule == "graph":
        launches = int(args.steps * (1 + warm) + (levels + 3).sum())
    elif args.schedule == "persistent":
        launches = args.steps * (2 + warm)
    else:
        launches = args.steps * (1 + warm)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": {"workload": "%s%dD L=%d T=%.6g J=1 seed %d, %s start, %d equilibration "
                               "updates, then per step the next %d recorded updates in one "
                               "launch from the restored equilibrated lattice"
                               % ("q=%d Potts, " % wl["q"] if wl.get("q") else "", dim, L, T, seed,
                                  wl["start"], equil, U),
                   "dim": dim, "L": L, "T": T, "seed": seed, "updates_per_step": U,
                   "schedule": args.schedule, "grid_blocks": info["grid_blocks"],
                   "t_up": args.t_up, "t_down": args.t_down,
                   "block_threads": info["block_threads"],
                   "helper_clusters": info.get("helper_clusters"),
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": "replicas x%d" % world},
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
        "clocks": clk,
        "detail": {"mean_cluster": flips / len(records), "mean_levels": float(levels.mean()),
                   "max_levels": int(levels.max()), "ms_per_update": total_ms / len(records),
                   "steps_and_e2e_records_identical": bool(repeat_identical),
                   # window mode commits updates in rounds, so the device time
                   # is per step (U updates), not per update
                   "step_ms_p50": float(np.percentile(step_ms, 50)),
                   "step_ms_p99": float(np.percentile(step_ms, 99)),
                   "step_counters": {k: stats1[k] - stats0[k] for k in stats1}},
    }


def run_small(args):
    """The small configuration, whole run on both sides: 2D L=16, J=1,
    T = T_c, Philox random start from seed 1, 10^4 updates with every record,
    timed on the GPU (one launch, CUDA events, after warm-up runs from the
    same start; the median of the timed runs, repeated for at least 0.6 s so
    that the clock sampler sees them) and by the oracle (one core); the
    records are compared."""
    import numpy as np
    import torch

    import oracle
    import paper_1110_0899_gb300 as w
    dim, L, T, seed, n = 2, 16, TC2, 1, 10000
    lat = w.WolffLattice(dim, L, T, seed=seed)
    info = lat.info()
    start, _ = lat.get_state()
    buf = lat.record_buffer(n)
    stream_times = []
    warm = max(3, args.warmup)
    clocks = ClockSampler(torch.cuda.current_device())
    k, t_first = 0, None
    while len(stream_times) < max(3, args.steps) or time.perf_counter() - t_first < 0.6:
        if k == warm:
            clocks.start()
            time.sleep(0.3)   # the sampler's start-up stays out of the timed runs
            t_first = time.perf_counter()
        lat.set_state(start, 0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        w.wolff_step(lat.handle, n, buf)
        b.record()
        b.synchronize()
        if k >= warm:
            stream_times.append(a.elapsed_time(b) / 1000.0)
        k += 1
    ck = clocks.stop()
    rec = w.records_to_numpy(buf, n)
    lat.close()
    thr = oracle.bond_threshold(1.0, T)
    s = oracle.init_lattice(dim, L, seed)
    t0 = time.perf_counter()
    ref = oracle.run(dim, L, thr, seed, 0, n, s)
    t_orc = time.perf_counter() - t0
    flips = int(rec["C"].astype(np.int64).sum())
    t_gpu = float(np.median(stream_times))
    return {"workload": "2D L=16 T=%.6g J=1 seed 1, random start, 10^4 updates with records, "
                        "the whole run on both sides" % T,
            "gpu_flips_per_s": flips / t_gpu, "gpu_ms": 1000.0 * t_gpu,
            "oracle_flips_per_s": flips / t_orc, "oracle_ms": 1000.0 * t_orc,
            "oracle": "E_bond and M recounted from their definitions after every update, one core",
            "records_equal_oracle": bool(np.array_equal(rec, ref)),
            "mean_cluster": flips / n,
            "mean_levels": float(rec["levels"].mean()),
            "gpu_us_per_update": 1e6 * t_gpu / n,
            "timed_runs": len(stream_times),
            "clocks": ck,
            # what bounds it: one SM (1 of the GPU's SMs) running a dependent
            # chain per breadth-first level; cycles per level at the sampled
            # clock (the maximum clock when no sample came)
            "cycles_per_level": (t_gpu / n) * 1e6 * float(ck.get("sm_mhz") or ck.get("sm_max_mhz")
                                                         or 2070.0) / float(rec["levels"].mean()),
            "sms_used": 1,
            "schedule": {w.SCHED_TINY: "tiny: one CTA of %d threads, the lattice in shared "
                                       "memory as bit planes" % info["block_threads"]}.get(
                info["schedule"], "schedule %d" % info["schedule"])}


def run_tiny_sizes(args):
    """The tiny schedule against the cluster schedule on the lattices it
    takes, per update, at 0.9, 1.0 and 1.1 T_c, from a fresh random lattice
    and after equilibration updates (random start seed 5; CUDA events; the
    best of two runs of the same updates from the same state)."""
    import torch

    import paper_1110_0899_gb300 as w
    torch.cuda.set_device(0)
    if args.sizes:
        cases = [tuple(int(v) for v in c.split(":")) for c in args.sizes.split(",")]
    else:
        cases = [(2, 16), (2, 32), (2, 48), (2, 64), (2, 96), (2, 128), (2, 181),
                 (3, 4), (3, 8), (3, 12), (3, 16), (3, 20), (3, 24), (3, 32)]
    temps = [float(v) for v in args.temps.split(",")]
    regimes = args.regimes.split(",")
    rows = []
    for dim, L in cases:
        N = L ** dim
        for tf in temps:
            T = (TC2 if dim == 2 else 4.5115) * tf
            for regime in regimes:
                pre = 0 if regime == "random" else (2000 if N <= 4096 else 600)
                n = 2000 if N <= 4096 else 400
                base = w.WolffLattice(dim, L, T, seed=5)
                base.set_schedule(w.SCHED_TINY)
                if pre:
                    base.step(pre, records=False)
                s0, t0 = base.get_state()
                base.close()
                row = {"dim": dim, "L": L, "T_over_Tc": tf, "regime": regime, "updates": n}
                recs = {}
                for name, sched in (("tiny", w.SCHED_TINY), ("cluster", w.SCHED_CLUSTER)):
                    lat = w.WolffLattice(dim, L, T, seed=5)
                    lat.set_schedule(sched)
                    buf = lat.record_buffer(n)
                    best = None
                    for _ in range(2):
                        lat.set_state(s0, t0)
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record()
                        w.wolff_step(lat.handle, n, buf)
                        b.record()
                        b.synchronize()
                        ms = a.elapsed_time(b)
                        best = ms if best is None else min(best, ms)
                    recs[name] = w.records_to_numpy(buf, n)
                    row["%s_us_per_update" % name] = 1000.0 * best / n
                    if name == "tiny":
                        row["tiny_threads"] = lat.info()["block_threads"]
                    lat.close()
                row["mean_cluster"] = float(recs["tiny"]["C"].mean())
                row["mean_levels"] = float(recs["tiny"]["levels"].mean())
                row["records_equal"] = bool((recs["tiny"] == recs["cluster"]).all())
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "microseconds per update, tiny vs cluster schedule",
                      "unit": "us", "higher_is_better": False, "tiny_sizes": rows}), flush=True)


def add_l2_side(line, l2):
    """The L2 side of a line's roofline: the same algorithmic bytes against
    the probe's L2 read bandwidth, and the ncu L2 bytes when fresh."""
    roof = line["roofline"]
    ms = line["ms_per_step"]
    l2_side = {"achieved": roof["achieved"], "peak": l2["read_gbs"], "unit": "GB/s",
               "frac": roof["achieved"] / l2["read_gbs"], "peak_kind": "measured live: " + l2["how"]}
    traffic = roof.pop("l2_traffic", None)
    l2_side["traffic"] = traffic
    if traffic is not None:
        l2_side["traffic_gbs"] = traffic / (ms / 1000.0) / 1e9
        l2_side["traffic_frac"] = l2_side["traffic_gbs"] / l2["read_gbs"]
    roof["l2"] = l2_side


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS.get(args.workload, {}).get("model") == "xy":
        return run_xy(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "binder":
        return run_binder(args)
    if args.workload == "small":
        import torch
        torch.cuda.set_device(0)
        sm = run_small(args)
        print(json.dumps({"metric": METRIC, "value": sm["gpu_flips_per_s"], "unit": UNIT,
                          "n_gpus": 1, "higher_is_better": True,
                          "config": {"workload": sm["workload"]}, "small": sm}), flush=True)
        return
    if args.workload == "tiny-sizes":
        return run_tiny_sizes(args)
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1110_0899_gb300 as w   # noqa: F401  (fails loudly without the library)

    line = run_ising(args, args.workload)
    headline = world == 1 and args.workload == "2d"
    l2 = None
    if world == 1 and not args.no_l2_probe and not WORKLOADS[args.workload].get("q"):
        l2 = l2_probe()
        add_l2_side(line, l2)
        line["l2_probe"] = l2
    if headline and not args.no_3d:
        d3 = run_ising(args, "3d")
        if l2 is not None:
            add_l2_side(d3, l2)
        line["3d"] = {k: d3[k] for k in ("value", "unit", "ms_per_step", "config", "roofline",
                                          "cpu_baseline", "e2e", "clocks", "gpu_launches",
                                          "detail")}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if headline and not args.no_small:
        line["small"] = run_small(args)
    if headline and not args.no_batched:
        class _A:   # the specified batched workload: 10^4 updates per replica
            steps, updates_per_step = 1, args.batched_updates
        line["batched"] = run_batched(_A, updates=args.batched_updates, embed=True,
                                      plain_every=args.plain_every)
    if headline and not args.no_served:
        class _S:
            serve_seconds = args.embed_serve_seconds
            no_tiny_engine = args.no_tiny_engine
            epoch_ms = args.epoch_ms
        line["served"] = run_served(_S, embed=True)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
