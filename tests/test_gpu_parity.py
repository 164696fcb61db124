"""GPU path vs the CPU oracle, bit for bit (section 2's update on the GPU).

Every test drives the CUDA kernels through the C ABI (the Python binding only
marshals arguments) and compares the per-update records (|C|, levels,
E_bond, M) and the lattice with the oracle on the same seeded inputs, for both
schedules and for several launch shapes, since the cluster is a connected
component and must not depend on the exploration order."""
import math

import numpy as np
import pytest

import oracle
from _gpu import assert_records_equal, oracle_trajectory, require_cuda

pytestmark = pytest.mark.gpu

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))
SCHEDS = ("persistent", "graph", "cluster")


def sched_id(w, name):
    return {"persistent": w.SCHED_PERSISTENT, "graph": w.SCHED_GRAPH,
            "cluster": w.SCHED_CLUSTER}[name]


def run_gpu(w, dim, L, T, seed, n, sched, blocks=0, threads=0):
    lat = w.WolffLattice(dim, L, T, seed=seed)
    if sched == "cluster" and blocks not in (0, 1, 2, 4, 8, 16):
        blocks = 8   # CTA counts of the other schedules map to a cluster size
    lat.set_schedule(sched_id(w, sched), blocks, threads)
    rec = lat.step(n)
    spins, t = lat.get_state()
    E, M, C = lat.measure()
    Ef, Mf = lat.measure_full()
    lat.close()
    assert t == n
    assert (E, M) == (Ef, Mf)
    if n:
        assert (E, M, C) == (rec["E"][-1], rec["M"][-1], rec["C"][-1])
    return rec, spins


def test_device_philox_matches_oracle():
    torch, w = require_cuda()
    rng = np.random.default_rng(5)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = [[0, 0, 0, 0], [0, 0, 0, 1], [0, 0, 0, 2], [2**32 - 1] * 4,
               [5, 1, 0, 0], [16777215, 11999, 0, 0], [1, 2**32 - 1, 7, 0], [3, 3, 3, 3]]
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    for key in ((0, 0), (1, 0), (0xDEADBEEF, 0x12345678), (2**32 - 1, 2**32 - 1)):
        w.wolff_philox(key[0], key[1], d_ctr, d_out, n)
        got = d_out.cpu().numpy().view(np.uint32)
        for k in list(range(8)) + list(rng.integers(0, n, 64)):
            assert np.array_equal(got[k], oracle.philox4x32_10(key, ctr[k])), (key, k)


@pytest.mark.parametrize("sched", SCHEDS)
def test_small_workload_2d_l16(sched):
    """2D L=16, J=1, T=Tc, seed 1, 10^4 updates: every record and the final lattice."""
    torch, w = require_cuda()
    ref, s_ref = oracle_trajectory(2, 16, TC2, 1, 10_000)
    rec, spins = run_gpu(w, 2, 16, TC2, 1, 10_000, sched)
    assert_records_equal(rec, ref, "2D L=16 " + sched)
    assert np.array_equal(spins, s_ref)


@pytest.mark.parametrize("sched", SCHEDS)
def test_3d_l8(sched):
    torch, w = require_cuda()
    ref, s_ref = oracle_trajectory(3, 8, 4.5115, 3, 2_000)
    rec, spins = run_gpu(w, 3, 8, 4.5115, 3, 2_000, sched)
    assert_records_equal(rec, ref, "3D L=8 " + sched)
    assert np.array_equal(spins, s_ref)


# ragged and degenerate shapes: L=2 (double bonds), odd L, non powers of two,
# a single CTA, a one-warp CTA and many CTAs over a tiny lattice
SHAPES = [
    (2, 2, 1.0, 300, 1, 32), (2, 3, TC2, 300, 0, 0), (3, 2, 4.5115, 300, 3, 64),
    (3, 3, 3.0, 300, 0, 0), (2, 37, TC2, 400, 5, 96), (2, 100, 2.0, 300, 0, 512),
    (3, 13, 4.5115, 300, 0, 0), (3, 17, 4.0, 200, 64, 256), (2, 64, 2.6, 400, 152, 128),
    (2, 255, TC2, 150, 0, 0),
]


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("dim,L,T,n,blocks,threads", SHAPES)
def test_ragged_shapes(sched, dim, L, T, n, blocks, threads):
    torch, w = require_cuda()
    seed = 1000 + L
    ref, s_ref = oracle_trajectory(dim, L, T, seed, n)
    rec, spins = run_gpu(w, dim, L, T, seed, n, sched, blocks, threads)
    assert_records_equal(rec, ref, "%dD L=%d %s" % (dim, L, sched))
    assert np.array_equal(spins, s_ref)


@pytest.mark.parametrize("sched", SCHEDS)
def test_degenerate_thresholds(sched):
    torch, w = require_cuda()
    # T = inf: thr = 0, every cluster is the seed alone
    rec, _ = run_gpu(w, 2, 32, float("inf"), 4, 100, sched)
    assert np.all(rec["C"] == 1) and np.all(rec["levels"] == 1)
    ref, _ = oracle_trajectory(2, 32, float("inf"), 4, 100)
    assert_records_equal(rec, ref, "T=inf")
    # T -> 0: thr = 2^32, clusters are whole aligned domains
    for dim, L in ((2, 48), (3, 10)):
        ref, s_ref = oracle_trajectory(dim, L, 1e-3, 6, 50)
        rec, spins = run_gpu(w, dim, L, 1e-3, 6, 50, sched)
        assert_records_equal(rec, ref, "T=0")
        assert np.array_equal(spins, s_ref)


@pytest.mark.parametrize("sched", SCHEDS)
def test_medium_lattices(sched):
    """Lattices spanning many CTAs: 2D L=512 at Tc, 3D L=64 at 4.5115."""
    torch, w = require_cuda()
    for dim, L, T, n in ((2, 512, TC2, 120), (3, 64, 4.5115, 60)):
        ref, s_ref = oracle_trajectory(dim, L, T, 7, n)
        rec, spins = run_gpu(w, dim, L, T, 7, n, sched)
        assert_records_equal(rec, ref, "%dD L=%d" % (dim, L))
        assert np.array_equal(spins, s_ref)


THRESHOLDS = [(0, 0), (1, 1), (8, 4), (64, 8), (512, 256), (2048, 2048)]


@pytest.mark.parametrize("sched", ["persistent", "cluster"])
@pytest.mark.parametrize("t_up,t_down", THRESHOLDS)
def test_leader_grid_handoffs(t_up, t_down, sched):
    """Large clusters from an ordered start cross between the leader-only and
    the all-CTA phases many times; every threshold gives the oracle's chain."""
    torch, w = require_cuda()
    for dim, L, T, n in ((2, 256, TC2, 40), (3, 32, 4.5115, 30), (2, 100, 2.1, 30)):
        up = np.ones(L ** dim, dtype=np.int8)
        ref, s_ref = oracle_trajectory(dim, L, T, 31, n, s=up)
        lat = w.WolffLattice(dim, L, T, seed=31)
        lat.set_schedule(w.SCHED_PERSISTENT if sched == "persistent" else w.SCHED_CLUSTER)
        lat.set_local_thresholds(t_up, t_down)
        lat.set_state(up, 0)
        rec = lat.step(n)
        spins, _ = lat.get_state()
        assert (lat.measure()[:2]) == lat.measure_full()
        lat.close()
        assert_records_equal(rec, ref, "%dD L=%d thresholds %d/%d" % (dim, L, t_up, t_down))
        assert np.array_equal(spins, s_ref)


def test_checkpoint_resume_and_segments():
    torch, w = require_cuda()
    dim, L, T, seed = 2, 128, TC2, 9
    ref, s_ref = oracle_trajectory(dim, L, T, seed, 300)
    a = w.WolffLattice(dim, L, T, seed=seed)
    r1 = a.step(120)
    snap, t = a.get_state()
    assert t == 120
    b = w.WolffLattice(dim, L, T, seed=seed, schedule=w.SCHED_GRAPH)
    b.set_state(snap, t)
    r2 = b.step(180)
    assert_records_equal(np.concatenate([r1, r2]), ref, "resume")
    spins, t2 = b.get_state()
    assert t2 == 300 and np.array_equal(spins, s_ref)
    # the same context switching schedule between calls
    c = w.WolffLattice(dim, L, T, seed=seed)
    parts = []
    for k, sched in enumerate([w.SCHED_PERSISTENT, w.SCHED_GRAPH] * 3):
        c.set_schedule(sched)
        parts.append(c.step(50))
    assert_records_equal(np.concatenate(parts), ref, "alternating schedules")
    for x in (a, b, c):
        x.close()


def test_set_state_rejects_non_spin_values():
    torch, w = require_cuda()
    lat = w.WolffLattice(2, 16, TC2, seed=1)
    bad = np.ones(256, dtype=np.int8)
    bad[17] = 0
    with pytest.raises(w.WolffError) as ei:
        lat.set_state(bad, 0)
    assert ei.value.status == w.WOLFF_EINVAL
    good = oracle.init_lattice(2, 16, 1)
    lat.set_state(good, 0)
    ref, _ = oracle_trajectory(2, 16, TC2, 1, 50)
    assert_records_equal(lat.step(50), ref, "after rejected restore")
    lat.close()


def test_host_buffer_path():
    torch, w = require_cuda()
    dim, L, T, seed = 3, 20, 4.5115, 12
    s0 = oracle.init_lattice(dim, L, seed)
    ref, s_ref = oracle_trajectory(dim, L, T, seed, 80, t0=40, s=s0)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    rec, spins = lat.run_host(80, spins_in=s0, t_in=40)
    assert_records_equal(rec, ref, "run_host")
    assert np.array_equal(spins, s_ref)
    # the upload and the updates are enqueued behind one synchronisation: a
    # lattice entry other than +-1 is still reported, and the context then
    # takes a valid lattice again
    bad = s0.copy()
    bad[5] = 3
    with pytest.raises(w.WolffError) as ei:
        lat.run_host(10, spins_in=bad, t_in=0)
    assert ei.value.status == w.WOLFF_EINVAL
    rec, spins = lat.run_host(80, spins_in=s0, t_in=40)
    assert_records_equal(rec, ref, "run_host after a rejected upload")
    assert np.array_equal(spins, s_ref)
    lat.close()


@pytest.mark.parametrize("dim,L", [(2, 37), (3, 11)])
def test_bit_packed_transfers(dim, L):
    """The bit-packed state transfers and host-buffer path give what the int8
    ones give (ragged N: the last word is partial)."""
    torch, w = require_cuda()
    T, seed = (2.5, 8) if dim == 2 else (4.8, 9)
    s0 = oracle.init_lattice(dim, L, seed)
    ref, s_ref = oracle_trajectory(dim, L, T, seed, 60, t0=13, s=s0)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    lat.set_state_bits(w.pack_spins(s0), 13)
    assert lat.measure()[:2] == (oracle.energy_bond(dim, L, s0), oracle.magnetisation(dim, L, s0))
    bits, t = lat.get_state_bits()
    assert t == 13 and np.array_equal(bits, w.pack_spins(s0))
    rec, bout = lat.run_host_bits(60, bits_in=w.pack_spins(s0), t_in=13)
    assert_records_equal(rec, ref, "run_host_bits")
    assert np.array_equal(w.unpack_bits(bout, L ** dim), s_ref)
    assert np.array_equal(lat.get_state()[0], s_ref)
    # the records straight into a caller-owned pinned buffer (longer than n)
    pinned = torch.empty(64 * w.RECORD_BYTES, dtype=torch.uint8, pin_memory=True)
    out = pinned.numpy().view(w.RECORD_DTYPE)
    rec2, _ = lat.run_host_bits(60, bits_in=w.pack_spins(s0), t_in=13, bits_out=False,
                                records_out=out)
    assert rec2.base is not None and len(rec2) == 60
    assert_records_equal(out[:60], ref, "run_host_bits into records_out")
    with pytest.raises(ValueError):
        lat.run_host_bits(60, bits_in=w.pack_spins(s0), t_in=13, records_out=out[:59])
    lat.close()


@pytest.mark.parametrize("dim,L", [(2, 32), (2, 96), (2, 1024), (3, 32), (3, 64), (2, 48),
                                   (3, 24)])
def test_word_parallel_measure_and_upload(dim, L):
    """Lattices whose side is a multiple of 32 take the 32-sites-per-thread
    recount and bit-packed upload (other sides the per-site ones): E_bond
    and M equal the oracle's definitions on random and ordered lattices, and
    the uploaded lattice reads back unchanged."""
    torch, w = require_cuda()
    rng = np.random.default_rng(1000 * dim + L)
    for s in (rng.choice(np.array([-1, 1], np.int8), size=L ** dim),
              np.ones(L ** dim, np.int8), -np.ones(L ** dim, np.int8)):
        lat = w.WolffLattice(dim, L, 2.5 if dim == 2 else 4.8, seed=5)
        lat.set_state_bits(w.pack_spins(s), 3)
        ref = (oracle.energy_bond(dim, L, s), oracle.magnetisation(dim, L, s))
        assert lat.measure()[:2] == ref
        assert lat.measure_full() == ref
        back, t = lat.get_state()
        assert t == 3 and np.array_equal(back, s)
        lat.close()


@pytest.mark.parametrize("dim,L", [(2, 4096), (3, 256)])
def test_full_size_state_transfer(dim, L):
    """The fused upload (int8 +-1 -> spin bytes, E_bond and M in the same
    pass) and the download at the benchmark's sizes: E_bond and M equal the
    oracle's definitions, the lattice comes back unchanged, and the cluster
    list is left empty for the next update (the next 50 updates match)."""
    torch, w = require_cuda()
    rng = np.random.default_rng(dim)
    s = rng.choice(np.array([-1, 1], np.int8), size=L ** dim)
    lat = w.WolffLattice(dim, L, 1.0 if dim == 2 else 4.5115, seed=31)
    lat.set_state(s, 77)
    E, M, _ = lat.measure()
    assert (E, M) == (oracle.energy_bond(dim, L, s), oracle.magnetisation(dim, L, s))
    back, t = lat.get_state()
    assert t == 77 and np.array_equal(back, s)
    bits, t = lat.get_state_bits()
    assert t == 77 and np.array_equal(bits, w.pack_spins(s))
    lat.set_state_bits(bits, 77)
    assert lat.measure()[:2] == (E, M)
    rec = lat.step(50)
    T = 1.0 if dim == 2 else 4.5115
    ref, s_ref = oracle_trajectory(dim, L, T, 31, 50, t0=77, s=s)
    assert_records_equal(rec, ref, "after a full-size upload")
    lat.close()


def test_bounded_wait_reports_timeout_and_context_survives():
    torch, w = require_cuda()
    lat = w.WolffLattice(2, 16, TC2, seed=1)
    assert lat.selftest_wait_timeout(20_000_000) == w.WOLFF_ETIMEOUT   # 20 ms limit
    ref, _ = oracle_trajectory(2, 16, TC2, 1, 100)
    assert_records_equal(lat.step(100), ref, "after self test")
    lat.close()


# ---- cluster ("team") schedule and the batched form --------------------------

@pytest.mark.parametrize("cluster", [1, 2, 4, 8, 16])
def test_cluster_schedule_matches_oracle(cluster):
    torch, w = require_cuda()
    for dim, L, T, n, start in ((2, 16, TC2, 2000, "random"), (3, 9, 4.5115, 400, "random"),
                                (2, 128, TC2, 40, "ordered"), (3, 24, 4.5115, 30, "ordered"),
                                (2, 37, 2.0, 60, "ordered")):
        s0 = oracle.init_lattice(dim, L, 77) if start == "random" else np.ones(L ** dim, np.int8)
        ref, s_ref = oracle_trajectory(dim, L, T, 77, n, s=s0)
        lat = w.WolffLattice(dim, L, T, seed=77)
        try:
            lat.set_schedule(w.SCHED_CLUSTER, cluster, 256)
        except w.WolffError:
            pytest.skip("cluster size %d not accepted" % cluster)
        lat.set_state(s0, 0)
        lat.set_local_thresholds(64, 16)
        try:
            rec = lat.step(n)
        except w.WolffError as e:
            if cluster == 16:
                pytest.skip("16-CTA clusters not launchable here: %s" % e)
            raise
        spins, t = lat.get_state()
        assert lat.measure()[:2] == lat.measure_full()
        lat.close()
        assert_records_equal(rec, ref, "cluster %d %dD L=%d" % (cluster, dim, L))
        assert np.array_equal(spins, s_ref) and t == n


@pytest.mark.parametrize("t_up,t_down", [(0, 0), (8, 2), (2048, 1024)])
def test_cluster_thresholds(t_up, t_down):
    torch, w = require_cuda()
    dim, L, T, n = 2, 200, TC2, 30
    up = np.ones(L * L, np.int8)
    ref, s_ref = oracle_trajectory(dim, L, T, 5, n, s=up)
    lat = w.WolffLattice(dim, L, T, seed=5, schedule=w.SCHED_CLUSTER, grid_blocks=8,
                         block_threads=512)
    lat.set_local_thresholds(t_up, t_down)
    lat.set_state(up, 0)
    rec = lat.step(n)
    spins, _ = lat.get_state()
    lat.close()
    assert_records_equal(rec, ref, "cluster thresholds %d/%d" % (t_up, t_down))
    assert np.array_equal(spins, s_ref)


def test_batched_replicas_match_each_alone():
    """Uneven lattices and temperatures in one launch, several calls in a row:
    every replica's records and lattice equal the oracle's chain alone."""
    torch, w = require_cuda()
    rng = np.random.default_rng(4)
    specs = []
    for i in range(24):
        dim = 2 if i % 4 else 3
        L = int(rng.choice([8, 13, 32, 64])) if dim == 2 else int(rng.choice([5, 8, 11]))
        T = float(rng.uniform(0.9, 1.1)) * (TC2 if dim == 2 else 4.5115)
        specs.append((dim, L, T, 1000 + i))
    lats = [w.WolffLattice(d, L, T, seed=s) for d, L, T, s in specs]
    batch = w.WolffBatch(len(lats))
    calls = [(60, 1, 128), (40, 2, 256), (75, 4, 256)]
    got = [[] for _ in lats]
    for n, cs, thr in calls:
        bufs = [lat.record_buffer(n) for lat in lats]
        batch.run(lats, [n] * len(lats), bufs, cluster_size=cs, block_threads=thr)
        torch.cuda.synchronize()
        for k, (lat, b) in enumerate(zip(lats, bufs)):
            got[k].append(w.records_to_numpy(b, n))
    total = sum(c[0] for c in calls)
    for k, ((dim, L, T, seed), lat) in enumerate(zip(specs, lats)):
        ref, s_ref = oracle_trajectory(dim, L, T, seed, total)
        assert_records_equal(np.concatenate(got[k]), ref, "replica %d" % k)
        spins, t = lat.get_state()
        assert t == total and np.array_equal(spins, s_ref)
        lat.close()
    batch.close()


@pytest.mark.parametrize("dim,L,T,n", [(2, 200, 5.0, 600), (2, 64, TC2, 600), (3, 16, 8.0, 600),
                                       (2, 4096, TC2, 300), (2, 12, 3.0, 400), (3, 5, 6.0, 400)])
def test_burst_mode_matches_oracle(dim, L, T, n):
    """Speculative bursts (many small updates grown at once, committed in
    order while they do not interact) give the serial chain exactly, on
    lattices where they mostly commit (high T, large L) and where conflicts
    and oversized clusters cut them short (small L, T_c)."""
    torch, w = require_cuda()
    seed = 123 + L
    ref, s_ref = oracle_trajectory(dim, L, T, seed, n)
    for threads in (256, 512):
        lat = w.WolffLattice(dim, L, T, seed=seed, schedule=w.SCHED_CLUSTER, grid_blocks=4,
                             block_threads=threads)
        lat.set_burst(True)
        rec = lat.step(n)
        st = lat.stats()
        spins, _ = lat.get_state()
        assert lat.measure()[:2] == lat.measure_full()
        lat.close()
        assert_records_equal(rec, ref, "burst %dD L=%d T=%g threads %d" % (dim, L, T, threads))
        assert np.array_equal(spins, s_ref)
        if T > 4.0 and L ** dim > 1000:
            assert st["burst_updates"] > n // 2


@pytest.mark.parametrize("dim,L,T,n", [(2, 32, 5.0, 1500), (2, 20, 3.2, 1200),
                                       (3, 8, 9.0, 1200), (3, 12, 6.0, 800)])
@pytest.mark.parametrize("levels,cs,threads", [(1, 16, 512), (2, 4, 256), (3, 1, 128),
                                               (6, 2, 512)])
def test_window_rounds_and_regrowth(dim, L, T, n, levels, cs, threads):
    """Window mode on small hot lattices, where the updates of a window often
    read each other's flips: short rounds (1-3 growth levels) make updates
    span several commits, so finished and half-grown updates are grown again,
    and the chain must still be the serial one, lattice included."""
    torch, w = require_cuda()
    seed = 900 + L + levels
    ref, s_ref = oracle_trajectory(dim, L, T, seed, n)
    check_run_window(w, dim, L, T, n, levels, cs, threads, seed, ref, s_ref)


@pytest.mark.parametrize("dim,L,T,n", [(2, 96, 2.5, 1500), (3, 20, 4.8, 1200)])
@pytest.mark.parametrize("levels,cs,threads", [(4, 16, 512), (32, 4, 256), (64, 1, 512)])
def test_window_resumes_after_oversized_update(dim, L, T, n, levels, cs, threads):
    """Near T_c some clusters outgrow a window update's member cap (64 in 2D at
    512 threads, else 128).  The window then hands that update to the ordinary
    path and resumes with the updates it had finished, each revalidated
    against the lattice the big flip left; the chain must stay the serial one."""
    torch, w = require_cuda()
    seed = 4200 + L + levels
    ref, s_ref = oracle_trajectory(dim, L, T, seed, n)
    cap = 128 if (threads <= 256 or dim == 3) else 64
    assert int((ref["C"] > cap).sum()) >= 3   # the resume path is exercised
    check_run_window(w, dim, L, T, n, levels, cs, threads, seed, ref, s_ref)


def check_run_window(w, dim, L, T, n, levels, cs, threads, seed, ref, s_ref):
    lat = w.WolffLattice(dim, L, T, seed=seed, schedule=w.SCHED_CLUSTER, grid_blocks=cs,
                         block_threads=threads)
    lat.set_burst(levels)
    rec = np.concatenate([lat.step(k) for k in (n // 3, n - n // 3)])
    st = lat.stats()
    spins, t = lat.get_state()
    assert lat.measure()[:2] == lat.measure_full()
    lat.close()
    tag = "window %dD L=%d T=%g levels %d cs %d threads %d" % (dim, L, T, levels, cs, threads)
    assert_records_equal(rec, ref, tag)
    assert t == n and np.array_equal(spins, s_ref)
    assert st["burst_updates"] > n // 4, (tag, st)


@pytest.mark.parametrize("dim,L,T,seed", [(2, 4096, TC2, 2), (3, 256, 4.5115, 3)])
def test_full_size_every_record_in_bench_configuration(dim, L, T, seed):
    """The workloads bench.py times, at full size and in its launch
    configuration (default schedule: one 16-CTA cluster, 512 threads, window
    mode): the specified equilibration in two launches of 1000 unrecorded
    updates, then the bench's step -- the equilibrated lattice restored
    through the bit-packed upload and the 10^4 measured updates in one
    launch.  The lattice after equilibration, every one of the 10^4 records
    (|C|, levels, E_bond, M) and the final lattice must equal the oracle's,
    and the incremental E and M a full recount."""
    torch, w = require_cuda()
    thr = oracle.bond_threshold(1.0, T)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    for _ in range(2):
        lat.step(1000, records=False)
    snap, t0 = lat.get_state()
    assert t0 == 2000
    lat.set_state_bits(w.pack_spins(snap), t0)
    rec = lat.step(10000)
    end, t1 = lat.get_state()
    E, M, _ = lat.measure()
    full = lat.measure_full()
    st = lat.stats()
    lat.close()
    s = oracle.init_lattice(dim, L, seed)
    oracle.run(dim, L, thr, seed, 0, 2000, s, records=False)
    assert np.array_equal(s, snap), "lattice after the equilibration"
    ref = oracle.run_local(dim, L, thr, seed, 2000, 10000, s)
    assert_records_equal(rec, ref, "full size %dD L=%d, all 10^4 records" % (dim, L))
    assert t1 == 12000 and np.array_equal(end, s)
    assert (E, M) == full == (int(ref["E"][-1]), int(ref["M"][-1]))
    assert st["burst_updates"] > 0   # the bench's window path is the one exercised


@pytest.mark.parametrize("dim,L,T,seed", [(2, 4096, TC2, 2), (3, 256, 4.5115, 3)])
def test_whole_trajectory_in_segments(dim, L, T, seed):
    """The full specified runs (2000 equilibration + 10^4 measured updates, in
    the benchmark's launch configuration): the GPU snapshots its lattice every
    500 updates; the oracle replays every segment from the previous snapshot
    and must reach the next one bit for bit, every record of the 10^4
    measured updates equal to its own; E_bond and M at every snapshot equal
    the definitions; every record obeys |dM| = 2|C| and E changes by an even
    amount.  The benchmark's own step,
    the 10^4 measured updates in one launch from the equilibrated lattice,
    must then give the same records and reach the oracle-checked end."""
    torch, w = require_cuda()
    thr = oracle.bond_threshold(1.0, T)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    snaps = [lat.get_state()]
    recs = []
    for k in range(24):                       # 12000 updates in steps of 500
        rec = lat.step(500)
        if k >= 4:
            recs.append(rec)
        snaps.append(lat.get_state())
    E, M, _ = lat.measure()
    lat.close()
    for k, ((s_a, t_a), (s_b, t_b)) in enumerate(zip(snaps, snaps[1:])):
        assert t_b == t_a + 500
        s = np.array(s_a, dtype=np.int8, copy=True)
        seg = oracle.run_local(dim, L, thr, seed, t_a, 500, s)
        assert np.array_equal(s, s_b), "segment starting at update %d" % t_a
        if k >= 4:
            assert_records_equal(recs[k - 4], seg, "segment starting at update %d" % t_a)
    assert (E, M) == (oracle.energy_bond(dim, L, snaps[-1][0]),
                      oracle.magnetisation(dim, L, snaps[-1][0]))
    rec = np.concatenate(recs)
    E_prev = oracle.energy_bond(dim, L, snaps[4][0])
    M_prev = oracle.magnetisation(dim, L, snaps[4][0])
    for k, r in enumerate(rec):
        assert abs(int(r["M"]) - M_prev) == 2 * int(r["C"]), k
        assert (int(r["E"]) - E_prev) % 2 == 0, k
        E_prev, M_prev = int(r["E"]), int(r["M"])
        if (k + 1) % 500 == 0:   # the record at a snapshot equals its recount
            s_k = snaps[4 + (k + 1) // 500][0]
            assert (E_prev, M_prev) == (oracle.energy_bond(dim, L, s_k),
                                        oracle.magnetisation(dim, L, s_k)), k
    # one launch of the 10^4 measured updates, as bench.py times them
    lat = w.WolffLattice(dim, L, T, seed=seed)
    lat.set_state(*snaps[4])
    one = lat.step(10000)
    end, t_end = lat.get_state()
    lat.close()
    assert t_end == snaps[-1][1] and np.array_equal(end, snaps[-1][0])
    assert np.array_equal(one, rec)


@pytest.mark.parametrize("dim,L,T,seed,n", [(2, 1024, TC2, 41, 3000), (3, 102, 4.5115, 42, 3000),
                                             (2, 2048, 2.4, 43, 2000), (2, 1024, 2.3, 44, 4000),
                                             # larger clusters: pre-grown updates are often
                                             # invalidated by earlier commits and grown again
                                             (2, 1024, 2.29, 45, 12000), (3, 102, 4.45, 46, 8000)])
def test_helper_teams_keep_the_chain(dim, L, T, seed, n):
    """One-lattice launches on lattices with a ring of pre-grown updates
    (2^20 sites or more): the helper clusters grow updates ahead and the main
    cluster takes those whose read set still holds.  Every record and the
    final lattice must equal the oracle's; pre-grown results must have been
    used; a second launch from the restored lattice (the benchmark's pattern:
    the same update indices again) must give the same records without reusing
    the first launch's results; and so must a launch without helpers."""
    torch, w = require_cuda()
    thr = oracle.bond_threshold(1.0, T)
    s = oracle.init_lattice(dim, L, seed)
    ref = oracle.run_local(dim, L, thr, seed, 0, n, s)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    assert lat.info()["helper_clusters"] >= 1
    start, _ = lat.get_state()
    rec = lat.step(n)
    st = lat.stats()
    end, t_end = lat.get_state()
    assert_records_equal(rec, ref, "helpers %dD L=%d T=%g" % (dim, L, T))
    assert t_end == n and np.array_equal(end, s)
    assert st["pregrown"] > 0 and st["burst_updates"] > 0, st
    # the same updates again from the restored lattice
    lat.set_state(start, 0)
    rec2 = lat.step(n)
    st2 = lat.stats()
    assert np.array_equal(rec2, rec) and st2["pregrown"] > 0
    # and without helper teams
    lat.set_helpers(0)
    assert lat.info()["helper_clusters"] == 0
    lat.set_state(start, 0)
    rec3 = lat.step(n)
    assert lat.stats()["pregrown"] == 0
    assert np.array_equal(rec3, rec)
    assert np.array_equal(lat.get_state()[0], s)
    lat.close()
