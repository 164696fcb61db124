"""Batched plans, the autotuner and the serving loop do not change results.

Every lattice follows the chain it would follow alone, whatever it shares a
launch with: records from the batched runner and from the server are
compared bit for bit with the same lattice run alone (and, for a few, with
the CPU oracle)."""
import numpy as np
import pytest

from _gpu import assert_records_equal, oracle_trajectory, require_cuda

pytestmark = pytest.mark.gpu


def _small_specs(n=40):
    from paper_1110_0899_gb300 import workloads
    specs = workloads.batched_replicas(n, sizes=(16, 32, 48, 64, 96))
    # a few 3D lattices too
    for i in range(0, n, 7):
        specs[i] = dict(dim=3, L=int(8 + i % 5), T=4.5115 * (0.9 + 0.01 * i), seed=specs[i]["seed"])
    return specs


def test_split_plan_runner_matches_alone():
    torch, w = require_cuda()
    from paper_1110_0899_gb300 import batched
    specs = _small_specs()
    lats = [w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"]) for s in specs]
    big = [i for i, s in enumerate(specs) if s["L"] ** s["dim"] >= 48 * 48]
    small = [i for i in range(len(specs)) if i not in big]
    plan = batched.Plan([(big, 4, 256), (small, 1, 128)], "test split")
    r = batched.BatchedRunner(lats, plan)
    got = []
    for n in (30, 45):
        bufs = r.run(n)
        torch.cuda.synchronize()
        got.append(r.records_numpy(bufs, n))
    r.close()
    for i, s in enumerate(specs):
        rec = np.concatenate([got[0][i], got[1][i]])
        if i % 5 == 0:
            ref, s_ref = oracle_trajectory(s["dim"], s["L"], s["T"], s["seed"], 75)
            assert_records_equal(rec, ref, "replica %d vs oracle" % i)
            assert np.array_equal(lats[i].get_state()[0], s_ref)
        else:
            alone = w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"])
            assert_records_equal(rec, alone.step(75), "replica %d vs alone" % i)
            alone.close()
    for x in lats:
        x.close()


def test_autotune_returns_a_working_plan():
    torch, w = require_cuda()
    from paper_1110_0899_gb300 import batched
    specs = _small_specs(16)
    plan, table = batched.autotune(specs, probe_updates=8, use_cache=False)
    # both stages: team shapes and split, then window slots and levels per
    # round around the best
    assert len(table) >= len(batched.candidate_plans(specs)) + 4
    assert all(t["seconds"] is None or t["seconds"] > 0 for t in table)
    assert any("slots=128" in t["plan"] for t in table)
    assert any("levels=12" in t["plan"] for t in table)
    lats = [w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"]) for s in specs]
    r = batched.BatchedRunner(lats, plan)
    bufs = r.run(20)
    torch.cuda.synchronize()
    got = r.records_numpy(bufs, 20)
    r.close()
    for i, s in enumerate(specs):
        ref, _ = oracle_trajectory(s["dim"], s["L"], s["T"], s["seed"], 20)
        assert_records_equal(got[i], ref, "autotuned plan replica %d" % i)
        lats[i].close()


@pytest.mark.parametrize("variant", ["slots32", "slots128", "no_window", "levels12",
                                     "launches"])
def test_every_plan_dimension_keeps_the_chains(variant):
    """Each dimension the autotuner searches -- window slots per CTA, window
    mode off, growth levels per round, and the large lattices run as one
    default launch each beside a batched launch -- leaves every replica's
    records equal to the oracle's, over two calls."""
    torch, w = require_cuda()
    from paper_1110_0899_gb300 import batched
    specs = _small_specs(24)
    lats = [w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"]) for s in specs]
    big = [i for i, s in enumerate(specs) if s["L"] ** s["dim"] >= 48 * 48]
    small = [i for i in range(len(specs)) if i not in big]
    G = batched.Group
    groups = {
        "slots32": [G(big, 4, 256, slots=32), G(small, 1, 128, slots=32)],
        "slots128": [G(big, 2, 256, slots=128), G(small, 1, 256, slots=128)],
        "no_window": [G(big, 4, 256, slots=0), G(small, 1, 128, slots=0)],
        "levels12": [G(big, 4, 512, levels=12), G(small, 1, 128, levels=3)],
        "launches": [G(big, kind=batched.LAUNCHES), G(small, 1, 256)],
    }[variant]
    r = batched.BatchedRunner(lats, batched.Plan(groups, variant))
    got = []
    for n in (25, 35):
        bufs = r.run(n)
        torch.cuda.synchronize()
        got.append(r.records_numpy(bufs, n))
    r.close()
    for i, s in enumerate(specs):
        ref, s_ref = oracle_trajectory(s["dim"], s["L"], s["T"], s["seed"], 60)
        assert_records_equal(np.concatenate([got[0][i], got[1][i]]), ref,
                             "%s replica %d" % (variant, i))
        assert np.array_equal(lats[i].get_state()[0], s_ref)
        lats[i].close()


def test_served_requests_equal_their_runs_alone():
    """Requests of mixed size and dimension arrive while others run; each
    result equals the same request run alone."""
    torch, w = require_cuda()
    from paper_1110_0899_gb300 import serving, workloads
    trace = workloads.serving_trace(24, rate=400.0, l2d=(16, 200), l3d=(6, 24),
                                    updates=(50, 3000))
    srv = serving.WolffServer(epoch_updates=400, big_sites=1 << 12, big_team=(2, 256),
                              memory_budget=1 << 30)
    reqs, summary = srv.serve(trace)
    srv.close()
    assert summary["completed"] == len(trace)
    assert summary["epochs"] > 1
    overlapped = sum(1 for r in reqs if r.spec["n_updates"] > 400)
    assert overlapped > 0   # some requests spanned several epochs next to others
    for k, r in enumerate(reqs):
        s = r.spec
        alone = w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"])
        ref = alone.step(s["n_updates"])
        E, M, _ = alone.measure()
        alone.close()
        assert_records_equal(r.result["records"], ref, "request %d" % s["id"])
        assert (r.result["E_bond"], r.result["M"]) == (E, M)
        if k < 3:
            orc, _ = oracle_trajectory(s["dim"], s["L"], s["T"], s["seed"], s["n_updates"])
            assert_records_equal(r.result["records"], orc, "request %d vs oracle" % s["id"])


def test_time_budget_stops_at_update_boundaries():
    """A batch with a device-time budget runs a prefix of each lattice's
    updates; the chain continues exactly where it stopped."""
    torch, w = require_cuda()
    specs = [(2, 96, 2.0, 5), (3, 12, 4.0, 6), (2, 40, 2.3, 7)]
    lats = [w.WolffLattice(d, L, T, seed=s) for d, L, T, s in specs]
    for lat in lats:
        lat.set_state(np.ones(lat.N, np.int8), 0)   # ordered: large clusters, slow updates
    batch = w.WolffBatch(len(lats))
    got = [[] for _ in lats]
    seen = [0] * len(lats)
    for call in range(6):
        bufs = [lat.record_buffer(400) for lat in lats]
        batch.run(lats, 400, bufs, cluster_size=2, block_threads=256, budget_ns=30_000)
        torch.cuda.synchronize()
        for k, lat in enumerate(lats):
            ran = lat.stats()["updates"] - seen[k]
            seen[k] += ran
            assert 1 <= ran <= 400
            got[k].append(w.records_to_numpy(bufs[k], ran))
    assert any(sum(len(x) for x in g) < 6 * 400 for g in got)   # the budget did stop some
    for k, (dim, L, T, seed) in enumerate(specs):
        rec = np.concatenate(got[k])
        ref, s_ref = oracle_trajectory(dim, L, T, seed, len(rec), s=np.ones(L ** dim, np.int8))
        assert_records_equal(rec, ref, "budgeted lattice %d" % k)
        spins, t = lats[k].get_state()
        assert t == len(rec) and np.array_equal(spins, s_ref)
        lats[k].close()
    batch.close()
