"""bench.py's host side on CPU: the command line the driver and the profile
recipes use, and the capture bookkeeping behind the roofline's traffic."""
import re
import sys

import pytest


@pytest.fixture
def bench():
    import bench as b
    return b


def parse(bench, monkeypatch, argv):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench.parse()


def test_driver_command_lines(bench, monkeypatch):
    a = parse(bench, monkeypatch, [])
    assert (a.gpus, a.workload, a.impl) == (1, "2d", "gb300") and a.warmup >= 3
    a = parse(bench, monkeypatch, ["--impl", "reference", "--gpus", "1", "--steps", "2",
                                   "--warmup", "3"])
    assert a.impl == "reference" and a.steps == 2


def test_workloads_of_the_profiles_and_design_notes(bench, monkeypatch):
    a = parse(bench, monkeypatch, ["--workload", "small", "--steps", "3", "--warmup", "3"])
    assert a.workload == "small"
    a = parse(bench, monkeypatch, ["--workload", "tiny-sizes", "--sizes", "3:32,2:16",
                                   "--temps", "1.0", "--regimes", "random"])
    assert a.sizes == "3:32,2:16" and a.temps == "1.0" and a.regimes == "random"
    a = parse(bench, monkeypatch, ["--workload", "served", "--serve-seconds", "30",
                                   "--epoch-ms", "10", "--no-tiny-engine"])
    assert a.epoch_ms == 10.0 and a.no_tiny_engine
    for w in ("2d", "3d", "2d-eq", "3d-eq", "batched", "binder", "xy-2d", "potts3-2d"):
        assert parse(bench, monkeypatch, ["--workload", w]).workload == w
    with pytest.raises(SystemExit):
        parse(bench, monkeypatch, ["--workload", "no-such-workload"])


def test_capture_bookkeeping(bench):
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{12}", h)
    for key, cap in bench.TRAFFIC_CAPTURES.items():
        assert key[0] in bench.WORKLOADS and key[1] > 0
        assert re.fullmatch(r"[0-9a-f]{12}", cap["src"])
        # every DRAM byte passes through L2
        assert 0 < cap["bytes_per_launch"] <= cap["l2_bytes_per_launch"]
        im = cap["imad"]
        assert 0 < im["pipe_frac_gpu"] <= im["pipe_frac_active_sms"] < 1
