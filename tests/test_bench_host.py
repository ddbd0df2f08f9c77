"""Host-side checks of bench.py (no GPU): the DRAM traffic it reports for the
fused kernel belongs to the kernel source it was measured on, and scales with
the shots of a launch."""
import importlib

import pytest


@pytest.fixture()
def bench():
    return importlib.import_module("bench")


def test_traffic_follows_the_source_hash(bench, monkeypatch):
    h = bench._sources_sha256()
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", {"shots": 1_000_000, "bytes": 300_000_000, "sources_sha256": h})
    assert bench._fused_traffic(1_000_000) == pytest.approx(300_000_000)
    assert bench._fused_traffic(500_000) == pytest.approx(150_000_000)
    # a capture taken on other sources is not reported
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", {"shots": 1_000_000, "bytes": 300_000_000, "sources_sha256": "0" * 64})
    assert bench._fused_traffic(1_000_000) is None
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", {"shots": 1_000_000, "bytes": None, "sources_sha256": h})
    assert bench._fused_traffic(1_000_000) is None


def test_source_hash_covers_the_kernel_sources(bench, tmp_path):
    a, b = tmp_path / "a.cu", tmp_path / "b.h"
    a.write_text("x")
    b.write_text("y")
    h0 = bench._sources_sha256((str(a), str(b)))
    b.write_text("z")
    assert bench._sources_sha256((str(a), str(b))) != h0


def test_clock_sampler_keeps_the_timed_region(bench, tmp_path):
    """Only samples whose timestamps fall inside the timed region count; a
    throttle reason seen outside it is not reported."""
    import datetime

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    t0 = 1_800_000_000.0
    path = tmp_path / "clocks.csv"
    rows = []
    for k, (mhz, pcap) in enumerate([(1500, "Active"), (2070, "Not Active"), (2060, "Not Active"),
                                     (2070, "Not Active"), (1400, "Active")]):
        ts = datetime.datetime.fromtimestamp(t0 + 0.1 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        rows.append(f"{ts}, 0, {mhz}, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, {pcap}")
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path, cs.fh = Done(), str(path), open(tmp_path / "unused", "w")
    got = cs.stop(window=(t0 + 0.1, t0 + 0.3))
    assert got["samples"] == 3 and got["sm_mhz"] == 2070 and got["reasons"] == []
    assert got["scope"] == "timed region"


def test_cpu_baseline_runs_in_a_child_process(bench):
    """The oracle's timing runs in its own process, on one thread and on all
    host cores, and reports both."""
    r = bench._cpu_baseline(budget_s=0.5)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    assert r["all_cores"]["cores"] >= 1 and r["all_cores"]["value"] > 0
