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
