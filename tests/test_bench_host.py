"""Host-side pieces of the benchmark (no GPU): the config description of every workload
is plain JSON (no infinities), and the roofline arithmetic follows its stated formulas."""
import json
import math

import bench
import synth


class _FakeCtx:
    def fma_peak(self, precision):
        return 1.0e12


class _FakeCss:
    FP32, FP64 = 1, 0


def test_every_workload_describes_itself_as_plain_json():
    for name in synth.CONFIG_NAMES:
        cfg = synth.make_config(name)
        d = bench.describe(cfg, 1)
        s = json.dumps(d, allow_nan=False)          # raises on inf / nan
        assert d["workload"] == name and "Infinity" not in s
        assert d["n_particles"] > 0


def test_roofline_arithmetic():
    pk = {"sm_max_mhz": 2000.0, "hbm_gbs": 6000.0}
    roof, mem = bench.roofline(_FakeCss, _FakeCtx(), pk, props_per_src=300.0, n=1000, pairs_per_launch=6000.0,
                               kern_s=1e-3, kernel_name="k", traffic=1.5e7)
    flops = 1000 * 300.0 * bench.FLOPS_PER_PROPAGATION + 6000.0 * bench.FLOPS_PER_PAIR
    peak = 152 * 128 * 2 * 2000.0e6
    assert math.isclose(roof["achieved"], flops / 1e-3 / 1e12)
    assert math.isclose(roof["peak"], peak / 1e12)
    assert math.isclose(roof["frac"], flops / 1e-3 / peak)
    assert roof["traffic"] == 1.5e7 and roof["bound"] == "alu"
    # per source: faces reached (half the propagations) x 64 B + 48 B per propagated window
    # + its 24 B force; 20 B per pair
    bytes_ = 1000 * (150.0 * 64.0 + 300.0 * 48.0 + 24.0) + 6000.0 * 20.0
    assert math.isclose(mem["bytes_per_launch"], bytes_)
    assert math.isclose(mem["frac"], bytes_ / 1e-3 / 6000.0e9)
    assert math.isclose(mem["traffic_over_algorithmic"], 1.5e7 / bytes_)
    json.dumps({"roofline": roof, "memory_roofline": mem}, allow_nan=False)


def test_traffic_is_dropped_when_the_kernel_changed(monkeypatch):
    """A stored DRAM figure is scaled to the launch's sources, and reported only while the
    kernel sources still have the digest it was captured on."""
    monkeypatch.setattr(bench, "TRAFFIC", {"w": {"bytes": 8.0e8, "sources": 8192, "kernel": bench.kernel_digest()}})
    assert math.isclose(bench.traffic_per_launch("w", 65536), 6.4e9)
    assert bench.traffic_per_launch("other", 10) is None
    monkeypatch.setattr(bench, "TRAFFIC", {"w": {"bytes": 8.0e8, "sources": 8192, "kernel": "0" * 16}})
    assert bench.traffic_per_launch("w", 65536) is None
