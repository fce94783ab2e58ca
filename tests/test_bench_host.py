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
    bytes_ = 1000 * 150.0 * bench.BYTES_PER_FACE + 6000.0 * 24.0
    assert math.isclose(mem["bytes_per_launch"], bytes_)
    assert math.isclose(mem["frac"], bytes_ / 1e-3 / 6000.0e9)
    json.dumps({"roofline": roof, "memory_roofline": mem}, allow_nan=False)
