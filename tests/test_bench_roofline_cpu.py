"""bench.py's roofline objects for every reconstruction path, assembled on the
CPU (the two device queries are stood in for): the keys the JSON line carries,
finite fractions, and the bound each path reports."""
import math

import pytest
import torch

import bench


class _Props:
    multi_processor_count = 152


class _Tcp:
    def __init__(self, kernel):
        self.kernel = kernel

    def get_backproject_config(self, *args):
        return (8, 16, 4, self.kernel)


@pytest.mark.parametrize("path,kernel,bound", [
    ("f32", 1, "alu"), ("f16", 1, "alu"), ("bf16", 1, "alu"), ("f16", 3, "alu"), ("bf16", 3, "alu"),
    ("f32_cuda", 0, "alu"), ("f32_frec", 0, "alu"), ("f16_frec", 0, "alu")])
def test_roofline_object(monkeypatch, path, kernel, bound):
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: _Props())
    r = bench.bp_roofline(_Tcp(kernel), None, path, 256, 2048, 2048, 175.0)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r, key
    assert r["bound"] == bound
    assert math.isfinite(r["frac"]) and r["frac"] > 0
    if path in bench.FOURIERREC:
        assert r["window_width"] == bench.FOURIERREC[path]
    else:
        # every LineRec path: frac = interpolations/s against the FP32 FMA
        # ceiling (2 FP32 operations per interpolation), whichever kernel runs
        clk = float(bench._peaks().get("sm_max_mhz", 2070.0))
        ceiling = 152 * 128 * clk * 1e6 / 2
        assert r["unit"] == "Ginterp/s"
        assert r["peak"] == pytest.approx(ceiling / 1e9, rel=1e-12)
        interps = 256 * 2048 * 2048 * 2048
        assert r["achieved"] == pytest.approx(interps / 0.175 / 1e9, rel=1e-12)
        assert r["frac"] == pytest.approx(interps / 0.175 / ceiling, rel=1e-12)
        if kernel in (1, 3):  # tensor cores: the dense MMA utilisation is a separately named diagnostic
            assert 0 < r["mma_frac_of_bf16_peak"] < 10
        else:
            assert 0 < r["frac_of_smem_roof"] < 10
