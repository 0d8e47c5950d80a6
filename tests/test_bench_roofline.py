"""bench.py's roofline object, from per-class timings of a profiled step (host arithmetic, no GPU): the
dominant class, the achieved bandwidth and its fraction of the peak, the two facet-sweep kernels counted as
one class with per-kernel parts, and the packed-triangle fraction."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SIZES = SimpleNamespace(ne=196608, nint=387072, n_c=48, mF=12, ncolours=4)


def _cls(launches, ms, bytes_, flops=0.0):
    return {"launches": launches, "ms": ms, "bytes": bytes_, "flops": flops}


def test_sweep_kernels_count_as_one_class():
    per = 520.2e6
    stats = {"condense": _cls(1, 327.0, 3.9e9, 186e9),
             "facet_gs_step": _cls(100, 100 * 0.0860, 100 * per),
             "facet_push": _cls(100, 100 * 0.0920, 100 * per),
             "apply_K": _cls(156, 133.0, 156 * 2.44e9)}
    roof = bench._roofline(stats, SIZES, 6789.3, "measured")
    # with 100 launches each the two sweep kernels (17.8 ms together) stay below the 327 ms
    # condensation, which is then the dominant class
    assert roof["kernel"] == "condense" and roof["bound"] == "alu"
    stats["facet_gs_step"] = _cls(2544, 2544 * 0.0860, 2544 * per)
    stats["facet_push"] = _cls(2544, 2544 * 0.0920, 2544 * per)
    roof = bench._roofline(stats, SIZES, 6789.3, "measured")
    assert roof["kernel"].startswith("facet_gs_step") and roof["bound"] == "hbm"
    avg_us = (0.0860 + 0.0920) / 2 * 1e3
    assert roof["avg_launch_us"] == pytest.approx(avg_us, abs=0.01)
    assert roof["achieved"] == pytest.approx(per / (avg_us * 1e-6) / 1e9, rel=1e-4)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6789.3, abs=1e-4)
    parts = roof["parts"]
    assert parts["row_products"]["frac"] == pytest.approx(per / 86e-6 / 1e9 / 6789.3, abs=1e-4)
    assert parts["push"]["frac"] == pytest.approx(per / 92e-6 / 1e9 / 6789.3, abs=1e-4)
    s8 = 4.0 * (SIZES.ne * 48 * 49 / 2 + SIZES.nint * 144) / 4
    assert roof["s8d_bytes_per_launch"] == pytest.approx(s8)
    assert roof["layout_over_s8d"] == pytest.approx(per / s8, abs=1e-3)
    # traffic: the launch-weighted mean of the committed per-kernel summaries, when both exist
    t_rows, t_push = bench._traffic("facet_gs_step", bench.HEADLINE), bench._traffic("facet_push", bench.HEADLINE)
    if t_rows is not None and t_push is not None:
        assert roof["traffic"] == pytest.approx((t_rows + t_push) / 2)


def test_single_sweep_kernel_has_no_parts():
    stats = {"facet_gs_step": _cls(10, 10 * 0.025, 10 * 97e6), "apply_K": _cls(1, 0.1, 0.46e9)}
    roof = bench._roofline(stats, SIZES, 6789.3, "measured")
    assert roof["kernel"] == "facet_gs_step" and "parts" not in roof
    assert roof["frac"] == pytest.approx(97e6 / 25e-6 / 1e9 / 6789.3, abs=1e-4)
