"""bench.py's host-side arithmetic, without a GPU: the cost table covers every
kernel class the library reports, the roofline entry is computed from it as
documented, and the clock sampler's parsing of nvidia-smi samples."""
import pytest

import bench

# kernel classes the library reports per family (fd_profile classes)
CLASSES = {"store_all": ["fused", "products", "deriv1", "deriv2"], "store_some": ["grad", "fused"],
           "recompute_all": ["fused"], "recompute_some": ["grad", "fused"], "store_none": ["fused"]}


@pytest.mark.parametrize("dtype", ["f64", "f32", "df64"])
@pytest.mark.parametrize("alg", bench.VARIANTS)
def test_cost_table_covers_every_reported_kernel(dtype, alg):
    for kclass in CLASSES[alg] + ["prims"]:
        c = bench.cost_of(dtype, alg, kclass)
        assert c is not None and len(c) == 3, (dtype, alg, kclass)
        flops, nbytes, instr = c
        assert flops > 0 and nbytes > 0 and instr >= 0
        if dtype != "f64":
            assert instr == 0  # binary32 and df64 steps issue no FP64 instructions


def test_binary64_flops_per_instruction_are_between_one_and_two():
    for alg in bench.VARIANTS:
        for kclass in CLASSES[alg]:
            flops, _, instr = bench.cost_of("f64", alg, kclass)
            assert instr <= flops <= 2 * instr, (alg, kclass)


def test_roofline_entry_for_binary64():
    n = 256**3
    kern = {"grad": {"ms_total": 12.5, "launches": 10, "ms_avg": 1.25},
            "fused": {"ms_total": 67.0, "launches": 10, "ms_avg": 6.7}}
    e = bench.roofline_of("f64", "store_some", kern, n, 6792.7, "measured")
    flops, nbytes, instr = bench.cost_of("f64", "store_some", "fused")
    sec = 6.7e-3
    assert e["kernel"] == "SS:fused" and e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["achieved"] == pytest.approx(flops * n / sec / 1e12, rel=1e-3)
    assert e["frac"] == pytest.approx(e["achieved"] / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert e["fp64_pipe_frac"] == pytest.approx(instr * n / sec / bench.FP64_PEAK_INSTR, rel=1e-3)
    assert e["hbm_achieved_gbs"] == pytest.approx(nbytes * n / sec / 1e9, rel=1e-3)
    assert e["share"] == pytest.approx(67.0 / 79.5, abs=1e-4)
    assert e["traffic"] == round(bench.TRAFFIC_BPP[("f64", "store_some", "fused")] * n)
    # the nominal FP64 peak: 152 SMs x 2 FMA lanes x 2 flop x 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.2586, abs=1e-4)


def test_roofline_entry_for_binary32_is_on_the_hbm_rate():
    n = 256**3
    kern = {"fused": {"ms_total": 7.0, "launches": 10, "ms_avg": 0.7}}
    e = bench.roofline_of("f32", "recompute_all", kern, n, 6792.7, "measured")
    _, nbytes, _ = bench.cost_of("f32", "recompute_all", "fused")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s" and e["peak"] == 6792.7
    assert e["achieved"] == pytest.approx(nbytes * n / 0.7e-3 / 1e9, rel=1e-3)
    assert e["frac"] == pytest.approx(e["achieved"] / 6792.7, rel=1e-3)
    assert e["share"] == 1.0
    e = bench.roofline_of("f32", "store_some", {"fused": kern["fused"]}, n, 6800.0, "fallback")
    assert e["traffic"] == round(bench.TRAFFIC_BPP[("f32", "store_some", "fused")] * n)
    assert e["peak_source"] == "fallback"


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _row(ts, sm, reasons=("Not Active",) * 4):
    return ", ".join([ts, "0", str(sm), "2070", "900.0", "0x0"] + list(reasons))


def test_clock_sampler_reads_the_timed_windows_only():
    import datetime as dt
    c = bench.ClockSampler()
    t = lambda s: dt.datetime(2026, 1, 1, 0, 0, s).timestamp()  # noqa: E731
    lines = [_row("2026/01/01 00:00:01.000", 1200),
             _row("2026/01/01 00:00:05.000", 2070),
             _row("2026/01/01 00:00:06.000", 2065, ("Not Active", "Not Active", "Not Active", "Active")),
             _row("2026/01/01 00:00:07.000", 2070),
             _row("2026/01/01 00:00:20.000", 900, ("Active", "Not Active", "Not Active", "Not Active")),
             "garbage line"]
    c.proc = _FakeProc("\n".join(lines))
    c.mark(t(4), t(8))
    r = c.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the window


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler()
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_roofline_entry_for_the_mixed_kernel_is_on_the_issue_slots():
    n = 256**3
    kern = {"grad": {"ms_total": 3.5, "launches": 10, "ms_avg": 0.35},
            "fused": {"ms_total": 36.0, "launches": 10, "ms_avg": 3.6}}
    e = bench.roofline_of("f64dw", "store_some", kern, n, 6787.2, "measured", fp64_peak=1.25)
    sec = 3.6e-3
    flops, nbytes, instr = bench.cost_of("f64dw", "store_some", "fused")
    assert e["bound"] == "alu" and e["unit"] == "Tinst/s"
    assert e["peak"] == pytest.approx(152 * 4 * 32 * 2.07e9 / 1e12, rel=1e-3)
    assert e["achieved"] == pytest.approx(bench.ISSUE_COST[("f64dw", "store_some", "fused")] * n / sec / 1e12,
                                          rel=1e-3)
    assert e["frac"] == pytest.approx(e["achieved"] / e["peak"], rel=1e-3)
    assert e["binary64_equivalent_tflops"] == pytest.approx(flops * n / sec / 1e12, rel=1e-3)
    assert e["fp64_pipe_frac"] == pytest.approx(instr * n / sec / (1.25e12 / 2), rel=1e-3)
    assert e["hbm_frac"] == pytest.approx(nbytes * n / sec / 1e9 / 6787.2, rel=1e-3)
    # the measured binary64 peak replaces the nominal one for the binary64 families
    e64 = bench.roofline_of("f64", "store_some", kern, n, 6787.2, "measured", fp64_peak=1.25)
    assert e64["peak"] == 1.25 and "measured" in e64["peak_source"]


@pytest.mark.parametrize("dtype", ["f64", "f32", "df64"])
@pytest.mark.parametrize("alg", bench.VARIANTS)
def test_every_reported_kernel_has_measured_traffic(dtype, alg):
    for kclass in CLASSES[alg]:
        bpp = bench.TRAFFIC_BPP.get((dtype, alg, kclass))
        assert bpp is not None and bpp > 0, (dtype, alg, kclass)
        # measured traffic stays within a factor of the algorithmic bytes
        _, nbytes, _ = bench.cost_of(dtype, alg, kclass)
        assert 0.4 * nbytes <= bpp <= 1.5 * nbytes, (dtype, alg, kclass, bpp, nbytes)
