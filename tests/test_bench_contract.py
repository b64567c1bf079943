"""The benchmark's JSON fields that are pure arithmetic, checked on the CPU:
the U-Net's FLOP count and the roofline object built from kernel times."""
import math

import bench


def test_unet_flops_by_hand():
    # 3x3 convolutions per level (H, W halve per level): 2 H W Cout 9 Cin each,
    # plus the 1x1 head; the 1024^2, 32-64-128-256 network is ~357 GFLOP.
    H = W = 1024
    convs = [(0, 32, 32), (0, 32, 32), (1, 64, 32), (1, 64, 64), (2, 128, 64), (2, 128, 128), (3, 256, 128),
             (3, 256, 256), (2, 128, 384), (2, 128, 128), (1, 64, 192), (1, 64, 64), (0, 32, 96), (0, 32, 32)]
    want = sum(2 * (H >> l) * (W >> l) * co * ci * 9 for l, co, ci in convs) + 2 * H * W * 4 * 32
    assert bench.unet_flops(H, W) == want
    assert abs(want / 1e9 - 357.4) < 0.5
    # executed by the BF16 network: each decoder block's first convolution over [up2(d) | e]
    # takes 9 taps of the skip channels and 4 of the low-resolution ones per output pixel
    sub = [(l, co, cs, cu) for l, co, cs, cu in ((2, 128, 128, 256), (1, 64, 64, 128), (0, 32, 32, 64))]
    plain = sum(2 * (H >> l) * (W >> l) * co * (cs + cu) * 9 for l, co, cs, cu in sub)
    subp = sum(2 * (H >> l) * (W >> l) * co * (cs * 9 + cu * 4) for l, co, cs, cu in sub)
    assert bench.unet_flops(H, W, subpixel=True) == want - plain + subp


def test_roofline_of_the_convolutions():
    frames = 10
    kt = {"conv_tc": (14 * frames, 14 * frames * 0.05), "composite_skip": (2 * frames, 0.3 * frames)}
    peaks = {"hbm_gbs": 6783.5, "bf16_tflops_sustained": 1713.7}
    r = bench.roofline(kt, {"instances": 900000}, peaks, "bf16_skip", 1000000, 32, frames)
    per_launch = bench.unet_flops(1024, 1024, subpixel=True) / 14  # (the BF16 network executes the sub-pixel form)
    assert r["flops_plain_definition"] == bench.unet_flops(1024, 1024)
    assert math.isclose(r["frac_plain_definition"] / r["frac"], bench.unet_flops(1024, 1024) / (per_launch * 14))
    assert r["kernel"] == "conv_tc" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], per_launch / 0.05e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / 1713.7, rel_tol=1e-12)
    assert r["peak_is"] == "measured sustained BF16"
    from paper_2202_05628_gb300.profile_capture import committed_traffic
    assert r["traffic"] == committed_traffic()  # the committed capture's figure, or None once the sources changed
    # the back-to-back launch time replaces the event time when given, against the burst peak
    peaks_b = dict(peaks, bf16_tflops=1934.1)
    r2 = bench.roofline(kt, {"instances": 900000}, peaks_b, "bf16_skip", 1000000, 32, frames, conv_launch_ms=0.04)
    assert math.isclose(r2["avg_ms"], 0.04) and math.isclose(r2["achieved"], per_launch / 0.04e-3 / 1e12)
    assert r2["peak"] == 1934.1 and r2["peak_is"] == "measured burst BF16"
    # no measured peaks: the fallback figures, labelled so
    r3 = bench.roofline(kt, {"instances": 900000}, {}, "bf16_skip", 1000000, 32, frames)
    assert r3["peak"] == 1700.0 and r3["peak_is"].startswith("fallback")
    # the FP8 form against twice the BF16 peak
    r4 = bench.roofline(kt, {"instances": 900000}, peaks, "fp8", 1000000, 32, frames)
    assert math.isclose(r4["peak"], 2 * 1713.7) and r4["traffic"] is None


def test_roofline_of_a_bandwidth_bound_kernel():
    kt = {"lbs": (10, 10 * 0.035)}
    r = bench.roofline(kt, {"instances": 900000}, {"hbm_gbs": 6783.5}, "bf16_skip", 1000000, 32, 10)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], 1000000 * 160 / 0.035e-3 / 1e9, rel_tol=1e-12)
    assert r["peak_is"] == "measured copy bandwidth"
    assert bench.roofline({}, {}, {}, "bf16_skip", 1, 32, 1) is None


def test_clock_summary_of_sampled_lines():
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 1965, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2010, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = cs.summary()
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.lines = ["0, 1200, 2070, 700, 0x8, Not Active, Active, Not Active, Not Active"]
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown"]
    cs.lines = []
    assert cs.summary()["reasons"] == ["unsampled"]


def test_step_schedule_covers_every_pose_and_azimuth():
    seen = {bench.step_indices(k) for k in range(bench.N_POSES * bench.N_AZ)}
    assert {p for p, _ in seen} == set(range(bench.N_POSES))
    assert {v for _, v in seen} == set(range(bench.N_AZ))
    # consecutive steps change both the pose and the view
    for k in range(50):
        a, b = bench.step_indices(k), bench.step_indices(k + 1)
        assert a[0] != b[0] and a[1] != b[1]


def test_quality_psnr():
    import numpy as np
    ref = np.zeros((4, 4, 4))
    q = bench.quality(ref + 0.01, ref)
    assert math.isclose(q["psnr_db"], 40.0, rel_tol=1e-12) and math.isclose(q["max_abs"], 0.01)


def test_composite_roofline_sums_its_kernels():
    frames = 4
    kt = {"composite_skip": (4, 4 * 0.15), "composite_merge": (4, 4 * 0.03), "conv_tc": (56, 2.4)}
    r = bench.composite_roofline(kt, {"instances": 900000}, {"hbm_gbs": 6783.5}, "bf16_skip", 32, frames)
    byts = 900000 * (8 + 64 + 8 + 64) + 1024 * 1024 * (64 + 4)
    assert r["kernels"] == ["composite_skip", "composite_merge"]
    assert math.isclose(r["ms_per_frame"], 0.18) and r["bytes_per_frame"] == byts
    assert math.isclose(r["frac"], byts / 0.18e-3 / 1e9 / 6783.5, rel_tol=1e-12)
    assert bench.composite_roofline({}, {"instances": 1}, {}, "bf16", 32, 1) is None
