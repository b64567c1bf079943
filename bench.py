"""Frame-rate benchmark of the GB300 ARTEMIS rendering path.

One step = one frame of one view: pose -> LBS warp of ~1M leaf voxels ->
screen-tile binning (by tile, then by depth) -> exact-hit front-to-back compositing of
F (32 channels) and A at 1024x1024 -> 4-level U-Net shading -> RGBA.
Poses follow a 60-frame walk cycle; the camera orbits 8 azimuths.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(the path has no exchange step): value = frames of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s @1M voxels 1024²: BF16+learned-skip vs FP32 plain, PSNR≥45dB vs FP64"
WORKLOAD = "1M-voxel quadruped octree (depth 10, C=32), 1024x1024 view, 4-level U-Net 32-64-128-256"
RES = 1024
N_AZ = 8
N_POSES = 60
PROPOSAL = os.path.join(ROOT, "paper_2202_05628_gb300", "weights", "proposal_quadruped_1m_1024.bin")
# form -> (feature storage, shading network dtype, learned skip, description)
FORMS = {
    "bf16_skip": ("bf16", "bf16", True, "BF16 features + learned interval skip + BF16 tensor-core U-Net"),
    "bf16": ("bf16", "bf16", False, "BF16 features + BF16 tensor-core U-Net (plain traversal)"),
    "f32": ("f32", "f32", False, "FP32 plain"),
    "fp8": ("bf16", "fp8", True, "BF16 features + learned interval skip + FP8-E4M3 tensor-core U-Net"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--form", default="bf16_skip", choices=list(FORMS))
    p.add_argument("--f32-steps", type=int, default=16, help="steps of the FP32 plain form measured beside")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--segment", type=int, default=256, help="list entries per composite segment")
    p.add_argument("--no-kernel-events", action="store_true", help="time frames without per-kernel events")
    p.add_argument("--side-steps", type=int, default=16,
                   help="frames of the FP8 form and of the backward pass measured beside")
    return p.parse_args()


# ---------------------------------------------------------------- workload

def workload():
    import scenegen as sg
    sc = sg.preset("paper")
    cams = [sg.orbit_camera(sc.centroid, RES, RES, az_deg=45.0 * k) for k in range(N_AZ)]
    poses = [sg.walk_pose(f, N_POSES) for f in range(N_POSES)]
    layers = sg.unet_weights(0, cin=sc.octree.C)
    return sc, cams, poses, layers


def step_indices(k):
    return k % N_POSES, (k // N_POSES + k) % N_AZ


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

def proposal_params(sc, cams):
    """Weights of the ray-interval proposal for this workload: the committed
    file, else trained now from the renderer's own labels (a smaller run)."""
    from paper_2202_05628_gb300 import proposal as prop
    if os.path.exists(PROPOSAL):
        return prop.load(PROPOSAL)[0]
    import scenegen as sg
    print("bench: proposal weights missing, training a small one", file=sys.stderr)
    r = setup_renderer(sc, cams, None, "bf16")
    X, Y = prop.collect(r, [sg.random_pose(k) for k in range(400)], list(range(len(cams))), cams, 4096,
                        views_per_pose=2)
    r.close()
    return prop.train(X, Y, steps=1500, batch=16384)


SEGMENT = 256


def configure(r, form, profile):
    r.set_config(tau=1e-4, profile=profile, skip=int(FORMS[form][2]), max_missed=1e-3, margin=1, segment=SEGMENT)


def setup_renderer(sc, cams, layers, form, profile=False, proposal=None):
    import paper_2202_05628_gb300 as art
    storage, net, skip, _ = FORMS[form]
    oc = sc.octree
    r = art.Renderer()
    r.load_octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, oc.features, oc.density, storage)
    r.load_skeleton(sc.skeleton.parent, sc.skeleton.rest)
    if layers is not None:
        r.load_shader(art.ART_NET_UNET, oc.C, [32, 64, 128, 256], 4, art.flat_params(layers), net)
    if skip:
        r.load_proposal(proposal if proposal is not None else proposal_params(sc, cams))
    configure(r, form, profile)
    for v, c in enumerate(cams):
        r.set_camera(v, c.W, c.H, c.fx, c.fy, c.cx, c.cy, c.world_to_cam, c.near, c.far)
    return r


def run_steps(r, poses, steps, warmup, flush, stream, rgba):
    """Warm-up, then `steps` frames timed one by one with CUDA events on the
    library's stream; the L2 is flushed between frames outside the events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(warmup):
        pi, vi = step_indices(k)
        p = poses[pi]
        r.render_frame(vi, p.axis_angle, p.R, p.T, rgba)
    torch.cuda.synchronize()
    return ev


def timed_region(r, poses, steps, warmup, flush, rgba):
    import torch
    stream = torch.cuda.current_stream()
    ev = run_steps(r, poses, steps, warmup, flush, stream, rgba)
    r.kernel_times(reset=True)
    l0 = r.sync_status()["kernel_launches"]
    for k in range(steps):
        pi, vi = step_indices(warmup + k)
        p = poses[pi]
        flush.zero_()
        ev[k][0].record(stream)
        r.render_frame(vi, p.axis_angle, p.R, p.T, rgba)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    launches = r.sync_status()["kernel_launches"] - l0
    return ms, launches


def unet_ms(r, view, C, rgba, flush, reps=20, warmup=3):
    """Mean CUDA-event time of the shading network on the current frame's
    feature map, called back to back (its launches queued without per-kernel
    events; the L2 flushed between calls outside the events)."""
    import torch
    stream = torch.cuda.current_stream()
    F = torch.empty((RES, RES, C), dtype=torch.bfloat16, device="cuda")
    A = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    r.render_feature_maps(view, F, A, "bf16")
    for _ in range(warmup):
        r.shade(view, F, rgba, "bf16")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        r.shade(view, F, rgba, "bf16")
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def roofline(kt, stats, peaks, form, n_vox, C, frames, conv_launch_ms=None):
    """Achieved rate of the dominant kernel from its measured launch times.
    Algorithmic work: U-Net FLOPs per frame spread over the convolution
    launches of a frame; composite bytes = per instance (key, value, 64-B
    unit-cube record, pixel rectangle, feature row) + per pixel (F row, A).
    For the convolutions the launch time is the shading network's back-to-back
    time over its launches (conv_launch_ms) when given: per-kernel events
    leave the GPU waiting on the host between those short launches."""
    storage, net, _, _ = FORMS[form]
    if not kt:
        return None
    name, (nl, tot) = max(kt.items(), key=lambda kv: kv[1][1])
    avg_ms = tot / max(nl, 1)
    out = {"kernel": name, "launches": nl, "avg_ms": avg_ms}
    if name.startswith("conv") and conv_launch_ms:
        avg_ms = conv_launch_ms
        out.update(avg_ms=avg_ms, avg_ms_from="shading network called back to back, time / its 14 "
                   "convolution launches (its one pooling launch included)")
    if name.startswith("conv"):
        # the FLOPs the network executes (BF16: the sub-pixel decoder convolution at level 0)
        flops = unet_flops(RES, RES, subpixel=(net == "bf16"))
        per_launch = flops * frames / max(nl, 1)
        out.update(flops_per_frame=flops, flops_plain_definition=unet_flops(RES, RES))
        ach = per_launch / (avg_ms * 1e-3) / 1e12
        # measured peaks of MEASURED_PEAKS.json, else the profiling recipe's fallback figures: the
        # burst figure, since the launch time comes from the network called back to back in isolation
        # (a ~12 ms loop); the sustained one where the per-kernel events of the whole frame give it
        isolated = bool(conv_launch_ms)
        key = "bf16_tflops" if isolated else "bf16_tflops_sustained"
        src = "measured" if key in peaks else "fallback"
        bf16 = peaks.get(key, 1900.0 if isolated else 1700.0)
        kind = "burst" if isolated else "sustained"
        if net == "f32":
            peak, bound, note = 2.0 * 152 * 128 * 2.07e9 / 1e12, "alu", "FP32 FMA issue rate of the CUDA cores"
        elif net == "fp8":
            peak, bound, note = 2.0 * bf16, "tensor", f"{src} {kind} BF16 x 2 (nominal FP8 / BF16 ratio)"
        else:
            peak, bound, note = bf16, "tensor", f"{src} {kind} BF16"
        # DRAM reads + writes per launch of the BF16 convolutions from the committed ncu capture
        # (paper_2202_05628_gb300/profile_capture.py), while it matches the current sources
        traffic = None
        if net == "bf16":
            from paper_2202_05628_gb300.profile_capture import committed_traffic
            traffic = committed_traffic()
        out.update(bound=bound, achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=traffic, peak_is=note)
        if flops != out["flops_plain_definition"]:  # the same launches credited with the plain definition's FLOPs
            out["frac_plain_definition"] = ach * out["flops_plain_definition"] / flops / peak
    else:
        fb = 2 if storage == "bf16" else 4
        inst = stats["instances"]
        per_inst = 4 + 4 + 64 + 8 + C * fb
        byts = inst * per_inst + RES * RES * (C * fb + 4)
        if name == "lbs":
            byts = n_vox * 160
        ach = byts / (avg_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out.update(bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak, traffic=None,
                   peak_is=("measured" if "hbm_gbs" in peaks else "fallback") + " copy bandwidth")
    return out


COMPOSITE_KERNELS = ("composite", "composite_skip", "composite_merge", "composite_clear", "composite_plan",
                     "composite_fallback", "composite_exact")


def composite_roofline(kt, stats, peaks, form, C, frames):
    """The composite stage as one unit: the summed per-frame time of its
    kernels (interval / plain walk, merge, clear, plan, sequential and
    exact walks) against its algorithmic bytes per frame: per instance the
    key and value (8 B), the 64-B voxel record, the 8-B pixel rectangle and
    the feature row (C x 2 B BF16 / 4 B FP32), each read once; per pixel the
    F row and A written once."""
    storage = FORMS[form][0]
    fb = 2 if storage == "bf16" else 4
    ms = sum(kt[k][1] for k in COMPOSITE_KERNELS if k in kt) / max(frames, 1)
    if ms <= 0:
        return None
    byts = stats["instances"] * (8 + 64 + 8 + C * fb) + RES * RES * (C * fb + 4)
    ach = byts / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"kernels": [k for k in COMPOSITE_KERNELS if k in kt], "ms_per_frame": ms, "bytes_per_frame": byts,
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_is": ("measured" if "hbm_gbs" in peaks else "fallback") + " copy bandwidth",
            "note": "per-kernel CUDA-event times of the second timed pass (events add gaps between launches)"}


def unet_flops(H, W, cin=32, ch=(32, 64, 128, 256), subpixel=False):
    """FLOPs of the 4-level U-Net on an H x W map.  subpixel: as the BF16
    tensor-core network executes it, each decoder block's first convolution
    over [up2(d) | e] in its sub-pixel form (the upsampled part through 4
    taps per output pixel instead of 9)."""
    import scenegen as sg
    tot = 0
    shapes = sg.unet_layer_shapes(cin, ch)
    lvl = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0]
    for idx, ((co, ci, k), l) in enumerate(zip(shapes, lvl)):
        if subpixel and idx in (8, 10, 12):
            tot += 2 * (H >> l) * (W >> l) * co * (9 * ch[l] + 4 * ch[l + 1])
        else:
            tot += 2 * (H >> l) * (W >> l) * co * ci * k * k
    return tot


def backward_timing(sc, cams, poses, layers, steps, flush, warmup=3):
    """Per-frame time of art_render_backward (dL/df, dL/dsigma, dL/dw of the
    F and A maps) on the workload, BF16 feature storage, with a dense random
    upstream gradient (every pixel traced again); the forward maps and the
    zeroing of the gradient buffers are outside the events."""
    import torch
    oc = sc.octree
    r = setup_renderer(sc, cams, layers, "bf16", profile=True)
    g = torch.Generator(device="cuda").manual_seed(7)
    Fm = torch.empty((RES, RES, oc.C), dtype=torch.float32, device="cuda")
    Am = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    dF = torch.randn((RES, RES, oc.C), generator=g, device="cuda") * 1e-3
    dA = torch.randn((RES, RES), generator=g, device="cuda") * 1e-3
    df = torch.zeros((oc.n, oc.C), dtype=torch.float32, device="cuda")
    ds = torch.zeros(oc.n, dtype=torch.float32, device="cuda")
    dw = torch.zeros((oc.n, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(warmup + steps):
        if k == warmup:
            r.kernel_times(reset=True)
        pi, vi = step_indices(k)
        p = poses[pi]
        r.set_pose(p.axis_angle, p.R, p.T)
        r.render_feature_maps(vi, Fm, Am, "f32")
        df.zero_(), ds.zero_(), dw.zero_(), flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.render_backward(vi, Fm, Am, dF, dA, df, ds, dw)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
    kt = r.kernel_times(reset=True)
    r.close()
    return {"ms_per_frame": float(np.mean(ms)), "frames_per_s": 1e3 / float(np.mean(ms)), "steps": steps,
            "kernels_ms": {k: round(v[1] / steps, 4) for k, v in kt.items() if "bwd" in k},
            "what": "dL/df, dL/dsigma, dL/dw through the F and A maps, dense upstream gradient"}


STEREO = (1920, 1080, 0.032)  # stereo VR pair: two 1920x1080 eyes, 6.4 cm baseline (camera offsets of +-3.2 cm)


def stereo_cams(sc, az_index):
    import scenegen as sg
    W, H, b = STEREO
    return [sg.orbit_camera(sc.centroid, W, H, az_deg=45.0 * az_index, shift_x=s) for s in (-b, b)]


def stereo_timing(sc, poses, layers, prop, flush, steps, warmup=3, oracle_psnr=True):
    """Stereo frames (both eyes of one pose) of the 1M-voxel octree at
    1920x1080 per eye: pose, both eyes' F and A maps, the U-Net on each.
    Forms: the BF16 plain traversal with both eyes in one pass
    (art_render_views: one tile space, one scan, scatter, sort and composite
    walk) and the same as two single-view passes; BF16 + learned skip (per
    eye); FP32 plain.  Cameras are set per frame (an orbit azimuth per step,
    as a moving head would); CUDA events around each stereo frame, the L2
    flushed between frames outside them."""
    import torch
    import paper_2202_05628_gb300 as art
    W, H, _ = STEREO
    oc = sc.octree
    out = {"resolution": [W, H], "baseline_m": 2 * STEREO[2], "steps": steps}
    Fe = [torch.empty((H, W, oc.C), dtype=torch.bfloat16, device="cuda") for _ in range(2)]
    F32 = [torch.empty((H, W, oc.C), dtype=torch.float32, device="cuda") for _ in range(2)]
    Ae = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(2)]
    rgba = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    first = {}

    def run(form, joint):
        storage, net, skip, desc = FORMS[form]
        rr = setup_renderer(sc, stereo_cams(sc, 0), layers, form, proposal=prop)
        Fo = F32 if storage == "f32" and net == "f32" else Fe
        fdt = "f32" if net == "f32" else "bf16"
        stream = torch.cuda.current_stream()

        def frame(k):
            pi, vi = step_indices(k)
            p = poses[pi]
            for v, c in enumerate(stereo_cams(sc, vi)):
                rr.set_camera(v, c.W, c.H, c.fx, c.fy, c.cx, c.cy, c.world_to_cam, c.near, c.far)
            rr.set_pose(p.axis_angle, p.R, p.T)
            if joint:
                rr.render_views([0, 1], Fo, Ae, fdt)
            else:
                for v in range(2):
                    rr.render_feature_maps(v, Fo[v], Ae[v], fdt)
            for v in range(2):
                rr.shade(v, Fo[v], rgba[v], fdt)

        n = steps if net != "f32" else max(2, steps // 8)
        for k in range(warmup):
            frame(k)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            frame(warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        frame(0)
        torch.cuda.synchronize()
        first[form + ("_joint" if joint else "")] = rgba[0].cpu().numpy()
        rr.close()
        return {"stereo_frames_per_s": 1e3 / ms, "ms_per_stereo_frame": ms, "steps": n, "form": desc,
                "eyes": ("art_render_views: the eyes one after another (learned skip)" if skip else
                         "one pass (art_render_views)") if joint else "two single-view passes"}

    out["bf16_one_pass"] = run("bf16", True)
    out["bf16_two_passes"] = run("bf16", False)
    out["bf16_skip"] = run("bf16_skip", True)
    out["f32_plain"] = run("f32", True)
    if oracle_psnr:
        import oracle
        pi, vi = step_indices(0)
        cam = stereo_cams(sc, vi)[0]
        ref = oracle.render_frame(sc, poses[pi], cam, layers)["rgba"]
        out["quality_left_eye"] = {k: quality(x, ref) for k, x in first.items()}
        out["quality_left_eye"]["frame"] = "pose %d, azimuth %d, left eye, against the FP64 oracle" % (pi, vi)
    return out


def two_branch_timing(sc, cams, poses, flush, reps=10):
    """The paper's two-branch shading network (appearance U-Net F -> I_f,
    opacity U-Net [A, I_f] -> alpha, both BF16 on the tensor cores) on one
    1024^2 frame's maps, per call, beside the single network."""
    import torch
    import paper_2202_05628_gb300 as art
    import scenegen as sg
    oc = sc.octree
    rgb, alpha = sg.two_branch_weights(0, cin=oc.C)
    r = setup_renderer(sc, cams, None, "bf16")
    r.load_shader(art.ART_NET_TWO_BRANCH, oc.C, sg.UNET_CHANNELS, 4, art.flat_params(rgb + alpha), "bf16",
                  ach=sg.ALPHA_CHANNELS)
    p = poses[0]
    r.set_pose(p.axis_angle, p.R, p.T)
    F = torch.empty((RES, RES, oc.C), dtype=torch.bfloat16, device="cuda")
    A = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    out = torch.empty((RES, RES, 4), dtype=torch.float32, device="cuda")
    r.render_feature_maps(0, F, A, "bf16")
    for _ in range(3):
        r.shade_with_opacity(0, F, A, out, "bf16")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        r.shade_with_opacity(0, F, A, out, "bf16")
        b.record(stream)
    torch.cuda.synchronize()
    r.close()
    return {"ms_per_call": float(np.mean([a.elapsed_time(b) for a, b in ev])),
            "what": "art_shade_with_opacity, BF16 tensor cores: appearance U-Net 32-64-128-256 + opacity U-Net "
                    + "-".join(str(c) for c in sg.ALPHA_CHANNELS) + " at 1024^2"}


def walk_quality(sc, cams, poses, layers, prop, psnr_frames=(20, 40), n_cov=48, n_bg=16):
    """Error against the FP64 oracle per frame over the 60-frame walk cycle
    (each frame at its azimuth of the timed schedule): max-abs of F and A on
    seeded sampled pixels (n_cov the animal covers, n_bg others; the oracle
    brute-forces each over all voxels, on the unrounded FP32 features) for
    the FP32 plain form and the BF16 + learned-skip form; pixels whose F the
    rounding of entry distances decides are left out of the FP32 figure and
    counted.  RGBA PSNR of the BF16 + learned-skip frame on psnr_frames
    (full oracle frames)."""
    import torch
    import oracle
    oc = sc.octree
    rf = setup_renderer(sc, cams, layers, "f32", proposal=prop)
    rs = setup_renderer(sc, cams, layers, "bf16_skip", proposal=prop)
    F32 = torch.empty((RES, RES, oc.C), dtype=torch.float32, device="cuda")
    A32 = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    Fb = torch.empty((RES, RES, oc.C), dtype=torch.bfloat16, device="cuda")
    Ab = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(1234)
    per = {"f32_plain": {"F_max_abs": [], "A_max_abs": [], "order_ambiguous_left_out": 0},
           "bf16_skip": {"F_max_abs": [], "A_max_abs": []}}
    for f in range(N_POSES):
        pi, vi = step_indices(f)
        p = poses[pi]
        for rr in (rf, rs):
            rr.set_pose(p.axis_angle, p.R, p.T)
        rf.render_feature_maps(vi, F32, A32, "f32")
        rs.render_feature_maps(vi, Fb, Ab, "bf16")
        torch.cuda.synchronize()
        a = A32.cpu().numpy().reshape(-1)
        cov, bg = np.flatnonzero(a > 0), np.flatnonzero(a <= 0)
        pick = np.concatenate([rng.choice(cov, min(n_cov, cov.size), replace=False),
                               rng.choice(bg, min(n_bg, bg.size), replace=False)])
        px, py = pick % RES, pick // RES
        _, A, _ = oracle.pose_transforms(sc, p)
        o = oracle.pixels(oc, A, cams[vi], px, py, tie_eps=1e-6)
        keep = o["tie"] <= 1e-5
        for name, Fm, Am, k in (("f32_plain", F32, A32, keep), ("bf16_skip", Fb, Ab, np.ones_like(keep))):
            Fg = Fm.float().cpu().numpy()[py, px]
            Ag = Am.cpu().numpy()[py, px]
            per[name]["F_max_abs"].append(float(np.abs(Fg - o["F"]).max(1)[k].max()))
            per[name]["A_max_abs"].append(float(np.abs(Ag - o["A"])[k].max()))
        per["f32_plain"]["order_ambiguous_left_out"] += int((~keep).sum())
    for v in per.values():
        v["worst_F"] = max(v["F_max_abs"])
        v["worst_A"] = max(v["A_max_abs"])
    rgba = torch.empty((RES, RES, 4), dtype=torch.float32, device="cuda")
    ps = {}
    for f in psnr_frames:
        pi, vi = step_indices(f)
        p = poses[pi]
        rs.render_frame(vi, p.axis_angle, p.R, p.T, rgba)
        torch.cuda.synchronize()
        ref = oracle.render_frame(sc, p, cams[vi], layers)["rgba"]
        ps[str(f)] = quality(rgba.cpu().numpy(), ref)
    rf.close()
    rs.close()
    return {"frames": N_POSES, "samples_per_frame": n_cov + n_bg, **per, "bf16_skip_rgba_by_frame": ps,
            "what": "per walk-cycle frame (pose f, azimuth of step f) against the FP64 oracle"}


def grid_timing(sc, cams, poses, flush, steps, warmup=3):
    """The paper's per-frame index (art_config.index = ART_INDEX_GRID: warped
    centres snapped to the leaf lattice, the smallest id surviving a cell,
    the occupied cells rendered as leaf boxes) against the exact warped
    boxes, BF16 features: time per frame of pose + F/A maps (CUDA events,
    L2 flushed between frames), the share of placed voxels lost to
    collisions, and the PSNR of the index's feature map against the exact
    boxes' (scaled to the boxes' feature range) on the walk-cycle frames."""
    import torch
    oc = sc.octree
    out = {}
    Fs = {}
    for name, index in (("boxes", 0), ("grid", 1)):
        r = setup_renderer(sc, cams, None, "bf16")
        r.set_config(tau=1e-4, skip=0, segment=SEGMENT, index=index)
        F = torch.empty((RES, RES, oc.C), dtype=torch.bfloat16, device="cuda")
        A = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(warmup + steps):
            pi, vi = step_indices(k)
            p = poses[pi]
            flush.zero_()
            if k >= warmup:
                ev[k - warmup][0].record(stream)
            r.set_pose(p.axis_angle, p.R, p.T)
            r.render_feature_maps(vi, F, A, "bf16")
            if k >= warmup:
                ev[k - warmup][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        st = r.sync_status()
        cells, placed = st["grid_cells"], oc.n - st["degenerate"]
        psnr = []
        for k in range(0, steps, max(1, steps // 4)):
            pi, vi = step_indices(warmup + k)
            p = poses[pi]
            r.set_pose(p.axis_angle, p.R, p.T)
            r.render_feature_maps(vi, F, A, "bf16")
            torch.cuda.synchronize()
            Fs.setdefault(name, []).append(F.float().cpu().numpy())
        r.close()
        out[name] = {"ms_per_frame": ms, "frames_per_s": 1e3 / ms}
        if index == 1:
            out[name]["occupied_cells_last_frame"] = int(cells)
            out[name]["collided_share_last_frame"] = 1.0 - cells / max(placed, 1)
    for a, b in zip(Fs["boxes"], Fs["grid"]):
        rng_ = float(np.abs(a).max())
        mse = float(np.mean((a - b) ** 2)) / max(rng_ * rng_, 1e-30)
        psnr.append(10.0 * np.log10(1.0 / max(mse, 1e-30)))
    out["feature_psnr_db_vs_boxes"] = psnr
    out["what"] = ("pose + F/A maps of one 1024^2 view per frame (BF16 features), plain traversal; "
                   "PSNR of F against the exact boxes' F, peak = the boxes' max |F|")
    return out


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sc, cams, poses, layers = workload()
    oc = sc.octree
    rgba = torch.empty((RES, RES, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    prop = proposal_params(sc, cams)
    r = setup_renderer(sc, cams, layers, args.form, profile=False, proposal=prop)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, launches = timed_region(r, poses, args.steps, args.warmup, flush, rgba)
    torch.cuda.synchronize()
    stats = r.sync_status(raise_on_overflow=False)
    # per-kernel CUDA events perturb the frame (~0.2 ms of extra API calls per frame),
    # so they are taken in a second timed pass over the same frames
    kt = {}
    conv_launch_ms = None
    if not args.no_kernel_events:
        configure(r, args.form, True)
        timed_region(r, poses, args.steps, args.warmup, flush, rgba)
        kt = r.kernel_times(reset=True)
        configure(r, args.form, False)
        if FORMS[args.form][1] != "f32":
            conv_launch_ms = unet_ms(r, step_indices(args.warmup + args.steps - 1)[1], oc.C, rgba, flush) / 14
            r.kernel_times(reset=True)
    t_local = float(np.sum(ms))
    t_max = max_over_ranks(t_local, world, "cuda")
    value = job_value(world, args.steps, t_max)
    storage, net, skip, desc = FORMS[args.form]
    result = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": net, "data": "synthetic",
        "config": {"workload": WORKLOAD, "voxels": oc.n, "resolution": [RES, RES], "features": oc.C,
                   "form": desc, "poses": "60-frame walk cycle x 8 azimuths",
                   "l2": "flushed between timed frames (256 MB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "roofline": roofline(kt, stats, peaks, args.form, oc.n, oc.C, args.steps, conv_launch_ms),
        "composite_roofline": composite_roofline(kt, stats, peaks, args.form, oc.C, args.steps) if kt else None,
        "kernels_ms_per_frame": {k: round(v[1] / args.steps, 4) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][1])},
        "kernel_events": "second timed pass over the same frames (per-kernel events slow the frame)",
        "instances": stats["instances"], "overflow": stats["status"],
    }
    if skip:  # fallback share over the walk cycle (untimed pass, one status read per frame)
        n_fb = n_act = 0
        tw = (RES + 7) // 8
        for k in range(N_POSES):
            pi, vi = step_indices(k)
            p = poses[pi]
            r.render_frame(vi, p.axis_angle, p.R, p.T, rgba)
            n_fb += r.sync_status(raise_on_overflow=False)["check_fail_tiles"]
            rg = r.debug_buffer(7, np.uint32).reshape(-1, 2)[:tw * ((RES + 3) // 4)]
            n_act += int(np.sum(rg[:, 1] > rg[:, 0]))
        result["skip"] = {"fallback_tiles_per_frame": n_fb / N_POSES, "active_tiles_per_frame": n_act / N_POSES,
                          "fallback_frac": n_fb / max(n_act, 1), "max_missed": 1e-3, "margin_bins": 1,
                          "proposal": os.path.relpath(PROPOSAL, ROOT) if os.path.exists(PROPOSAL) else "trained in run"}
    frames = {}  # RGBA of the frame that the oracle also renders, per form

    def first_frame(rr, form):
        pi, vi = step_indices(0)
        p = poses[pi]
        rr.render_frame(vi, p.axis_angle, p.R, p.T, rgba)
        torch.cuda.synchronize()
        frames[form] = rgba.cpu().numpy()

    first_frame(r, args.form)
    # depth buffer (Sec. 3.1 "Hybrid Rendering"): projection, binning and the
    # depth walk of one view at the median density as threshold, per call
    Dbuf = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    thr = float(np.median(oc.density))
    vi0 = step_indices(0)[1]
    r.render_depth(vi0, thr, Dbuf)
    dev_ = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in dev_:
        flush.zero_()
        a.record(torch.cuda.current_stream())
        r.render_depth(vi0, thr, Dbuf)
        b.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    result["depth_buffer"] = {"ms_per_call": float(np.mean([a.elapsed_time(b) for a, b in dev_])),
                              "sigma_min": thr, "covered_pixels": int(torch.isfinite(Dbuf).sum().item()),
                              "what": "art_render_depth of one 1024^2 view: projection, binning, depth walk"}
    # view-dependent features (Eq. 2) of degree 2: 9 coefficient vectors per voxel, plain traversal
    configure(r, "bf16", False)
    sh_deg = 2
    coef = 0.3 * torch.randn((oc.n, (sh_deg + 1) ** 2, oc.C), dtype=torch.float32, device="cuda")
    r.load_sh_features(sh_deg, coef)
    Fs = torch.empty((RES, RES, oc.C), dtype=torch.bfloat16, device="cuda")
    As = torch.empty((RES, RES), dtype=torch.float32, device="cuda")
    r.render_feature_maps(vi0, Fs, As, "bf16")
    sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in sev:
        flush.zero_()
        a.record(torch.cuda.current_stream())
        r.render_feature_maps(vi0, Fs, As, "bf16")
        b.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    result["sh_features"] = {"ms_per_call": float(np.mean([a.elapsed_time(b) for a, b in sev])), "degree": sh_deg,
                             "what": "art_render_feature_maps of one 1024^2 view with SH features: projection, "
                                     "binning, the split walk evaluating each hit's harmonics"}
    r.load_sh_features(-1)
    del coef
    r.close()

    def side(form, steps):
        rr = setup_renderer(sc, cams, layers, form, proposal=prop, profile=False)
        ms_s, _ = timed_region(rr, poses, steps, 3, flush, rgba)
        configure(rr, form, True)  # per-kernel times from a second pass
        timed_region(rr, poses, steps, 1, flush, rgba)
        kts = rr.kernel_times(reset=True)
        configure(rr, form, False)
        first_frame(rr, form)
        rr.close()
        top = sorted(kts.items(), key=lambda kv: -kv[1][1])[:4]
        return {"value": 1e3 * steps / float(np.sum(ms_s)), "ms_per_step": float(np.mean(ms_s)), "steps": steps,
                "form": FORMS[form][3], "top_kernels_ms_per_frame": {k: round(v[1] / steps, 4) for k, v in top}}

    # the other forms beside it (same workload, fewer frames)
    if args.form != "f32" and args.f32_steps > 0:
        result["f32_plain"] = side("f32", args.f32_steps)
    if args.side_steps > 0:
        for form in FORMS:
            if form not in (args.form, "f32"):
                result[form + "_form"] = side(form, args.side_steps)
        result["backward"] = backward_timing(sc, cams, poses, layers, args.side_steps, flush)
        result["two_branch"] = two_branch_timing(sc, cams, poses, flush)
        result["grid_index"] = grid_timing(sc, cams, poses, flush, args.side_steps)
        result["stereo_1080p"] = stereo_timing(sc, poses, layers, prop, flush, max(4, args.side_steps // 2),
                                               oracle_psnr=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    # end to end through the public call with host buffers
    if not args.no_e2e:
        r = setup_renderer(sc, cams, layers, args.form, proposal=prop)
        host_out = [torch.empty((RES, RES, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        host_pose = [(torch.from_numpy(p.axis_angle).pin_memory(), torch.from_numpy(p.R).pin_memory(),
                      torch.from_numpy(p.T).pin_memory()) for p in poses]
        k_e2e = max(4, min(args.steps, 30))

        def e2e_loop(pipelined):
            """Host wall clock of k_e2e frames through the public call with host
            buffers: each frame uploads its pose from pinned memory and copies its
            RGBA back to a pinned host buffer.  Pipelined: art_render_frame_async
            (two frames in flight, the buffers alternating) and art_wait_frames
            at the end; else art_render_frame, which waits for each frame."""
            for k in range(2):
                pi, vi = step_indices(k)
                r.render_frame(vi, *host_pose[pi], host_out[0])
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            for k in range(k_e2e):
                pi, vi = step_indices(k)
                if pipelined:
                    r.render_frame_async(vi, *host_pose[pi], host_out[k % 2])
                else:
                    r.render_frame(vi, *host_pose[pi], host_out[0])
            if pipelined:
                r.wait_frames()
            t1 = time.perf_counter()
            return max_over_ranks(1e3 * (t1 - t0), world, "cuda")  # ms, the slowest replica

        t_sync = e2e_loop(False)
        t_e2e = e2e_loop(True)
        result["e2e"] = {"value": job_value(world, k_e2e, t_e2e), "unit": "frames/s",
                         "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in host_pose[0])),
                         "d2h_bytes_per_step": int(host_out[0].numel() * 4), "steps": k_e2e,
                         "call": "art_render_frame_async, two frames in flight, then art_wait_frames",
                         "sync": {"value": job_value(world, k_e2e, t_sync),
                                  "call": "art_render_frame, waiting for each frame"}}
        r.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline: one GPU runs only
        result["cpu_baseline"], ref = cpu_baseline(sc, cams, poses, layers)
        result["quality"] = {f: quality(x, ref) for f, x in frames.items()}
        result["quality"]["frame"] = "pose %d, azimuth %d against the FP64 oracle" % step_indices(0)
        result["quality"]["walk_cycle"] = walk_quality(sc, cams, poses, layers, prop)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


# ---------------------------------------------------------------- oracle arm

def cpu_baseline(sc, cams, poses, layers):
    """The FP64 oracle as it stands on the host cores: one whole frame
    (FK, LBS, F and A maps, U-Net) of the same workload.  Returns the record
    and the oracle's RGBA of that frame."""
    import oracle
    pi, vi = step_indices(0)
    t0 = time.perf_counter()
    out = oracle.render_frame(sc, poses[pi], cams[vi], layers)
    dt = time.perf_counter() - t0
    rec = {"value": 1.0 / dt, "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"1 full frame (pose {pi}, azimuth {vi}): FP64 render + U-Net"}
    return rec, out["rgba"]


def quality(rgba, ref):
    """PSNR (peak 1) and largest difference of an RGBA frame against the
    oracle's."""
    d = np.asarray(rgba, np.float64) - ref
    mse = float(np.mean(d * d))
    return {"psnr_db": 10.0 * np.log10(1.0 / max(mse, 1e-30)), "max_abs": float(np.abs(d).max())}


TILE = 256  # side of the oracle arm's sampled square of the view


def max_over_ranks(t_local: float, world: int, device) -> float:
    """Duration of the whole job's timed region: the max over the ranks (ms)."""
    if world == 1:
        return t_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, t_max_ms: float) -> float:
    """Frames of all replicas per second of the slowest one."""
    return world * steps / (t_max_ms * 1e-3)


def reference_arm(args):
    """The FP64 oracle timed on the host cores.  Each step is a bounded
    sample of the workload: FK and LBS of all voxels, the F and A maps of one
    256x256 square of the 1024x1024 view (a camera with the principal point
    shifted, so the rays are those of the full view), and the U-Net over that
    square; a step counts as 1/16 of a frame.  16 consecutive steps cover
    the whole view."""
    import dataclasses
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, cams, poses, layers = workload()
    import oracle
    oracle.build()
    per = RES // TILE

    posed = {}

    def step(k):
        # 16 consecutive steps are one frame: its FK + LBS once (in the
        # frame's first step), the F / A maps and the U-Net of one square each
        f = k // (per * per)
        pi, vi = step_indices(f)
        c = cams[vi]
        q = k % (per * per)
        x0, y0 = TILE * (q % per), TILE * (q // per)
        crop = dataclasses.replace(c, W=TILE, H=TILE, cx=c.cx - x0, cy=c.cy - y0)
        if posed.get("frame") != f:
            posed["frame"], posed["A"] = f, oracle.pose_transforms(sc, poses[pi])[1]
        F = oracle.render(sc.octree, posed["A"], crop)["F"]
        oracle.shade_unet(F, layers)

    w0 = per * per * ((args.warmup + per * per - 1) // (per * per))  # timed steps start on a frame
    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(w0 + k)
    t_all = time.perf_counter() - t0
    frac = (TILE * TILE) / float(RES * RES)
    v = args.steps * frac / t_all
    sample = (f"{args.steps} steps, each the F/A maps of one {TILE}x{TILE} square of the {RES}x{RES} view and the "
              f"U-Net over it (1/{per * per} frame per step), FK + LBS of {sc.octree.n} voxels once per frame "
              f"({per * per} steps)")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "voxels": sc.octree.n, "resolution": [RES, RES],
                      "sample": f"{TILE}x{TILE} squares"},
           "cpu_baseline": {"value": v, "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    global SEGMENT
    args = parse()
    SEGMENT = args.segment
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
