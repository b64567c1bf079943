"""DRAM traffic of the BF16 U-Net's convolutions, from one ncu capture, for
the benchmark's ``roofline.traffic``.

    python -m paper_2202_05628_gb300.profile_capture workload   # the captured program (run it plainly first)
    python -m paper_2202_05628_gb300.profile_capture capture    # ncu on it; writes profiles/conv_unet_1024_traffic.md

The workload shades one 1024x1024 feature map (32 BF16 channels, seeded)
through the 4-level 32-64-128-256 U-Net three times; the capture takes the
14 convolution launches of the last call (ncu flushes the caches before
each, so every layer reads its inputs from DRAM), with the counters
dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum.
The summary records a hash of the convolution sources it measured; the
benchmark reports the traffic only while the sources still hash the same.
"""
from __future__ import annotations

import csv
import hashlib
import io
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SUMMARY = os.path.join(ROOT, "profiles", "conv_unet_1024_traffic.md")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("cnn_tc.cu", "cnn_sub.cu", "tc.cuh", "cnn.cu")]
RES = 1024
CALLS = 3
LAUNCHES = 14


def source_hash() -> str:
    h = hashlib.sha256()
    for p in SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def workload() -> None:
    import numpy as np
    import torch

    sys.path.insert(0, ROOT)
    import paper_2202_05628_gb300 as art
    import scenegen as sg

    sc = sg.preset("mini")
    oc = sc.octree
    layers = sg.unet_weights(0, cin=32)
    r = art.Renderer()
    f32 = np.zeros((oc.n, 32), np.float32)
    r.load_octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, f32, oc.density, "bf16")
    r.load_shader(art.ART_NET_UNET, 32, sg.UNET_CHANNELS, 4, art.flat_params(layers), "bf16")
    cam = sg.orbit_camera(sc.centroid, RES, RES)
    r.set_camera(0, cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, cam.world_to_cam, cam.near, cam.far)
    g = torch.Generator(device="cuda").manual_seed(0)
    F = (0.3 * torch.randn((RES, RES, 32), generator=g, device="cuda")).to(torch.bfloat16)
    out = torch.empty((RES, RES, 4), dtype=torch.float32, device="cuda")
    for _ in range(CALLS):
        r.shade(0, F, out, "bf16")
    torch.cuda.synchronize()
    r.close()
    print("workload ok")


def capture() -> None:
    cmd = ["ncu", "--metrics", "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum",
           "--clock-control", "none", "-k", "regex:conv_", "-s", str(LAUNCHES * (CALLS - 1)), "-c", str(LAUNCHES),
           "--csv", sys.executable, "-m", "paper_2202_05628_gb300.profile_capture", "workload"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout[-4000:] + res.stderr[-4000:])
        raise SystemExit(res.returncode)
    text = res.stdout[res.stdout.index('"ID"'):]
    per = {}
    for row in csv.DictReader(io.StringIO(text)):
        m = re.search(r"(\w+_kernel)", row["Kernel Name"])  # the kernel, without namespace and arguments
        k = (int(row["ID"]), m.group(1) if m else row["Kernel Name"][:40])
        v = float(row["Metric Value"].replace(",", ""))
        unit = row["Metric Unit"].strip()
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "ns": 1e-3,
                 "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(unit, 1.0)
        per.setdefault(k, {})[row["Metric Name"]] = v * scale
    rows = sorted(per.items())
    total = sum(m.get("dram__bytes_read.sum", 0) + m.get("dram__bytes_write.sum", 0) for _, m in rows)
    us = sum(m.get("gpu__time_duration.sum", 0) for _, m in rows)
    lines = ["# DRAM traffic of the BF16 U-Net convolutions at 1024x1024", "",
             "Command (on one GB300, after `python -m paper_2202_05628_gb300.profile_capture workload`",
             "exited 0 without ncu):", "",
             "    python -m paper_2202_05628_gb300.profile_capture capture", "",
             "which runs `" + " ".join(cmd[:-3]) + " python -m paper_2202_05628_gb300.profile_capture workload`.",
             "ncu flushes the caches before each launch (cold), so every layer reads its inputs from DRAM.", "",
             "| launch | kernel | us (cold) | DRAM read MB | DRAM write MB |", "|---:|---|---:|---:|---:|"]
    for (i, name), m in rows:
        lines.append(f"| {i} | {name} | {m.get('gpu__time_duration.sum', 0):.1f} | "
                     f"{m.get('dram__bytes_read.sum', 0) / 1e6:.1f} | {m.get('dram__bytes_write.sum', 0) / 1e6:.1f} |")
    lines += ["", f"Sum over the {len(rows)} launches: {total / 1e6:.1f} MB, {us:.1f} us (cold, serialised).", "",
              f"traffic_per_launch_bytes: {total / max(len(rows), 1):.0f}",
              f"launches: {len(rows)}",
              f"source_sha256: {source_hash()}", ""]
    with open(SUMMARY, "w") as f:
        f.write("\n".join(lines))
    print(f"wrote {SUMMARY}: {total / 1e6:.1f} MB over {len(rows)} launches")


def committed_traffic():
    """Traffic per launch from the committed summary when it was captured on
    the current convolution sources, else None."""
    try:
        with open(SUMMARY) as f:
            kv = dict(line.split(": ", 1) for line in f.read().splitlines() if ": " in line and "_" in line[:30])
        if kv.get("source_sha256", "").strip() != source_hash():
            return None
        return float(kv["traffic_per_launch_bytes"])
    except (OSError, KeyError, ValueError):
        return None


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "capture":
        capture()
    else:
        workload()
