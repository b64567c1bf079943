"""Offline training of the learned ray-interval proposal.

The proposal is a per-ray MLP (pose + ray -> depth interval) that lets the
compositing kernel skip depth a ray does not need (project addition; the
paper's nearest passage is the early-stop rule of Sec. 3.1 "Dynamic Volume
Rendering").  Its inference runs in the library (``art_run_proposal`` and the
learned-skip render); this module produces its weights:

* labels come from the plain renderer itself (``Renderer.render_labels``:
  the bin interval that keeps every hit of weight > 1e-6 and that the coarse
  check passes);
* the network is trained in BF16 (autocast) with a cross-entropy loss on the
  near and far bins;
* weights are stored in a small versioned binary file.

The input encoding here must equal the library's: [72 joint axis-angles,
unit world ray direction, sin / cos (2^k pi u), sin / cos (2^k pi v), k < 8],
u = (x + 1/2) / W, v = (y + 1/2) / H.
"""
from __future__ import annotations

import math
import struct
from typing import List, Sequence, Tuple

import numpy as np

N_BINS = 64
SHAPES = [(64, 107), (64, 64), (64, 64), (64, 64), (128, 64)]
N_PARAMS = sum(o * i + o for o, i in SHAPES)
_MAGIC = b"ARTPROP1"


def encode_rays(axis_angle, cam, pix, device="cuda"):
    """Proposal inputs of the pixels ``pix`` (flat indices y * W + x) of
    `cam` under the pose, [len(pix), 107] FP32."""
    import torch
    H, W = cam.H, cam.W
    pix = torch.as_tensor(pix, device=device).long()
    pose = torch.as_tensor(np.asarray(axis_angle, np.float32).reshape(-1), device=device)
    xs = (pix % W).double()
    ys = (pix // W).double()
    dc = torch.stack([(xs + 0.5 - cam.cx) / cam.fx, (ys + 0.5 - cam.cy) / cam.fy, torch.ones_like(xs)], -1)
    R = torch.as_tensor(np.asarray(cam.world_to_cam, np.float64)[:, :3], device=device)
    d = dc @ R  # R^T dc for each row
    d = (d / d.norm(dim=1, keepdim=True)).float()
    u = ((xs.float() + 0.5) / W).reshape(-1, 1)
    v = ((ys.float() + 0.5) / H).reshape(-1, 1)
    fr = math.pi * (2.0 ** torch.arange(8, device=device, dtype=torch.float32))[None, :]
    four = torch.cat([torch.sin(fr * u), torch.cos(fr * u), torch.sin(fr * v), torch.cos(fr * v)], 1)
    return torch.cat([pose[None, :].expand(pix.numel(), 72), d, four], 1)


def encode(axis_angle, cam, device="cuda"):
    """Proposal inputs of every pixel of `cam` under the pose, [H*W, 107] FP32."""
    import torch
    return encode_rays(axis_angle, cam, torch.arange(cam.H * cam.W, device=device), device)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, flat in the library's layout."""
    rng = np.random.default_rng(seed)
    out = []
    for n_out, n_in in SHAPES:
        out.append((rng.standard_normal((n_out, n_in)) * math.sqrt(2.0 / n_in)).reshape(-1))
        out.append(np.zeros(n_out))
    return np.concatenate(out).astype(np.float32)


def _module(params, device):
    import torch
    layers = []
    o = 0
    for n_out, n_in in SHAPES:
        lin = torch.nn.Linear(n_in, n_out).to(device)
        with torch.no_grad():
            lin.weight.copy_(torch.as_tensor(params[o:o + n_out * n_in].reshape(n_out, n_in)))
            o += n_out * n_in
            lin.bias.copy_(torch.as_tensor(params[o:o + n_out]))
            o += n_out
        layers.append(lin)
    seq = []
    for i, lin in enumerate(layers):
        seq.append(lin)
        if i < len(layers) - 1:
            seq.append(torch.nn.ReLU())
    return torch.nn.Sequential(*seq)


def _flat(module) -> np.ndarray:
    out = []
    for m in module:
        if hasattr(m, "weight"):
            out.append(m.weight.detach().float().cpu().numpy().reshape(-1))
            out.append(m.bias.detach().float().cpu().numpy().reshape(-1))
    return np.concatenate(out).astype(np.float32)


def collect(renderer, poses: Sequence, views: Sequence[int], cams: Sequence, rays_per_view: int = 8192,
            seed: int = 0, views_per_pose: int = 0):
    """Labels of the plain renderer: for every pose and view (or
    ``views_per_pose`` random views of each pose), a random sample of the
    rays of the screen tiles around the animal (tiles holding a significant
    hit, grown by one tile), their inputs and label bins.  Returns
    (X [M,107] FP32, Y [M,2] int64) on the device."""
    import torch
    import torch.nn.functional as Fn
    g = torch.Generator(device="cuda").manual_seed(seed)
    rng = np.random.default_rng(seed)
    Xs, Ys = [], []
    for p in poses:
        renderer.set_pose(p.axis_angle, p.R, p.T)
        vsel = list(views) if not views_per_pose else list(rng.choice(list(views), views_per_pose, replace=False))
        for vi in vsel:
            cam = cams[vi]
            H, W = cam.H, cam.W
            bins = torch.zeros((H, W, 2), dtype=torch.uint8, device="cuda")
            lab = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
            renderer.render_labels(vi, lab, bins)
            th, tw = (H + 3) // 4, (W + 7) // 8
            sig = torch.zeros((th * 4, tw * 8), dtype=torch.float32, device="cuda")
            sig[:H, :W] = torch.isfinite(lab[..., 0]).float()
            t = sig.reshape(th, 4, tw, 8).amax((1, 3))
            t = Fn.max_pool2d(t[None, None], 3, stride=1, padding=1)[0, 0] > 0
            act = t.repeat_interleave(4, 0).repeat_interleave(8, 1)[:H, :W].reshape(-1)
            idx = torch.nonzero(act).reshape(-1)
            if idx.numel() == 0:
                continue
            pick = idx[torch.randint(0, idx.numel(), (min(rays_per_view, idx.numel()),), generator=g, device="cuda")]
            Xs.append(encode_rays(p.axis_angle, cam, pick))
            Ys.append(bins.reshape(-1, 2)[pick].long())
    collect.overflow_order = renderer.sync_status(raise_on_overflow=False)["overflow_order"]
    return torch.cat(Xs), torch.cat(Ys)


def train(X, Y, params=None, steps: int = 3000, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          log_every: int = 0) -> np.ndarray:
    """Cross-entropy on the near and far bins, Adam, BF16 autocast; returns
    the flat FP32 parameters (library layout)."""
    import torch
    torch.manual_seed(seed)
    net = _module(init_params(seed) if params is None else np.asarray(params, np.float32), "cuda")
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    ce = torch.nn.CrossEntropyLoss()
    M = X.shape[0]
    for it in range(steps):
        idx = torch.randint(0, M, (min(batch, M),), device="cuda")
        with torch.autocast("cuda", dtype=torch.bfloat16):
            lg = net(X[idx])
        lg = lg.float()
        loss = ce(lg[:, :N_BINS], Y[idx, 0]) + ce(lg[:, N_BINS:], Y[idx, 1])
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss.item():.4f}")
    return _flat(net)


def accuracy(params, X, Y) -> Tuple[float, float, float]:
    """(near-bin accuracy, far-bin accuracy, fraction of rays whose predicted
    interval contains the label interval) of the FP32 network."""
    import torch
    net = _module(np.asarray(params, np.float32), "cuda")
    with torch.no_grad():
        lg = net(X)
    bn = lg[:, :N_BINS].argmax(1)
    bf = lg[:, N_BINS:].argmax(1)
    cover = ((bn <= Y[:, 0]) & (bf >= Y[:, 1])).float().mean().item()
    return (bn == Y[:, 0]).float().mean().item(), (bf == Y[:, 1]).float().mean().item(), cover


def save(path: str, params, meta: str = "") -> None:
    p = np.asarray(params, np.float32).reshape(-1)
    assert p.size == N_PARAMS
    m = meta.encode()
    with open(path, "wb") as f:
        f.write(_MAGIC + struct.pack("<II", p.size, len(m)) + m + p.tobytes())


def load(path: str) -> Tuple[np.ndarray, str]:
    with open(path, "rb") as f:
        b = f.read()
    if b[:8] != _MAGIC:
        raise ValueError(f"{path}: not a proposal weights file")
    n, lm = struct.unpack("<II", b[8:16])
    meta = b[16:16 + lm].decode()
    p = np.frombuffer(b[16 + lm:16 + lm + 4 * n], np.float32).copy()
    if p.size != N_PARAMS:
        raise ValueError(f"{path}: {p.size} parameters, {N_PARAMS} expected")
    return p, meta


def evaluate(renderer, params, poses, cams, margin: int = 1, max_missed: float = 1e-3) -> dict:
    """Learned skip against the plain render on held-out poses (one view per
    pose, cycling): fallback tiles / active tiles, and the largest
    difference of F and A."""
    import torch
    renderer.load_proposal(params)
    renderer.sync_status(raise_on_overflow=False)  # clear earlier flags
    n_fb = n_act = n_over = 0
    dF = dA = 0.0
    C = renderer.C
    for k, p in enumerate(poses):
        vi = k % len(cams)
        cam = cams[vi]
        F0 = torch.empty((cam.H, cam.W, C), dtype=torch.float32, device="cuda")
        A0 = torch.empty((cam.H, cam.W), dtype=torch.float32, device="cuda")
        F1, A1 = torch.empty_like(F0), torch.empty_like(A0)
        renderer.set_pose(p.axis_angle, p.R, p.T)
        renderer.set_config(skip=0)
        renderer.render_feature_maps(vi, F0, A0)
        renderer.set_config(skip=1, max_missed=max_missed, margin=margin)
        renderer.render_feature_maps(vi, F1, A1)
        st = renderer.sync_status(raise_on_overflow=False)
        n_over += st["overflow_order"]
        rg = renderer.debug_buffer(7, np.uint32).reshape(-1, 2)[:((cam.W + 7) // 8) * ((cam.H + 3) // 4)]
        n_act += int(np.sum(rg[:, 1] > rg[:, 0]))
        n_fb += st["check_fail_tiles"]
        dF = max(dF, torch.abs(F1 - F0).max().item())
        dA = max(dA, torch.abs(A1 - A0).max().item())
    renderer.set_config(skip=0)
    return {"fallback_tiles": n_fb, "active_tiles": n_act, "fallback_frac": n_fb / max(n_act, 1), "max_dF": dF,
            "max_dA": dA, "reorder_overflows": n_over}


def main(argv=None) -> None:
    """Train the proposal for a synthetic workload of ``scenegen`` and write
    the weights file: labels over random poses (each joint up to 30 deg)
    seen from the workload's orbit cameras, evaluation on held-out poses."""
    import argparse
    import json
    import os
    import sys
    import time
    p = argparse.ArgumentParser(description=main.__doc__)
    p.add_argument("--preset", default="paper")
    p.add_argument("--res", type=int, default=1024)
    p.add_argument("--azimuths", type=int, default=8)
    p.add_argument("--poses", type=int, default=2000)
    p.add_argument("--views-per-pose", type=int, default=2)
    p.add_argument("--rays", type=int, default=4096, help="rays sampled per (pose, view)")
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--batch", type=int, default=16384)
    p.add_argument("--eval-poses", type=int, default=200)
    p.add_argument("--out", required=True)
    a = p.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import scenegen as sg
    from . import Renderer, flat_params  # noqa: F401  (the library must load)
    t0 = time.time()
    sc = sg.preset(a.preset)
    oc = sc.octree
    cams = [sg.orbit_camera(sc.centroid, a.res, a.res, az_deg=360.0 / a.azimuths * k) for k in range(a.azimuths)]
    r = Renderer()
    r.load_octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, oc.features, oc.density, "bf16")
    r.load_skeleton(sc.skeleton.parent, sc.skeleton.rest)
    r.set_config()
    for k, c in enumerate(cams):
        r.set_camera(k, c.W, c.H, c.fx, c.fy, c.cx, c.cy, c.world_to_cam, c.near, c.far)
    train_poses = [sg.random_pose(k) for k in range(a.poses)]
    X, Y = collect(r, train_poses, list(range(len(cams))), cams, a.rays, seed=0, views_per_pose=a.views_per_pose)
    t1 = time.time()
    params = train(X, Y, steps=a.steps, batch=a.batch, lr=2e-3)
    t2 = time.time()
    acc = accuracy(params, X, Y)
    held = [sg.random_pose(100000 + k) for k in range(a.eval_poses)]
    ev = evaluate(r, params, held, cams)
    walk = evaluate(r, params, [sg.walk_pose(f, 60) for f in range(60)], cams)
    meta = {"preset": a.preset, "res": a.res, "azimuths": a.azimuths, "train_poses": a.poses,
            "samples": int(X.shape[0]), "label_reorder_overflows": int(collect.overflow_order), "steps": a.steps, "train_acc_near_far_cover": acc,
            "held_out": ev, "walk_cycle": walk, "label_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1)}
    save(a.out, params, json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
