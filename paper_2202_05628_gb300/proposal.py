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


def ray_dirs(cam, device="cuda"):
    """Unit world-space ray directions of every pixel centre, [H*W, 3]."""
    import torch
    H, W = cam.H, cam.W
    ys, xs = torch.meshgrid(torch.arange(H, device=device, dtype=torch.float64),
                            torch.arange(W, device=device, dtype=torch.float64), indexing="ij")
    dc = torch.stack([(xs + 0.5 - cam.cx) / cam.fx, (ys + 0.5 - cam.cy) / cam.fy, torch.ones_like(xs)], -1)
    R = torch.as_tensor(np.asarray(cam.world_to_cam, np.float64)[:, :3], device=device)
    d = dc.reshape(-1, 3) @ R  # R^T dc for each row
    return (d / d.norm(dim=1, keepdim=True)).float()


def encode(axis_angle, cam, device="cuda"):
    """Proposal inputs of every pixel of `cam` under the pose, [H*W, 107] FP32."""
    import torch
    H, W = cam.H, cam.W
    pose = torch.as_tensor(np.asarray(axis_angle, np.float32).reshape(-1), device=device)
    d = ray_dirs(cam, device)
    ys, xs = torch.meshgrid(torch.arange(H, device=device, dtype=torch.float32),
                            torch.arange(W, device=device, dtype=torch.float32), indexing="ij")
    u = ((xs + 0.5) / W).reshape(-1, 1)
    v = ((ys + 0.5) / H).reshape(-1, 1)
    fr = math.pi * (2.0 ** torch.arange(8, device=device, dtype=torch.float32))[None, :]
    four = torch.cat([torch.sin(fr * u), torch.cos(fr * u), torch.sin(fr * v), torch.cos(fr * v)], 1)
    return torch.cat([pose[None, :].expand(H * W, 72), d, four], 1)


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
            seed: int = 0, active_only: bool = True):
    """Labels of the plain renderer: for every (pose, view), a random sample
    of the rays of tiles that hold instances (or all rays), their inputs and
    label bins.  Returns (X [M,107] FP32, Y [M,2] int64) on the device."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    Xs, Ys = [], []
    for p in poses:
        renderer.set_pose(p.axis_angle, p.R, p.T)
        for vi in views:
            cam = cams[vi]
            bins = torch.zeros((cam.H, cam.W, 2), dtype=torch.uint8, device="cuda")
            lab = torch.empty((cam.H, cam.W, 3), dtype=torch.float32, device="cuda")
            renderer.render_labels(vi, lab, bins)
            b = bins.reshape(-1, 2).long()
            if active_only:
                hist = torch.as_tensor(renderer.debug_buffer(12, np.float32), device="cuda")
                tw, th = (cam.W + 7) // 8, (cam.H + 3) // 4
                act_t = hist[:tw * th * N_BINS].reshape(th, tw, N_BINS).sum(-1) > 0
                act = act_t.repeat_interleave(4, 0).repeat_interleave(8, 1)[:cam.H, :cam.W].reshape(-1)
                idx = torch.nonzero(act).reshape(-1)
            else:
                idx = torch.arange(cam.H * cam.W, device="cuda")
            if idx.numel() == 0:
                continue
            pick = idx[torch.randint(0, idx.numel(), (min(rays_per_view, idx.numel()),), generator=g, device="cuda")]
            X = encode(p.axis_angle, cam)[pick]
            Xs.append(X)
            Ys.append(b[pick])
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
