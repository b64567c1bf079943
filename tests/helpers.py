"""Shared helpers for the parity tests: drive the library through the C ABI
and compare with the oracle."""
import numpy as np

import scenegen as sg


def renderer(scene, storage="f32", tau=1e-4, profile=False, instance_cap=0, segment=256):
    import paper_2202_05628_gb300 as art
    r = art.Renderer()
    oc = scene.octree
    r.load_octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, oc.features, oc.density,
                  storage)
    r.load_skeleton(scene.skeleton.parent, scene.skeleton.rest)
    r.set_config(tau=tau, profile=profile, instance_cap=instance_cap, segment=segment)
    return r


def set_cam(r, view, cam):
    r.set_camera(view, cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, cam.world_to_cam, cam.near, cam.far)


def set_pose(r, pose):
    r.set_pose(pose.axis_angle, pose.R, pose.T)


def render_maps(r, view, cam, C, F_dtype="f32"):
    import torch
    dt = torch.float32 if F_dtype == "f32" else torch.bfloat16
    F = torch.empty((cam.H, cam.W, C), dtype=dt, device="cuda")
    A = torch.empty((cam.H, cam.W), dtype=torch.float32, device="cuda")
    r.render_feature_maps(view, F, A, F_dtype)
    torch.cuda.synchronize()
    return F.float().cpu().numpy(), A.cpu().numpy()


def tie_groups(t0, eps):
    """Indices grouped into runs whose consecutive t0 differ by < eps."""
    groups, cur = [], [0] if len(t0) else []
    for k in range(1, len(t0)):
        if t0[k] - t0[k - 1] < eps:
            cur.append(k)
        else:
            groups.append(cur)
            cur = [k]
    if cur:
        groups.append(cur)
    return groups


def compare_hit_lists(o_ids, o_t0, o_t1, g_ids, g_t0, g_t1, face_eps=1e-5, tie_eps=1e-6):
    """Hit lists equal up to hits with chord < face_eps (a ray within face_eps
    of a box face or edge) and up to order within near-ties of t0.  Returns a
    message, or None when they agree."""
    keep_o = (o_t1 - o_t0) >= face_eps
    keep_g = (g_t1 - g_t0) >= face_eps
    oi, ot0 = o_ids[keep_o], o_t0[keep_o]
    gi = g_ids[keep_g]
    # a grazing hit may exist on one side only: drop ids present on one side
    # whose chord on that side is below 2 face_eps
    if len(oi) != len(gi) or not np.array_equal(np.sort(oi), np.sort(gi)):
        so, sg_ = set(oi.tolist()), set(gi.tolist())
        od = {int(i): float(b - a) for i, a, b in zip(o_ids, o_t0, o_t1)}
        gd = {int(i): float(b - a) for i, a, b in zip(g_ids, g_t0, g_t1)}
        bad = [i for i in so ^ sg_ if max(od.get(i, 0.0), gd.get(i, 0.0)) >= 2 * face_eps]
        if bad:
            return f"hit sets differ: only oracle {sorted(so - sg_)[:8]}, only gpu {sorted(sg_ - so)[:8]}"
        common = so & sg_
        m_o = np.array([i in common for i in oi.tolist()], bool)
        m_g = np.array([i in common for i in gi.tolist()], bool)
        oi, ot0, gi = oi[m_o], ot0[m_o], gi[m_g]
    pos = 0
    for grp in tie_groups(ot0, tie_eps):
        a = oi[grp]
        b = gi[pos:pos + len(grp)]
        if not np.array_equal(np.sort(a), np.sort(b)):
            return f"order differs near t0={ot0[grp[0]]:.7f}: oracle {a.tolist()} gpu {b.tolist()}"
        pos += len(grp)
    return None


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def tiny_setup(az=0.0, pose_seed=1, res=128):
    sc = sg.preset("tiny")
    cam = sg.orbit_camera(sc.centroid, res, res, az_deg=az)
    return sc, cam, sg.random_pose(pose_seed)



def order_ambiguous(o, octree, H, W, tie_eps=1e-6, effect=1e-5, features=None):
    """Pixels of an oracle render (``hits=True``) whose F the rounding of
    entry distances decides: two consecutive composited hits (or the last
    composited one and the next) with entry distances within ``tie_eps`` whose
    swap changes a channel by more than ``effect`` (T_i alpha_i alpha_j
    |f_i - f_j|, the difference of the two orders' sums)."""
    feat = np.asarray(octree.features if features is None else features, np.float64)
    sig = np.asarray(octree.density, np.float64)
    off, ids, t0, t1 = o["hit_off"], o["hit_id"], o["hit_t0"], o["hit_t1"]
    used = o["nused"].ravel()
    out = np.zeros(H * W, bool)
    for p in np.flatnonzero(o["nhit"].ravel() > 1):
        a, b = off[p], off[p + 1]
        last = min(b - a - 1, int(used[p]))
        optical = 0.0
        for i in range(last):
            k = a + i
            ai = 1.0 - np.exp(-sig[ids[k]] * (t1[k] - t0[k]))
            if t0[k + 1] - t0[k] < tie_eps:
                aj = 1.0 - np.exp(-sig[ids[k + 1]] * (t1[k + 1] - t0[k + 1]))
                df = np.abs(feat[ids[k]] - feat[ids[k + 1]]).max()
                if np.exp(-optical) * ai * aj * df > effect:
                    out[p] = True
                    break
            optical += sig[ids[k]] * (t1[k] - t0[k])
    return out.reshape(H, W)


def subpixel_cat_conv(d, e, layer, bf16=True):
    """ReLU(conv3x3([up2(d) | e]) + b) as the sub-pixel decoder convolution
    computes it: the skip part e with the BF16-rounded 3x3 weights; the
    upsampled part per output phase (py, px) as a 3x3-footprint convolution
    of the low-resolution d whose taps are the FP32 sums (in the kernel's
    order dy, dx = -1 .. 1) of the weights that land on the same
    low-resolution pixel, rounded once to BF16 (bf16=False: no rounding,
    the exact identity with the concatenated convolution)."""
    import torch
    import torch.nn.functional as Fn
    bf = (lambda t: t.to(torch.bfloat16).to(torch.float64)) if bf16 else (lambda t: t)
    w, b = np.asarray(layer[0], np.float32), np.asarray(layer[1], np.float64)
    cu = d.shape[1]
    ws = bf(torch.from_numpy(w[..., cu:].astype(np.float64))).permute(0, 3, 1, 2)
    out = Fn.conv2d(e, ws, padding=1)
    half = lambda v: (v + 2) // 2 - 1  # floor(v / 2) for v in -1 .. 2
    for py in (0, 1):
        for px in (0, 1):
            kd = np.float32 if bf16 else np.float64
            K = np.zeros((w.shape[0], 3, 3, cu), kd)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    K[:, half(py + dy) + 1, half(px + dx) + 1] += w[:, dy + 1, dx + 1, :cu].astype(kd)
            Kb = bf(torch.from_numpy(K.astype(np.float64))).permute(0, 3, 1, 2)
            out[:, :, py::2, px::2] += Fn.conv2d(d, Kb, padding=1)
    return torch.relu(out + torch.from_numpy(b)[None, :, None, None])
