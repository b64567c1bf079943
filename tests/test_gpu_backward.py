"""GPU parity of the hand-written backward (composite + LBS) against the FP64
oracle's analytic gradient, which tests/test_oracle_pins.py pins to central
finite differences.  Gradients w.r.t. voxel features, densities and skinning
weights, through the C ABI and through torch.autograd."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import renderer, set_cam, set_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _gpu_grads(sc, pose, cams, gFs, gAs, storage="f32", segment=256, tau=1e-4):
    import torch
    oc = sc.octree
    r = renderer(sc, storage=storage, segment=segment, tau=tau)
    set_pose(r, pose)
    gf = torch.zeros((oc.n, oc.C), dtype=torch.float32, device="cuda")
    gd = torch.zeros(oc.n, dtype=torch.float32, device="cuda")
    gw = torch.zeros((oc.n, 4), dtype=torch.float32, device="cuda")
    for v, (cam, gF, gA) in enumerate(zip(cams, gFs, gAs)):
        set_cam(r, v, cam)
        F = torch.empty((cam.H, cam.W, oc.C), dtype=torch.float32, device="cuda")
        A = torch.empty((cam.H, cam.W), dtype=torch.float32, device="cuda")
        r.render_feature_maps(v, F, A, "f32")
        dF = torch.from_numpy(np.ascontiguousarray(gF, np.float32)).cuda()
        dA = torch.from_numpy(np.ascontiguousarray(gA, np.float32)).cuda()
        r.render_backward(v, F, A, dF, dA, gf, gd, gw)
    st = r.sync_status()
    assert st["overflow_order"] == 0
    return gf.cpu().numpy().astype(np.float64), gd.cpu().numpy().astype(np.float64), gw.cpu().numpy().astype(np.float64)


def _oracle_grads(sc, pose, cams, gFs, gAs, features=None, tau=1e-4):
    oc = sc.octree
    G, A, _ = oracle.pose_transforms(sc, pose)
    gf = np.zeros((oc.n, oc.C))
    gd = np.zeros(oc.n)
    gN = np.zeros((oc.n, 3, 4))
    for cam, gF, gA in zip(cams, gFs, gAs):
        a, b, c = oracle.render_backward(oc, A, cam, gF, gA, tau=tau, features=features)
        gf += a
        gd += b
        gN += c
    _, gw = oracle.lbs_backward(oc, G, A, gN)
    return gf, gd, gw


# FP32 ray parameters carry ~2.4e-7 m of rounding at 2 m; chords are a few
# mm, so alpha = 1 - exp(-sigma delta) and with it every gradient term carries
# ~1e-4 relative error (more for grazing chords and, through 1 / d'_a, for the
# geometric terms of the skinning weights).
def _close(g, o, rel_l2, what):
    scale = np.linalg.norm(o)
    assert scale > 0, what
    err = np.linalg.norm(g - o) / scale
    assert err < rel_l2, f"{what}: relative L2 error {err:.2e} (max abs {np.abs(g - o).max():.2e}, scale {np.abs(o).max():.2e})"


def test_backward_matches_oracle_small():
    sc = sg.preset("tiny")
    pose = sg.random_pose(13)
    cams = [sg.orbit_camera(sc.centroid, 96, 96, az_deg=a) for a in (10.0, 130.0)]
    rng = np.random.default_rng(0)
    gFs = [rng.standard_normal((96, 96, sc.octree.C)) for _ in cams]
    gAs = [rng.standard_normal((96, 96)) for _ in cams]
    g = _gpu_grads(sc, pose, cams, gFs, gAs)
    o = _oracle_grads(sc, pose, cams, gFs, gAs)
    _close(g[0], o[0], 3e-4, "dL/df")
    _close(g[1], o[1], 1e-3, "dL/dsigma")
    _close(g[2], o[2], 5e-3, "dL/dw")


@pytest.mark.parametrize("segment,tau", [(32, 1e-4), (96, 0.7)])
def test_backward_split_walk_matches_oracle(segment, tau):
    """Lists walked in short depth segments by separate warps (a pass for
    each segment's own transmittance and <P, g>, a prefix over segments, the
    gradient pass) against the oracle and against one segment per tile; with
    tau = 0.7 the stop falls inside later segments."""
    sc = sg.preset("tiny")
    pose = sg.random_pose(17)
    cams = [sg.orbit_camera(sc.centroid, 64, 64, az_deg=a, fov_deg=8.0) for a in (40.0, 200.0)]
    rng = np.random.default_rng(2)
    gFs = [rng.standard_normal((64, 64, sc.octree.C)) for _ in cams]
    gAs = [rng.standard_normal((64, 64)) for _ in cams]
    g = _gpu_grads(sc, pose, cams, gFs, gAs, segment=segment, tau=tau)
    g1 = _gpu_grads(sc, pose, cams, gFs, gAs, segment=1 << 24, tau=tau)
    o = _oracle_grads(sc, pose, cams, gFs, gAs, tau=tau)
    for a, b, what in zip(g, g1, ("dL/df", "dL/dsigma", "dL/dw")):
        _close(a, b, 1e-5, what + " split vs one segment")  # the same sums, atomics in another order
    _close(g[0], o[0], 3e-4, "dL/df")
    _close(g[1], o[1], 1e-3, "dL/dsigma")
    _close(g[2], o[2], 5e-3, "dL/dw")


def test_backward_config4_random_rays():
    """200k voxels (C=16), 8 views at 512x512, MSE of F to a random target on
    65,536 random rays."""
    import torch
    sc = sg.preset("diff")
    oc = sc.octree
    pose = sg.random_pose(21, max_deg=20.0)
    cams = [sg.orbit_camera(sc.centroid, 512, 512, az_deg=45.0 * k) for k in range(8)]
    rng = np.random.default_rng(4)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    gFs, gAs = [], []
    n_rays = 65536 // len(cams)
    for cam in cams:
        # rays drawn where the animal is
        cov = oracle.render(oc, A_or, cam)
        on = np.flatnonzero(cov["A"].ravel() > 0)
        pick = rng.choice(on, min(n_rays, on.size), replace=False)
        target = 0.3 * rng.standard_normal((cam.H * cam.W, oc.C))
        gF = np.zeros((cam.H * cam.W, oc.C))
        gF[pick] = 2.0 * (cov["F"].reshape(-1, oc.C)[pick] - target[pick]) / 65536.0
        gFs.append(gF.reshape(cam.H, cam.W, oc.C))
        gAs.append(np.zeros((cam.H, cam.W)))
    g = _gpu_grads(sc, pose, cams, gFs, gAs)
    o = _oracle_grads(sc, pose, cams, gFs, gAs)
    _close(g[0], o[0], 3e-4, "dL/df")
    _close(g[1], o[1], 1e-3, "dL/dsigma")
    # Skinning weights: each chord's derivative is piecewise smooth.  A hit
    # within rounding of a piece boundary (a ray leaving near an edge, a
    # vanishing chord, entry distances of overlapping warped voxels that tie,
    # which flips the compositing order and with it the feature mass behind
    # every earlier hit) takes the other piece in FP32 for a few voxels and
    # changes their gradient by O(1); FP64 finite differences land on either
    # side there.  Checked: nearly all voxels agree tightly, and the aggregate.
    carried = np.abs(o[2]).max(1) > 0
    per_voxel = np.abs(g[2] - o[2]).max(1) <= 2e-2 * np.abs(o[2]).max(1) + 1e-3 * np.abs(o[2]).max()
    assert per_voxel[carried].mean() > 0.99, per_voxel[carried].mean()
    _close(g[2], o[2], 0.1, "dL/dw (aggregate)")
    del torch


def test_autograd_function_equals_direct_call():
    import torch
    import paper_2202_05628_gb300 as art
    sc = sg.preset("mini")
    oc = sc.octree
    pose = sg.random_pose(2)
    cam = sg.orbit_camera(sc.centroid, 64, 64, az_deg=40.0)
    r = renderer(sc)
    set_cam(r, 0, cam)
    f = torch.from_numpy(oc.features).cuda().requires_grad_(True)
    d = torch.from_numpy(oc.density).cuda().requires_grad_(True)
    w = torch.from_numpy(oc.weights).cuda().requires_grad_(True)
    pz = (pose.axis_angle, pose.R, pose.T)
    F, A = art.render_features(r, 0, f, d, w, pz)
    tgt = torch.randn_like(F) * 0.1
    loss = ((F - tgt) ** 2).sum() + (A ** 2).sum()
    loss.backward()
    gF = (2 * (F - tgt)).detach().cpu().numpy()
    gA = (2 * A).detach().cpu().numpy()
    o = _oracle_grads(sc, pose, [cam], [gF], [gA])
    _close(f.grad.cpu().numpy().astype(np.float64), o[0], 3e-4, "autograd dL/df")
    _close(d.grad.cpu().numpy().astype(np.float64), o[1], 1e-3, "autograd dL/dsigma")
    _close(w.grad.cpu().numpy().astype(np.float64), o[2], 5e-3, "autograd dL/dw")
    o_F = oracle.render(oc, oracle.pose_transforms(sc, pose)[1], cam)
    assert np.abs(F.detach().cpu().numpy() - o_F["F"]).max() < 1e-4


def test_backward_bf16_storage_uses_rounded_features():
    import torch
    sc = sg.preset("tiny")
    pose = sg.random_pose(17)
    cam = sg.orbit_camera(sc.centroid, 96, 96, az_deg=70.0)
    rng = np.random.default_rng(3)
    gF = rng.standard_normal((96, 96, sc.octree.C))
    gA = rng.standard_normal((96, 96))
    g = _gpu_grads(sc, pose, [cam], [gF], [gA], storage="bf16")
    fb = torch.from_numpy(sc.octree.features).to(torch.bfloat16).to(torch.float64).numpy()
    o = _oracle_grads(sc, pose, [cam], [gF], [gA], features=fb)
    _close(g[0], o[0], 3e-4, "dL/df (bf16 storage)")
    _close(g[1], o[1], 1e-3, "dL/dsigma (bf16 storage)")
    _close(g[2], o[2], 5e-3, "dL/dw (bf16 storage)")
