"""GPU parity of the shading network (Sec. 3.1 "Neural Shading") against the
FP64 oracle, through the C ABI: FP32 form within 1e-4, BF16 form by PSNR."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import psnr, render_maps, renderer, set_cam, set_pose, tiny_setup

pytestmark = pytest.mark.gpu
TOL_F32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shade(r, view, F, cam, cout=4, F_dtype="f32"):
    import torch
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).cuda()
    if F_dtype == "bf16":
        Ft = Ft.to(torch.bfloat16)
    out = torch.empty((cam.H, cam.W, cout), dtype=torch.float32, device="cuda")
    r.shade(view, Ft, out, F_dtype)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_tiny_net_f32_matches_oracle():
    import paper_2202_05628_gb300 as art
    sc, cam, pose = tiny_setup(az=10.0, pose_seed=2)
    layers = sg.tiny_net_weights(0, cin=16)
    r = renderer(sc)
    r.load_shader(art.ART_NET_TINY, 16, [32], 4, art.flat_params(layers), "f32")
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, 16)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(sc.octree, A_or, cam)
    rgba_or = oracle.shade(o["F"], layers)
    rgba = _shade(r, 0, F, cam)
    assert np.abs(rgba - rgba_or).max() < TOL_F32
    # whole frame through art_render_frame, host output
    out = np.zeros((cam.H, cam.W, 4), np.float32)
    r.render_frame(0, pose.axis_angle, pose.R, pose.T, out)
    assert np.abs(out - rgba_or).max() < TOL_F32


@pytest.mark.parametrize("H,W", [(64, 64), (96, 160)])
def test_unet_f32_matches_oracle(H, W):
    import paper_2202_05628_gb300 as art
    rng = np.random.default_rng(H + W)
    F = (rng.standard_normal((H, W, 32)) * 0.3).astype(np.float32)
    F[rng.uniform(size=(H, W)) < 0.5] = 0.0
    layers = sg.unet_weights(1, cin=32)
    ref = oracle.shade_unet(F.astype(np.float64), layers)
    sc = sg.preset("mini")
    r = renderer(sc)
    cam = sg.orbit_camera(sc.centroid, W, H)
    set_cam(r, 0, cam)
    r.load_shader(art.ART_NET_UNET, 32, sg.UNET_CHANNELS, 4, art.flat_params(layers), "f32")
    rgba = _shade(r, 0, F, cam)
    assert np.abs(rgba - ref).max() < TOL_F32


def test_unet_bf16_psnr():
    import paper_2202_05628_gb300 as art
    H = W = 128
    rng = np.random.default_rng(7)
    F = (rng.standard_normal((H, W, 32)) * 0.3).astype(np.float32)
    layers = sg.unet_weights(2, cin=32)
    ref = oracle.shade_unet(F.astype(np.float64), layers)
    sc = sg.preset("mini")
    r = renderer(sc)
    cam = sg.orbit_camera(sc.centroid, W, H)
    set_cam(r, 0, cam)
    r.load_shader(art.ART_NET_UNET, 32, sg.UNET_CHANNELS, 4, art.flat_params(layers), "bf16")
    rgba = _shade(r, 0, F, cam, F_dtype="bf16")
    p = psnr(rgba, ref)
    assert p >= 45.0, (p, np.abs(rgba - ref).max())
