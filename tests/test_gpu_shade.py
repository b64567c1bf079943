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


def _unet_bf16_emulated(F, layers):
    """FP64 U-Net that rounds to BF16 exactly where the tensor-core path
    stores BF16: the input, the 3x3 weights and every stored activation; the
    1x1 head reads the last convolution's FP32 output (fused epilogue)."""
    import torch
    import torch.nn.functional as Fn
    bf = lambda t: t.to(torch.bfloat16).to(torch.float64)
    L = [(bf(torch.from_numpy(w.astype(np.float64))).permute(0, 3, 1, 2), torch.from_numpy(b.astype(np.float64)))
         for w, b in layers]
    conv = lambda t, i: torch.relu(Fn.conv2d(t, L[i][0], L[i][1], padding=1))
    up = lambda z: Fn.interpolate(z, scale_factor=2, mode="nearest")
    t = bf(torch.from_numpy(F.astype(np.float64)).permute(2, 0, 1)[None])
    e0 = bf(conv(bf(conv(t, 0)), 1))
    e1 = bf(conv(bf(conv(Fn.max_pool2d(e0, 2), 2)), 3))
    e2 = bf(conv(bf(conv(Fn.max_pool2d(e1, 2), 4)), 5))
    e3 = bf(conv(bf(conv(Fn.max_pool2d(e2, 2), 6)), 7))
    d2 = bf(conv(bf(conv(torch.cat([up(e3), e2], 1), 8)), 9))
    d1 = bf(conv(bf(conv(torch.cat([up(d2), e1], 1), 10)), 11))
    d0 = conv(bf(conv(torch.cat([up(d1), e0], 1), 12)), 13)  # FP32 in the fused epilogue
    wh = torch.from_numpy(layers[14][0].astype(np.float64)).to(torch.bfloat16).to(torch.float64)
    head = Fn.conv2d(d0, wh.permute(0, 3, 1, 2), torch.from_numpy(layers[14][1].astype(np.float64)))
    return torch.sigmoid(head)[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("H,W", [(64, 64), (136, 264)])
def test_unet_bf16_tensor_cores_match_emulation(H, W):
    """Every 3x3 layer on tcgen05 (BF16 x BF16 -> FP32): equal to the emulated
    BF16 network up to FP32 summation order and the BF16 roundings it flips."""
    import paper_2202_05628_gb300 as art
    rng = np.random.default_rng(H * W)
    F = (rng.standard_normal((H, W, 32)) * 0.3).astype(np.float32)
    F[rng.uniform(size=(H, W)) < 0.3] = 0.0
    layers = sg.unet_weights(5, cin=32)
    ref = _unet_bf16_emulated(F, layers)
    sc = sg.preset("mini")
    r = renderer(sc, profile=True)
    cam = sg.orbit_camera(sc.centroid, W, H)
    set_cam(r, 0, cam)
    r.load_shader(art.ART_NET_UNET, 32, sg.UNET_CHANNELS, 4, art.flat_params(layers), "bf16")
    rgba = _shade(r, 0, F, cam, F_dtype="bf16")
    r.sync_status()
    kt = r.kernel_times()
    assert kt.get("conv_tc", (0, 0))[0] == 14, kt  # the 14 3x3 layers ran on the tensor cores
    # A different FP32 summation order flips a few BF16 roundings per layer
    # (one BF16 ulp, 2^-8 relative, each) and the flips spread through 15
    # layers: mean ~3e-4 here, while an indexing or swizzle slip gives ~1e-1.
    d = np.abs(rgba - ref)
    assert d.mean() < 1e-3 and d.max() < 2e-2, (d.mean(), d.max())
    assert psnr(rgba, ref) > 60.0


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
