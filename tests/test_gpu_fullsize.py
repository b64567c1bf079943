"""GPU parity at the workloads' full sizes, on sampled pixels that the FP64
oracle computes one by one (brute force over every voxel), in the launch
configuration the benchmark times.

- 1M voxels, FP32 features, one 1024x1024 view of the walk cycle: the plain
  FP32 form, within 1e-4 on every sampled pixel except those whose F the
  rounding of entry distances decides: two consecutive composited hits with
  entry distances within 1e-6 m (2.5x the FP32 error of a difference of two
  entry distances at 2 m) whose swap would move a channel by more than
  1e-5 (the oracle reports T alpha_i alpha_j |f_i - f_j| per pixel).
- 1M voxels, BF16 features, the stereo pair of 1920x1080 views (6.4 cm
  baseline) with the learned interval skip and the trained proposal: every
  sampled pixel within the skip's lost-mass bound (max_missed = 1e-3 of the
  feature scale and of alpha) of the oracle run on the same BF16-rounded
  features.
"""
import os

import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import renderer, set_cam, set_pose

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROPOSAL = os.path.join(ROOT, "paper_2202_05628_gb300", "weights", "proposal_quadruped_1m_1024.bin")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _samples(A, n_cov, n_bg, seed):
    """Seeded pixel sample: n_cov pixels the animal covers (A > 0), n_bg others."""
    rng = np.random.default_rng(seed)
    cov = np.flatnonzero(A.reshape(-1) > 0)
    bg = np.flatnonzero(A.reshape(-1) <= 0)
    pick = np.concatenate([rng.choice(cov, min(n_cov, cov.size), replace=False),
                           rng.choice(bg, min(n_bg, bg.size), replace=False)])
    W = A.shape[1]
    return pick % W, pick // W


def _check(F, A, o, px, py, tol_f, tol_a, what, exclude=None):
    dF = np.abs(F[py, px] - o["F"]).max(1)
    dA = np.abs(A[py, px] - o["A"])
    keep = np.ones(dF.shape, bool) if exclude is None else ~exclude
    ok = (dF <= tol_f) & (dA <= tol_a)
    msg = (f"{what}: {int(ok[keep].sum())} of {int(keep.sum())} compared pixels within ({tol_f:.2e}, {tol_a:.2e}) "
           f"({int((~keep).sum())} order-ambiguous left out); max |dF| {dF[keep].max():.3e}, "
           f"max |dA| {dA[keep].max():.3e}; over all samples max |dF| {dF.max():.3e}")
    print(msg)
    assert ok[keep].all(), msg


def test_fullsize_plain_f32_1024_sampled():
    import torch
    sc = sg.preset("paper")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 1024, 1024, az_deg=135.0)
    pose = sg.walk_pose(17, 60)
    r = renderer(sc, storage="f32")
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F = torch.zeros((cam.H, cam.W, oc.C), dtype=torch.float32, device="cuda")
    A = torch.zeros((cam.H, cam.W), dtype=torch.float32, device="cuda")
    r.render_feature_maps(0, F, A)
    st = r.sync_status()
    assert st["overflow_inst"] == 0 and st["overflow_order"] == 0
    F, A = F.cpu().numpy(), A.cpu().numpy()
    px, py = _samples(A, 384, 64, seed=11)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.pixels(oc, A_or, cam, px, py, tie_eps=1e-6)
    tied = o["tie"] > 1e-5
    assert tied.mean() <= 0.1, tied.mean()
    _check(F, A, o, px, py, 1e-4, 1e-4, "1M voxels, FP32 plain, 1024^2", exclude=tied)


def test_fullsize_stereo_1080p_bf16_learned_skip_sampled():
    import torch
    from paper_2202_05628_gb300 import proposal as prop
    if not os.path.exists(PROPOSAL):
        pytest.skip("trained proposal weights missing")
    sc = sg.preset("paper")
    oc = sc.octree
    cams = [sg.orbit_camera(sc.centroid, 1920, 1080, az_deg=60.0, shift_x=s) for s in (-0.032, 0.032)]
    pose = sg.walk_pose(41, 60)
    r = renderer(sc, storage="bf16")
    r.load_proposal(prop.load(PROPOSAL)[0])
    r.set_config(skip=1, max_missed=1e-3, margin=1)
    set_pose(r, pose)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    feat16 = oracle.round_bf16(oc.features)
    fmax = float(np.abs(feat16).max())
    fb, act = 0, 0
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
        F = torch.zeros((cam.H, cam.W, oc.C), dtype=torch.float32, device="cuda")
        A = torch.zeros((cam.H, cam.W), dtype=torch.float32, device="cuda")
        r.render_feature_maps(v, F, A)
        st = r.sync_status()
        assert st["overflow_inst"] == 0 and st["overflow_order"] == 0
        ranges = r.debug_buffer(7, np.uint32).reshape(-1, 2)
        act += int(np.sum(ranges[:, 1] > ranges[:, 0]))
        fb += st["check_fail_tiles"]
        F, A = F.cpu().numpy(), A.cpu().numpy()
        px, py = _samples(A, 256, 32, seed=20 + v)
        o = oracle.pixels(oc, A_or, cam, px, py, features=feat16)
        _check(F, A, o, px, py, 1e-3 * fmax * (1 + 1e-3) + 1e-4, 1e-3 * (1 + 1e-3) + 1e-4,
               f"1M voxels, BF16 + learned skip, 1920x1080 eye {v}")
    print(f"stereo 1080p: {fb} of {act} active tiles fell back to the full traversal")
    assert fb < act
