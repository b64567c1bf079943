"""View-dependent features (Eq. 2, with the ray mapped into each voxel's
canonical frame, Sec. 3.1) on the GPU against the FP64 oracle, through the
C ABI."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import order_ambiguous, renderer, set_cam, set_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _maps(r, cam, C):
    import torch
    F = torch.empty((cam.H, cam.W, C), dtype=torch.float32, device="cuda")
    A = torch.empty((cam.H, cam.W), dtype=torch.float32, device="cuda")
    r.render_feature_maps(0, F, A)
    return F.cpu().numpy().astype(np.float64), A.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("L,pose_seed,az", [(0, 2, 30.0), (1, 5, 150.0), (3, 7, 250.0)])
def test_sh_features_match_oracle(L, pose_seed, az):
    """Within 1e-4 of the oracle on every pixel whose hit order rounding
    cannot decide (no two consecutive composited hits with entry distances
    within 1e-6 m)."""
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 128, 96, az_deg=az, fov_deg=12.0)
    pose = sg.random_pose(pose_seed)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F0, A0 = _maps(r, cam, oc.C)  # plain features, for the switch back below
    p = oracle.render(oc, A_or, cam, hits=True)
    good = ~order_ambiguous(p, oc, cam.H, cam.W, effect=0.0)
    assert good.mean() > 0.8, good.mean()
    coef = (0.3 * np.random.default_rng(10 + L).standard_normal((oc.n, (L + 1) ** 2, oc.C))).astype(np.float32)
    r.load_sh_features(L, coef)
    F, A = _maps(r, cam, oc.C)
    o = oracle.render_sh(oc, A_or, cam, L, coef.astype(np.float64))
    assert (o["A"] > 0).sum() > 500
    np.testing.assert_allclose(A[good], o["A"][good], atol=1e-4)
    np.testing.assert_allclose(F[good], o["F"][good], atol=1e-4)
    # back to the per-voxel features
    r.load_sh_features(-1)
    F1, A1 = _maps(r, cam, oc.C)
    np.testing.assert_array_equal(F1, F0)
    np.testing.assert_array_equal(A1, A0)


def test_sh_features_refuse_unsupported_uses():
    import torch
    import paper_2202_05628_gb300 as art
    sc = sg.preset("tiny")
    oc = sc.octree
    r = renderer(sc)
    with pytest.raises(art.ArtemisError):
        r.load_sh_features(4, np.zeros((oc.n, 25, oc.C), np.float32))  # degree above 3
    r.load_sh_features(1, np.zeros((oc.n, 4, oc.C), np.float32))
    cam = sg.orbit_camera(sc.centroid, 32, 32)
    set_cam(r, 0, cam)
    set_pose(r, sg.random_pose(1))
    z = torch.zeros((32, 32, oc.C), device="cuda")
    a = torch.zeros((32, 32), device="cuda")
    with pytest.raises(art.ArtemisError):
        r.render_backward(0, z, a, z, a, torch.zeros_like(torch.from_numpy(oc.features)).cuda(),
                          torch.zeros(oc.n, device="cuda"), torch.zeros((oc.n, 4), device="cuda"))
