"""Edge sizes of the rendering path on the GPU against the FP64 oracle:
ragged screen tiles (image sides that are not multiples of the 8 x 4 tile),
a one-pixel image, a one-voxel octree, and a view that sees nothing.

Pixels whose F the rounding of entry distances decides are left out of the
element-wise comparison (helpers.order_ambiguous: two consecutive hits with
entry distances within 1e-6 m whose swap moves a channel by more than 1e-5);
a grazing hit missing on one side changes F by less than 1e-5 and needs no
exclusion."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import order_ambiguous, render_maps, renderer, set_cam, set_pose

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("W,H,az,fov", [(100, 70, 30.0, 12.0), (37, 29, 150.0, 8.0), (1, 1, 60.0, 2.0)])
def test_ragged_tiles_match_oracle(W, H, az, fov):
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, W, H, az_deg=az, fov_deg=fov)
    pose = sg.random_pose(3)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, oc.C)
    assert F.shape == (H, W, oc.C) and np.all(np.isfinite(F)) and np.all(np.isfinite(A))
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(oc, A_or, cam, hits=True)
    keep = ~order_ambiguous(o, oc, H, W)
    cov = o["A"] > 0
    assert cov.sum() >= min(W * H // 4, 50), cov.sum()
    assert (keep & cov).sum() >= 0.9 * cov.sum()
    assert np.abs(F - o["F"])[keep].max() < TOL_F32
    assert np.abs(A - o["A"])[keep].max() < TOL_F32
    # the split walk with short segments on the same ragged tiles
    r.set_config(segment=32)
    F2, A2 = render_maps(r, 0, cam, oc.C)
    assert np.abs(F2 - F).max() < 1e-6 and np.abs(A2 - A).max() < 1e-6


def test_view_that_sees_nothing():
    sc = sg.preset("tiny")
    oc = sc.octree
    # from the centroid's far side, looking away from the animal
    c = sg.orbit_camera(sc.centroid, 64, 48, az_deg=0.0)
    M = np.asarray(c.world_to_cam, np.float64).reshape(3, 4)
    eye = -M[:, :3].T @ M[:, 3]
    away = eye + (eye - sc.centroid)
    cam = sg.Camera(c.W, c.H, c.fx, c.fy, c.cx, c.cy, sg.look_at(eye, away), c.near, c.far)
    r = renderer(sc)
    set_pose(r, sg.random_pose(2))
    set_cam(r, 0, cam)
    r.set_config(segment=32)
    F, A = render_maps(r, 0, cam, oc.C)
    st = r.sync_status()
    assert st["instances"] == 0
    assert np.all(F == 0.0) and np.all(A == 0.0)
    _, A_or, _ = oracle.pose_transforms(sc, sg.random_pose(2))
    o = oracle.render(oc, A_or, cam)
    assert np.all(o["A"] == 0.0)


def test_one_voxel_octree_matches_the_closed_form():
    # a single leaf on the optical axis at the rest pose: the centre pixel's
    # chord is the leaf's side h and F = (1 - exp(-sigma h)) f
    depth, extent = 4, 1.0
    h = extent / (1 << depth)
    ijk = np.array([[8, 8, 8]], np.uint16)
    f = np.array([[0.5, -1.0, 2.0, 0.25, -0.75, 1.5, 0.0, 3.0]], np.float32)
    sigma = np.array([30.0], np.float32)
    jidx = np.zeros((1, 4), np.uint8)
    w = np.array([[1.0, 0.0, 0.0, 0.0]], np.float32)
    oc = sg.Octree(depth, np.array([-0.5, -0.5, -0.5], np.float32), extent, ijk, jidx, w, f, sigma,
                   np.zeros(1, np.float32))
    skel = sg.Skeleton(np.array([-1, 0], np.int32), np.array([[0, 0, 0], [0.1, 0, 0]], np.float32))
    sc = sg.Scene(oc, skel, np.zeros(3), 1.0, None, None)
    centre = oc.centers()[0].astype(np.float64)
    eye = centre + np.array([0.0, 0.0, -1.0])
    cam = sg.Camera(9, 9, 200.0, 200.0, 4.5, 4.5, sg.look_at(eye, centre), 0.1, 3.0)
    r = renderer(sc)
    set_pose(r, sg.rest_pose(2))
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, 8)
    a = 1.0 - np.exp(-30.0 * h)
    np.testing.assert_allclose(A[4, 4], a, atol=1e-5)
    np.testing.assert_allclose(F[4, 4], a * f[0], atol=1e-5)
    o = oracle.render(oc, oracle.pose_transforms(sc, sg.rest_pose(2))[1], cam)
    np.testing.assert_allclose(F, o["F"], atol=TOL_F32)
    np.testing.assert_allclose(A, o["A"], atol=TOL_F32)
