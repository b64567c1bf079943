"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test fixes one function of ``oracle/`` against a closed form, brute
force, an invariant of the method, or an independent library routine, chosen
so that a plausible slip (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.  Paper: arXiv 2202.05628, Sec. 3.1.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers: hand-made scenes
# ---------------------------------------------------------------------------

def one_joint_skeleton(J=2):
    parent = np.array([-1] + list(range(J - 1)), np.int32)
    rest = np.zeros((J, 3), np.float32)
    for j in range(1, J):
        rest[j] = rest[j - 1] + np.array([0.1, 0.0, 0.0], np.float32)
    return sg.Skeleton(parent, rest)


def make_octree(ijk, depth=4, extent=1.0, origin=(-0.5, -0.5, -0.5), feats=None, dens=None,
                jidx=None, w=None, C=3, seed=0):
    ijk = np.asarray(ijk, np.uint16).reshape(-1, 3)
    n = ijk.shape[0]
    rng = np.random.default_rng(seed)
    feats = rng.standard_normal((n, C)).astype(np.float32) if feats is None else np.asarray(feats, np.float32)
    dens = np.full(n, 3.0, np.float32) if dens is None else np.asarray(dens, np.float32)
    jidx = np.zeros((n, 4), np.uint8) if jidx is None else np.asarray(jidx, np.uint8)
    if w is None:
        w = np.zeros((n, 4), np.float32)
        w[:, 0] = 1.0
    return sg.Octree(depth, np.asarray(origin, np.float32), extent, ijk, jidx, np.asarray(w, np.float32),
                     feats, dens, np.zeros(n, np.float32))


def axis_camera(target, direction, dist=1.0, W=1, H=1, f=100.0, near=0.05, far=5.0):
    """Camera whose pixel (0, 0) centre ray passes through ``target`` along
    unit ``direction`` (the optical axis, since cx = cy = 0.5)."""
    d = np.asarray(direction, np.float64)
    d /= np.linalg.norm(d)
    eye = np.asarray(target, np.float64) - dist * d
    up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.9 else (1.0, 0.0, 0.0)
    M = sg.look_at(eye, target, up)
    return sg.Camera(W=W, H=H, fx=f, fy=f, cx=0.5, cy=0.5, world_to_cam=M,
                     near=near, far=far)


def identity_A(n):
    A = np.zeros((n, 3, 4))
    A[:, 0, 0] = A[:, 1, 1] = A[:, 2, 2] = 1.0
    return A


def voxel_center(oc, i):
    return oc.centers()[i]


# ---------------------------------------------------------------------------
# Eq. 4: forward kinematics and LBS
# ---------------------------------------------------------------------------

def test_rodrigues_matches_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(3)
    for _ in range(50):
        r = rng.standard_normal(3) * rng.uniform(0, 3)
        np.testing.assert_allclose(oracle.rodrigues(r), Rot.from_rotvec(r).as_matrix(), atol=1e-13)
    np.testing.assert_array_equal(oracle.rodrigues(np.zeros(3)), np.eye(3))


def test_fk_rest_pose_is_identity():
    sc = sg.preset("mini")
    G = oracle.fk(sc.skeleton, sg.rest_pose())
    for j in range(G.shape[0]):
        np.testing.assert_allclose(G[j], np.hstack([np.eye(3), np.zeros((3, 1))]), atol=1e-15)


def test_fk_two_joint_closed_form():
    # root at origin, child at (0.1, 0, 0); rotate the root 90 deg about z:
    # the child joint moves to (0, 0.1, 0) and a point on the child's bone
    # (0.15, 0, 0) moves to (0, 0.15, 0).
    sk = one_joint_skeleton(2)
    aa = np.zeros((2, 3), np.float32)
    aa[0] = [0, 0, math.pi / 2]
    G = oracle.fk(sk, sg.Pose(aa, np.zeros(3, np.float32), np.zeros(3, np.float32)))
    p = np.array([0.15, 0.0, 0.0, 1.0])
    np.testing.assert_allclose(G[1] @ p, [0.0, 0.15, 0.0], atol=1e-7)
    np.testing.assert_allclose(G[1] @ np.array([0.1, 0, 0, 1.0]), [0.0, 0.1, 0.0], atol=1e-7)
    # a child rotation about z by -90 deg restores the orientation beyond the
    # child joint, which itself sits at (0, 0.1, 0)
    aa[1] = [0, 0, -math.pi / 2]
    G = oracle.fk(sk, sg.Pose(aa, np.zeros(3, np.float32), np.zeros(3, np.float32)))
    np.testing.assert_allclose(G[1] @ p, [0.05, 0.1, 0.0], atol=1e-7)


def test_fk_preserves_bones_and_global_rigid():
    sc = sg.preset("mini")
    sk = sc.skeleton
    pose = sg.random_pose(5)
    G = oracle.fk(sk, pose)
    rest = sk.rest.astype(np.float64)
    posed = np.einsum("jab,jb->ja", G[:, :, :3], rest) + G[:, :, 3]
    for j in range(1, sk.J):
        p = sk.parent[j]
        assert abs(np.linalg.norm(posed[j] - posed[p]) - np.linalg.norm(rest[j] - rest[p])) < 1e-6
        Rj = G[j, :, :3]
        np.testing.assert_allclose(Rj @ Rj.T, np.eye(3), atol=1e-6)
        assert abs(np.linalg.det(Rj) - 1) < 1e-6
    # global R, T compose on the left of every joint transform
    Rg = np.array([0.3, -0.2, 0.5], np.float32)
    Tg = np.array([0.1, 0.2, -0.3], np.float32)
    G2 = oracle.fk(sk, sg.Pose(pose.axis_angle, Rg, Tg))
    Rm = oracle.rodrigues(Rg)
    for j in range(sk.J):
        np.testing.assert_allclose(G2[j, :, :3], Rm @ G[j, :, :3], atol=1e-12)
        np.testing.assert_allclose(G2[j, :, 3], Rm @ G[j, :, 3] + Tg, atol=1e-7)


def test_fk_rejects_bad_parent():
    sk = sg.Skeleton(np.array([-1, 2, 0], np.int32), np.zeros((3, 3), np.float32))
    with pytest.raises(ValueError):
        oracle.fk(sk, sg.rest_pose(3))


def test_lbs_one_hot_and_linearity():
    sc = sg.preset("mini")
    oc = sc.octree
    G = oracle.fk(sc.skeleton, sg.random_pose(2))
    w1 = np.zeros_like(oc.weights)
    w1[:, 0] = 1.0
    A1, det = oracle.lbs(oc, G, w1)
    np.testing.assert_allclose(A1, G[oc.joint_idx[:, 0]], atol=0)
    np.testing.assert_allclose(det, 1.0, atol=1e-6)
    # A is linear in the weights: A(a w + b w') = a A(w) + b A(w')
    rng = np.random.default_rng(0)
    wa = rng.uniform(0, 1, oc.weights.shape)
    wb = rng.uniform(0, 1, oc.weights.shape)
    Aa, _ = oracle.lbs(oc, G, wa)
    Ab, _ = oracle.lbs(oc, G, wb)
    Ac, _ = oracle.lbs(oc, G, 0.3 * wa + 0.7 * wb)
    np.testing.assert_allclose(Ac, 0.3 * Aa + 0.7 * Ab, atol=1e-12)
    # rest pose: every voxel keeps its canonical position
    A0, det0 = oracle.lbs(oc, oracle.fk(sc.skeleton, sg.rest_pose()))
    np.testing.assert_allclose(A0, identity_A(oc.n), atol=1e-7)


# ---------------------------------------------------------------------------
# rays
# ---------------------------------------------------------------------------

def test_pixel_ray_reprojects_to_pixel_centre():
    sc = sg.preset("mini")
    cam = sg.orbit_camera(sc.centroid, 40, 30, az_deg=37.0)
    M = cam.world_to_cam.astype(np.float64)
    for (x, y) in [(0, 0), (39, 29), (17, 11), (5, 28)]:
        o, d = oracle.pixel_ray(cam, x, y)
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        np.testing.assert_allclose(M[:, :3] @ o + M[:, 3], 0, atol=1e-6)
        p = M[:, :3] @ (o + 1.7 * d) + M[:, 3]
        np.testing.assert_allclose([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy],
                                   [x + 0.5, y + 0.5], atol=1e-5)


# ---------------------------------------------------------------------------
# Eq. 5-6: closed forms for one and two voxels
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("direction", [(0, 0, 1), (1, 0, 0), (0.3, -0.2, 1.0), (1.0, 0.9, -0.4), (-0.2, 1.0, 0.05)])
def test_single_voxel_chord_through_centre(direction):
    # A ray through the centre of an axis-aligned cube of side h travels
    # h / max_a |d_a| inside it.
    oc = make_octree([[7, 8, 9]], C=4)
    c = voxel_center(oc, 0)
    cam = axis_camera(c, direction)
    d = np.asarray(direction, float) / np.linalg.norm(direction)
    chord = oc.h / np.max(np.abs(d))
    r = oracle.render(oc, identity_A(1), cam, hits=True)
    sigma = float(oc.density[0])
    a = 1 - math.exp(-sigma * chord)
    np.testing.assert_allclose(r["F"][0, 0], a * oc.features[0].astype(float), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["A"][0, 0], a, rtol=1e-12)
    np.testing.assert_allclose(r["hit_t1"] - r["hit_t0"], [chord], rtol=1e-12)


def test_single_warped_voxel_chord():
    # A = blend of two rotations (not rigid).  In the canonical frame the
    # direction is d' = A_lin^-1 d (unnormalised) and, through the centre, the
    # ray is inside the cube for |t d'_a| <= h/2 on every axis: chord =
    # h / max_a |d'_a|.
    oc = make_octree([[3, 4, 5]], C=2)
    R1 = oracle.rodrigues([0.0, 0.0, 0.6])
    R2 = oracle.rodrigues([0.4, 0.1, 0.0])
    L = 0.5 * (R1 + R2)
    c = voxel_center(oc, 0)
    t = np.array([0.05, -0.02, 0.03])
    A = np.zeros((1, 3, 4))
    A[0, :, :3] = L
    A[0, :, 3] = t
    cw = L @ c + t
    for direction in [(0, 0, 1), (0.5, 0.2, -1.0), (1, 1, 1)]:
        cam = axis_camera(cw, direction, dist=1.3)
        d = np.asarray(direction, float) / np.linalg.norm(direction)
        dl = np.linalg.solve(L, d)
        chord = oc.h / np.max(np.abs(dl))
        r = oracle.render(oc, A, cam, hits=True)
        np.testing.assert_allclose(r["hit_t1"] - r["hit_t0"], [chord], rtol=1e-10)
        np.testing.assert_allclose(r["hit_t0"] + r["hit_t1"], [2 * 1.3], rtol=1e-10)


def test_two_stacked_voxels_closed_form():
    # F = a1 f1 + (1 - a1) a2 f2, A = 1 - (1 - a1)(1 - a2) for two voxels
    # stacked along the ray (exclusive transmittance, Eq. 6 read with j < i).
    oc = make_octree([[5, 5, 5], [5, 5, 6]], dens=[7.0, 11.0], C=3)
    c0, c1 = voxel_center(oc, 0), voxel_center(oc, 1)
    cam = axis_camera(c0, (0, 0, 1))  # enters voxel 0 first
    r = oracle.render(oc, identity_A(2), cam, hits=True)
    a1 = 1 - math.exp(-7.0 * oc.h)
    a2 = 1 - math.exp(-11.0 * oc.h)
    f = oc.features.astype(float)
    np.testing.assert_allclose(r["F"][0, 0], a1 * f[0] + (1 - a1) * a2 * f[1], rtol=1e-12)
    np.testing.assert_allclose(r["A"][0, 0], 1 - (1 - a1) * (1 - a2), rtol=1e-12)
    assert list(r["hit_id"]) == [0, 1]
    # looking from the other side reverses the order
    cam = axis_camera(c1, (0, 0, -1))
    r = oracle.render(oc, identity_A(2), cam, hits=True)
    np.testing.assert_allclose(r["F"][0, 0], a2 * f[1] + (1 - a2) * a1 * f[0], rtol=1e-12)
    assert list(r["hit_id"]) == [1, 0]


def test_pixels_tie_effect_closed_form():
    # Two coincident voxels (the same cell, different features and
    # densities) are entered at the same distance: their order is a tie, and
    # swapping them changes F by alpha_1 alpha_2 (f_1 - f_2) (T = 1 before
    # them); a third voxel stacked behind is no tie.  The oracle's per-pixel
    # report is the largest channel of that change, 0 for tie_eps below every
    # gap, and 0 for a pixel with a single hit.
    oc = make_octree([[5, 5, 5], [5, 5, 5], [5, 5, 6]], dens=[7.0, 11.0, 5.0], C=3)
    c0 = voxel_center(oc, 0)
    cam = axis_camera(c0, (0, 0, 1))
    a1 = 1 - math.exp(-7.0 * oc.h)
    a2 = 1 - math.exp(-11.0 * oc.h)
    f = oc.features.astype(float)
    o = oracle.pixels(oc, identity_A(3), cam, [0], [0], tie_eps=1e-6)
    np.testing.assert_allclose(o["tie"][0], a1 * a2 * np.abs(f[0] - f[1]).max(), rtol=1e-12)
    # the two orders' sums, written out
    F01 = a1 * f[0] + (1 - a1) * a2 * f[1]
    F10 = a2 * f[1] + (1 - a2) * a1 * f[0]
    np.testing.assert_allclose(np.abs(F01 - F10).max(), o["tie"][0], rtol=1e-12)
    assert oracle.pixels(oc, identity_A(3), cam, [0], [0], tie_eps=0.0)["tie"][0] == 0.0
    one = make_octree([[5, 5, 5]], C=3)
    assert oracle.pixels(one, identity_A(1), cam, [0], [0])["tie"][0] == 0.0


def test_near_far_clip():
    oc = make_octree([[8, 8, 8]], C=1)
    c = voxel_center(oc, 0)
    # camera 1.0 from the centre; near plane cuts the voxel 0.3 h past its entry
    near = 1.0 - 0.5 * oc.h + 0.3 * oc.h
    cam = axis_camera(c, (0, 0, 1), dist=1.0, near=near)
    r = oracle.render(oc, identity_A(1), cam, hits=True)
    np.testing.assert_allclose(r["hit_t1"] - r["hit_t0"], [0.7 * oc.h], rtol=1e-9)
    far = 1.0 - 0.5 * oc.h + 0.2 * oc.h
    cam = axis_camera(c, (0, 0, 1), dist=1.0, near=0.1, far=far)
    r = oracle.render(oc, identity_A(1), cam, hits=True)
    np.testing.assert_allclose(r["hit_t1"] - r["hit_t0"], [0.2 * oc.h], rtol=1e-9)
    cam = axis_camera(c, (0, 0, 1), dist=1.0, near=1.1)
    assert oracle.render(oc, identity_A(1), cam)["nhit"][0, 0] == 0


def test_golden_fixtures():
    """Closed-form fixtures written by tests/golden/make_golden.py (exact
    arithmetic in sympy, independent of the oracle)."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as fh:
        cases = json.load(fh)["cases"]
    assert len(cases) >= 3
    for case in cases:
        oc = make_octree(case["ijk"], depth=case["depth"], feats=case["features"], dens=case["density"],
                         C=len(case["features"][0]))
        cam = axis_camera(np.asarray(case["target"]), case["direction"], dist=case["dist"])
        r = oracle.render(oc, identity_A(oc.n), cam, tau=case["tau"], hits=True)
        np.testing.assert_allclose(r["F"][0, 0], case["F"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["A"][0, 0], case["A"], rtol=1e-12)
        assert list(r["hit_id"]) == case["order"]
        assert int(r["nused"][0, 0]) == case["used"]


# ---------------------------------------------------------------------------
# hit lists: brute force, invariants
# ---------------------------------------------------------------------------

def test_candidate_lists_equal_brute_force():
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 64, 64, az_deg=30)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(11))
    r = oracle.render(oc, A, cam, hits=True)
    rng = np.random.default_rng(0)
    ys, xs = np.nonzero(r["nhit"] >= 0)
    pick = rng.choice(len(ys), 60, replace=False)
    covered = np.argwhere(r["nhit"] > 0)
    pick_c = covered[rng.choice(len(covered), min(60, len(covered)), replace=False)]
    for y, x in list(zip(ys[pick], xs[pick])) + [tuple(p) for p in pick_c]:
        b = oracle.pixel_brute(oc, A, cam, int(x), int(y))
        p = y * cam.W + x
        ids = r["hit_id"][r["hit_off"][p]:r["hit_off"][p + 1]]
        np.testing.assert_array_equal(b["ids"], ids)
        np.testing.assert_array_equal(b["F"], r["F"][y, x])


def test_all_ones_features_give_accumulated_alpha():
    # With f_i = 1, F = sum_i T_i a_i must equal A = 1 - T_final (exclusive T).
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 128, 128, az_deg=80)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(4))
    ones = np.ones((oc.n, 1))
    r = oracle.render(oc, A, cam, features=ones)
    np.testing.assert_allclose(r["F"][..., 0], r["A"], atol=1e-13)
    assert r["A"].min() >= 0 and r["A"].max() <= 1
    assert (r["A"] > 0).sum() > 100


def test_transmittance_monotone_and_early_stop():
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 128, 128)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(4))
    dens = oc.density.astype(float) * 60.0  # opaque animal so that the stop fires
    tau = 1e-4
    r = oracle.render(oc, A, cam, tau=tau, hits=True, density=dens)
    stopped = np.argwhere(r["nused"] < r["nhit"])
    assert len(stopped) > 20
    for y, x in stopped[:50]:
        p = y * cam.W + x
        s, e = r["hit_off"][p], r["hit_off"][p + 1]
        ids = r["hit_id"][s:e]
        delta = r["hit_t1"][s:e] - r["hit_t0"][s:e]
        assert np.all(delta > 0)
        T = np.exp(-np.cumsum(dens[ids] * delta))  # T after each hit: non-increasing
        assert np.all(np.diff(T) <= 0)
        u = r["nused"][y, x]
        assert T[u - 1] < tau and (u == 1 or T[u - 2] >= tau)
        np.testing.assert_allclose(r["A"][y, x], 1 - T[u - 1], rtol=1e-12)
    # tau = 0 composites every hit
    r0 = oracle.render(oc, A, cam, tau=0.0, density=dens)
    assert np.array_equal(r0["nused"], r0["nhit"])


def test_zero_density_voxels_invisible():
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 96, 96, az_deg=200)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(8))
    rng = np.random.default_rng(1)
    drop = rng.uniform(size=oc.n) < 0.4
    dens = oc.density.astype(float).copy()
    dens[drop] = 0.0
    r1 = oracle.render(oc, A, cam, density=dens)
    keep = np.nonzero(~drop)[0]
    r2 = oracle.render(oc.subset(keep), A[keep], cam)
    np.testing.assert_allclose(r1["F"], r2["F"], atol=1e-14)
    np.testing.assert_allclose(r1["A"], r2["A"], atol=1e-14)


def _cam64(cam, M=None):
    """The same camera with an FP64 (exactly orthonormal up to rounding) matrix."""
    if M is None:
        M = sg.look_at(*_eye_target(cam))
    return sg.Camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, M, cam.near, cam.far)


def _eye_target(cam):
    M = cam.world_to_cam.astype(np.float64)
    eye = -M[:, :3].T @ M[:, 3]
    return eye, eye + M[2, :3]


def test_rigid_pose_equals_rigid_camera_motion():
    sc = sg.preset("tiny")
    oc = sc.octree
    pose = sg.random_pose(9)
    Rg = np.array([0.2, -0.4, 0.1], np.float32)
    Tg = np.array([0.05, -0.03, 0.02], np.float32)
    cam = _cam64(sg.orbit_camera(sc.centroid, 128, 128, az_deg=20))
    w64 = oc.weights.astype(np.float64)
    w64 /= w64.sum(1, keepdims=True)
    G1 = oracle.fk(sc.skeleton, sg.Pose(pose.axis_angle, Rg, Tg))
    A1, _ = oracle.lbs(oc, G1, w64)
    r1 = oracle.render(oc, A1, cam)
    # same animal without the global motion, camera moved by it:
    # x_cam = R_c (Rg x + Tg) + t_c
    Rm = oracle.rodrigues(Rg)
    M = cam.world_to_cam
    M2 = np.concatenate([M[:, :3] @ Rm, (M[:, :3] @ Tg.astype(np.float64) + M[:, 3])[:, None]], 1)
    cam2 = _cam64(cam, M2)
    G2 = oracle.fk(sc.skeleton, sg.Pose(pose.axis_angle, np.zeros(3, np.float32), np.zeros(3, np.float32)))
    A2, _ = oracle.lbs(oc, G2, w64)
    r2 = oracle.render(oc, A2, cam2)
    assert (r1["A"] > 0).sum() > 100
    np.testing.assert_allclose(r1["A"], r2["A"], atol=1e-9)
    np.testing.assert_allclose(r1["F"], r2["F"], atol=1e-9)


def test_one_hot_weights_equal_rigid_camera():
    # All voxels bound to one joint: the warp is G_j, i.e. the canonical animal
    # seen by the camera world_to_cam * G_j.
    sc = sg.preset("tiny")
    oc = sc.octree
    w = np.zeros_like(oc.weights)
    w[:, 0] = 1.0
    jidx = np.full_like(oc.joint_idx, 5)
    oc1 = sg.Octree(oc.depth, oc.origin, oc.extent, oc.ijk, jidx, w, oc.features, oc.density, oc.sdf)
    sc1 = sg.Scene(oc1, sc.skeleton, sc.centroid, sc.scale, sc.bones, sc.capsules)
    G, A, _ = oracle.pose_transforms(sc1, sg.random_pose(12))
    cam = _cam64(sg.orbit_camera(sc.centroid, 128, 128, az_deg=-40))
    r1 = oracle.render(oc1, A, cam)
    M = cam.world_to_cam
    Gj = G[5]
    M2 = np.concatenate([M[:, :3] @ Gj[:, :3], (M[:, :3] @ Gj[:, 3] + M[:, 3])[:, None]], 1)
    cam2 = sg.Camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, M2, cam.near, cam.far)
    r2 = oracle.render(oc1, identity_A(oc.n), cam2)
    assert (r1["A"] > 0).sum() > 50
    np.testing.assert_allclose(r1["A"], r2["A"], atol=1e-10)
    np.testing.assert_allclose(r1["F"], r2["F"], atol=1e-10)


def test_voxel_order_invariance():
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 64, 64, az_deg=120)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(3))
    perm = np.random.default_rng(2).permutation(oc.n)
    r1 = oracle.render(oc, A, cam)
    r2 = oracle.render(oc.subset(perm), A[perm], cam)
    np.testing.assert_allclose(r1["F"], r2["F"], atol=1e-12)
    np.testing.assert_allclose(r1["A"], r2["A"], atol=1e-12)


def test_degenerate_blend_dropped():
    # Blending a joint with its 180-degree rotated copy gives det ~ 0.
    oc = make_octree([[8, 8, 8]], C=1, jidx=[[0, 1, 0, 0]], w=[[0.5, 0.5, 0.0, 0.0]])
    sk = one_joint_skeleton(2)
    aa = np.zeros((2, 3), np.float32)
    aa[1] = [0, math.pi, 0]
    G = oracle.fk(sk, sg.Pose(aa, np.zeros(3, np.float32), np.zeros(3, np.float32)))
    sc = sg.Scene(oc, sk, np.zeros(3), 1.0, None, [])
    A, det = oracle.lbs(oc, G)
    assert det[0] < 1e-3
    cam = axis_camera(A[0][:, 3] + A[0][:, :3] @ voxel_center(oc, 0), (0, 0, 1))
    assert oracle.render(oc, A, cam)["nhit"][0, 0] == 0
    assert oracle.voxel_bounds(oc, A, cam)[0, 0] == 0


# ---------------------------------------------------------------------------
# screen-tile coverage
# ---------------------------------------------------------------------------

def test_tile_pairs_match_brute_force_bbox_and_cover_hits():
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 80, 72, az_deg=60)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(6))
    ts, tsy = 16, 8
    tiles, vids = oracle.tile_pairs(oc, A, cam, ts, tsy)
    vb = oracle.voxel_bounds(oc, A, cam)
    tw = (cam.W + ts - 1) // ts
    px = np.arange(cam.W) + 0.5
    py = np.arange(cam.H) + 0.5
    want = set()
    for i in range(oc.n):
        ok, u0, u1, v0, v1, d0, d1 = vb[i]
        if not ok or d0 > cam.far or d1 < cam.near:
            continue
        xs = np.nonzero((px >= u0) & (px <= u1))[0]
        ys = np.nonzero((py >= v0) & (py <= v1))[0]
        for ty in set(ys // tsy):
            for tx in set(xs // ts):
                want.add((int(ty * tw + tx), i))
    got = set(zip(tiles.tolist(), vids.tolist()))
    assert got == want
    r = oracle.render(oc, A, cam, hits=True)
    for p in range(cam.W * cam.H):
        y, x = divmod(p, cam.W)
        t = (y // tsy) * tw + x // ts
        for i in r["hit_id"][r["hit_off"][p]:r["hit_off"][p + 1]]:
            assert (t, int(i)) in got


# ---------------------------------------------------------------------------
# shading network primitives vs torch (FP64, CPU)
# ---------------------------------------------------------------------------

def test_conv_pool_upsample_match_torch():
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    rng = np.random.default_rng(0)
    for (H, W, Cin, Cout, k) in [(9, 7, 5, 6, 3), (8, 12, 3, 4, 1), (1, 1, 2, 3, 3)]:
        x = rng.standard_normal((H, W, Cin))
        w = rng.standard_normal((Cout, k, k, Cin))
        b = rng.standard_normal(Cout)
        tx = torch.from_numpy(x).permute(2, 0, 1)[None]
        tw = torch.from_numpy(w).permute(0, 3, 1, 2)
        ref = Fn.conv2d(tx, tw, torch.from_numpy(b), padding=k // 2)[0].permute(1, 2, 0).numpy()
        np.testing.assert_allclose(oracle.conv2d(x, w, b, oracle.ACT_NONE), ref, atol=1e-12)
        np.testing.assert_allclose(oracle.conv2d(x, w, b, oracle.ACT_RELU), np.maximum(ref, 0), atol=1e-12)
        np.testing.assert_allclose(oracle.conv2d(x, w, b, oracle.ACT_SIGMOID),
                                   torch.sigmoid(torch.from_numpy(ref)).numpy(), atol=1e-12)
    x = rng.standard_normal((6, 10, 3))
    tx = torch.from_numpy(x).permute(2, 0, 1)[None]
    np.testing.assert_array_equal(oracle.maxpool2(x), Fn.max_pool2d(tx, 2)[0].permute(1, 2, 0).numpy())
    np.testing.assert_array_equal(oracle.upsample2(x),
                                  Fn.interpolate(tx, scale_factor=2, mode="nearest")[0].permute(1, 2, 0).numpy())


def test_unet_matches_torch_composition():
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    layers = sg.unet_weights(3, cin=5, ch=(4, 6, 8, 10))
    x = np.random.default_rng(1).standard_normal((16, 24, 5))
    got = oracle.shade_unet(x, layers)

    def conv(t, wb, act):
        w, b = wb
        y = Fn.conv2d(t, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                      torch.from_numpy(b.astype(np.float64)), padding=w.shape[1] // 2)
        return torch.relu(y) if act == "relu" else torch.sigmoid(y)

    t = torch.from_numpy(x).permute(2, 0, 1)[None]
    L = list(layers)
    e0 = conv(conv(t, L[0], "relu"), L[1], "relu")
    e1 = conv(conv(Fn.max_pool2d(e0, 2), L[2], "relu"), L[3], "relu")
    e2 = conv(conv(Fn.max_pool2d(e1, 2), L[4], "relu"), L[5], "relu")
    e3 = conv(conv(Fn.max_pool2d(e2, 2), L[6], "relu"), L[7], "relu")
    up = lambda z: Fn.interpolate(z, scale_factor=2, mode="nearest")
    d2 = conv(conv(torch.cat([up(e3), e2], 1), L[8], "relu"), L[9], "relu")
    d1 = conv(conv(torch.cat([up(d2), e1], 1), L[10], "relu"), L[11], "relu")
    d0 = conv(conv(torch.cat([up(d1), e0], 1), L[12], "relu"), L[13], "relu")
    ref = conv(d0, L[14], "sigmoid")[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(got, ref, atol=1e-12)


# ---------------------------------------------------------------------------
# gradients vs central finite differences
# ---------------------------------------------------------------------------

def _loss_setup(seed=0):
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 48, 48, az_deg=70)
    pose = sg.random_pose(seed + 21)
    G, A, _ = oracle.pose_transforms(sc, pose)
    rng = np.random.default_rng(seed)
    tgtF = rng.standard_normal((cam.H, cam.W, oc.C)) * 0.1
    tgtA = rng.uniform(0, 1, (cam.H, cam.W))
    return sc, oc, cam, pose, G, A, tgtF, tgtA


def _loss(oc, A, cam, tgtF, tgtA, features=None, density=None):
    r = oracle.render(oc, A, cam, features=features, density=density)
    return 0.5 * np.sum((r["F"] - tgtF) ** 2) + 0.5 * np.sum((r["A"] - tgtA) ** 2), r


def test_backward_matches_finite_differences():
    sc, oc, cam, pose, G, A, tgtF, tgtA = _loss_setup()
    L0, r = _loss(oc, A, cam, tgtF, tgtA)
    gF, gA = r["F"] - tgtF, r["A"] - tgtA
    gfeat, gsig, gAinv = oracle.render_backward(oc, A, cam, gF, gA)
    _, gw = oracle.lbs_backward(oc, G, A, gAinv)
    hitv = np.nonzero(np.abs(gsig) > 0)[0]
    assert len(hitv) > 50
    rng = np.random.default_rng(5)
    h = 1e-3
    feats = oc.features.astype(np.float64)
    dens = oc.density.astype(np.float64)
    # features: F is linear in f, so the central difference is exact
    for i in rng.choice(hitv, 20, replace=False):
        c = int(rng.integers(oc.C))
        fp, fm = feats.copy(), feats.copy()
        fp[i, c] += h
        fm[i, c] -= h
        fd = (_loss(oc, A, cam, tgtF, tgtA, features=fp)[0] - _loss(oc, A, cam, tgtF, tgtA, features=fm)[0]) / (2 * h)
        np.testing.assert_allclose(gfeat[i, c], fd, rtol=1e-6, atol=1e-10)
    # densities
    for i in rng.choice(hitv, 20, replace=False):
        dp, dm = dens.copy(), dens.copy()
        dp[i] += h
        dm[i] -= h
        fd = (_loss(oc, A, cam, tgtF, tgtA, density=dp)[0] - _loss(oc, A, cam, tgtF, tgtA, density=dm)[0]) / (2 * h)
        np.testing.assert_allclose(gsig[i], fd, rtol=1e-5, atol=1e-9)
    # skinning weights (geometry): skip samples whose hit set changes under +-h
    checked = 0
    w = oc.weights.astype(np.float64)
    base_hits = oracle.render(oc, A, cam, hits=True)
    for i in rng.choice(hitv, 60, replace=False):
        k = int(rng.integers(4))
        wp, wm = w.copy(), w.copy()
        hw = 1e-5
        wp[i, k] += hw
        wm[i, k] -= hw
        Ap, _ = oracle.lbs(oc, G, wp)
        Am, _ = oracle.lbs(oc, G, wm)
        rp = oracle.render(oc, Ap, cam, hits=True)
        rm = oracle.render(oc, Am, cam, hits=True)
        same = (np.array_equal(rp["hit_id"], base_hits["hit_id"]) and np.array_equal(rm["hit_id"], base_hits["hit_id"])
                and np.array_equal(rp["hit_off"], base_hits["hit_off"]) and np.array_equal(rm["hit_off"], base_hits["hit_off"]))
        if not same:
            continue
        Lp = 0.5 * np.sum((rp["F"] - tgtF) ** 2) + 0.5 * np.sum((rp["A"] - tgtA) ** 2)
        Lm = 0.5 * np.sum((rm["F"] - tgtF) ** 2) + 0.5 * np.sum((rm["A"] - tgtA) ** 2)
        fd = (Lp - Lm) / (2 * hw)
        np.testing.assert_allclose(gw[i, k], fd, rtol=2e-4, atol=1e-7)
        checked += 1
    assert checked >= 20


def test_lbs_backward_matrix_inverse_gradient():
    # dL/dA from dL/dAinv against finite differences of the affine inverse.
    rng = np.random.default_rng(0)
    oc = make_octree([[1, 2, 3]], C=1, jidx=[[0, 1, 0, 0]], w=[[0.6, 0.4, 0.0, 0.0]])
    G = np.stack([np.hstack([oracle.rodrigues(rng.standard_normal(3) * 0.5), rng.standard_normal((3, 1)) * 0.1])
                  for _ in range(2)])
    A, _ = oracle.lbs(oc, G)
    gAinv = rng.standard_normal((1, 3, 4))

    def inv_aff(M):
        M4 = np.vstack([M, [0, 0, 0, 1]])
        return np.linalg.inv(M4)[:3]

    gA, gw = oracle.lbs_backward(oc, G, A, gAinv)
    h = 1e-6
    for r_ in range(3):
        for c_ in range(4):
            Ap, Am = A[0].copy(), A[0].copy()
            Ap[r_, c_] += h
            Am[r_, c_] -= h
            fd = (np.sum(gAinv[0] * inv_aff(Ap)) - np.sum(gAinv[0] * inv_aff(Am))) / (2 * h)
            np.testing.assert_allclose(gA[0, r_, c_], fd, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(gw[0, 0], np.sum(gA[0] * G[0]), rtol=1e-12)
    np.testing.assert_allclose(gw[0, 1], np.sum(gA[0] * G[1]), rtol=1e-12)


def test_wrapper_keeps_converted_inputs_alive():
    # float32 inputs are converted before the C call; the converted arrays must
    # stay alive during it (results equal those for the same values in FP64)
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 48, 48, az_deg=40.0)
    G, A, _ = oracle.pose_transforms(sc, sg.random_pose(2))
    rng = np.random.default_rng(0)
    g32 = rng.standard_normal((48, 48, oc.C)).astype(np.float32)
    a32 = rng.standard_normal((48, 48)).astype(np.float32)
    r1 = oracle.render_backward(oc, A, cam, g32, a32)
    r2 = oracle.render_backward(oc, A, cam, g32.astype(np.float64), a32.astype(np.float64))
    for x, y in zip(r1, r2):
        np.testing.assert_array_equal(x, y)
    gN = r1[2].astype(np.float32)
    np.testing.assert_array_equal(oracle.lbs_backward(oc, G, A.astype(np.float32), gN)[1],
                                  oracle.lbs_backward(oc, G, A.astype(np.float32).astype(np.float64),
                                                      gN.astype(np.float64))[1])
    np.testing.assert_array_equal(oracle.rodrigues(np.float32([0.1, 0.2, 0.3])),
                                  oracle.rodrigues(np.float32([0.1, 0.2, 0.3]).astype(np.float64)))


# ---------------------------------------------------------------------------
# learned ray-interval proposal (project addition; the paper's nearest
# passage is the early-stop rule of Sec. 3.1)
# ---------------------------------------------------------------------------

def _proposal_scene(seed=3):
    sc = sg.preset("tiny")
    cam = sg.orbit_camera(sc.centroid, 96, 64, az_deg=30.0, fov_deg=6.0)  # the animal fills the view
    G, A, _ = oracle.pose_transforms(sc, sg.random_pose(seed))
    return sc, cam, A


def test_proposal_inputs_closed_form():
    """Pixel (0, 0) of a 2 x 4 image: u = 1/4, v = 1/8; the Fourier features
    take the values of sin / cos at multiples of pi/4 and pi/8."""
    cam = sg.orbit_camera(np.zeros(3), 2, 4)
    aa = np.arange(72, dtype=np.float64).reshape(24, 3) * 0.01
    x = oracle.proposal_inputs(aa, cam)
    assert x.shape == (8, 107)
    np.testing.assert_array_equal(x[:, :72], np.broadcast_to(aa.reshape(-1), (8, 72)))
    _, d = oracle.pixel_ray(cam, 1, 2)
    np.testing.assert_allclose(x[2 * 2 + 1, 72:75], d, atol=1e-15)
    r = math.sqrt(0.5)
    sin_u = [r, 1, 0, 0, 0, 0, 0, 0]
    cos_u = [r, 0, -1, 1, 1, 1, 1, 1]
    s8, c8 = math.sin(math.pi / 8), math.cos(math.pi / 8)
    sin_v = [s8, r, 1, 0, 0, 0, 0, 0]
    cos_v = [c8, r, 0, -1, 1, 1, 1, 1]
    np.testing.assert_allclose(x[0, 75:107], sin_u + cos_u + sin_v + cos_v, atol=1e-12)


def test_proposal_mlp_selector_network():
    """Weights that route input 106 - i to hidden unit i (a transposed or
    shifted weight layout picks other inputs), identity hidden layers, and an
    output layer giving +h and 2h + bias on the two halves."""
    layers = []
    W0 = np.zeros((64, 107))
    W0[np.arange(64), 106 - np.arange(64)] = 1.0
    b0 = np.zeros(64)
    layers += [W0, b0]
    for _ in range(3):
        layers += [np.eye(64), np.zeros(64)]
    W4 = np.concatenate([np.eye(64), 2 * np.eye(64)])
    b4 = np.concatenate([np.zeros(64), np.arange(64) * 0.5])
    layers += [W4, b4]
    params = np.concatenate([a.reshape(-1) for a in layers])
    assert params.size == oracle.PROPOSAL_PARAMS
    rng = np.random.default_rng(0)
    x = rng.uniform(0.1, 1.0, (5, 107))
    lg = oracle.proposal_mlp(x, params)
    h = x[:, 106 - np.arange(64)]
    np.testing.assert_allclose(lg[:, :64], h, atol=1e-15)
    np.testing.assert_allclose(lg[:, 64:], 2 * h + np.arange(64) * 0.5, atol=1e-15)
    # ReLU clips negative routed inputs
    lg2 = oracle.proposal_mlp(-x, params)
    np.testing.assert_allclose(lg2[:, :64], 0.0)


def test_proposal_bins_first_argmax_and_interval():
    lg = np.zeros((3, 128))
    lg[0, [5, 9]] = 1.0         # tie: first index
    lg[0, 64 + 20] = 3.0
    lg[1, 63] = 1.0
    lg[1, 64 + 0] = 1.0         # bf < bn: empty
    b = oracle.proposal_bins(lg)
    np.testing.assert_array_equal(b, [[5, 20], [63, 0], [0, 0]])


def test_round_bf16_ties_to_even_and_matches_torch():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert oracle.round_bf16(one + 2.0 ** -8) == 1.0                      # tie -> even (1.0)
    assert oracle.round_bf16(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even (odd neighbour up)
    assert oracle.round_bf16(one + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(1).standard_normal(10000) * 10.0 ** np.random.default_rng(2).integers(-6, 6, 10000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), ref)


def test_render_interval_whole_range_is_plain_render():
    sc, cam, A = _proposal_scene()
    f = oracle.render(sc.octree, A, cam)
    for bins in (None, np.tile([0, oracle.PROPOSAL_BINS - 1], (cam.H * cam.W, 1))):
        r = oracle.render_interval(sc.octree, A, cam, bins)
        np.testing.assert_array_equal(r["F"], f["F"])
        np.testing.assert_array_equal(r["A"], f["A"])
        assert r["missed"].max() == 0.0


def test_render_interval_empty_loses_all_mass():
    """An empty interval composites nothing and loses 1 - exp(-sum of
    sigma delta over all of the ray's hits) (brute force over the hit lists)."""
    sc, cam, A = _proposal_scene()
    full = oracle.render(sc.octree, A, cam, hits=True, tau=0.0)
    bins = np.tile([1, 0], (cam.H * cam.W, 1))
    r = oracle.render_interval(sc.octree, A, cam, bins)
    assert np.abs(r["F"]).max() == 0.0 and np.abs(r["A"]).max() == 0.0
    sig = sc.octree.density.astype(np.float64)
    off = full["hit_off"]
    tau_all = np.array([np.sum(sig[full["hit_id"][off[p]:off[p + 1]]] *
                               (full["hit_t1"][off[p]:off[p + 1]] - full["hit_t0"][off[p]:off[p + 1]]))
                        for p in range(cam.H * cam.W)])
    np.testing.assert_allclose(r["missed"].reshape(-1), 1.0 - np.exp(-tau_all), atol=1e-14)
    assert tau_all.max() > 0.05


def test_render_interval_error_within_missed_mass():
    """For random intervals the restricted feature map differs from the full
    one by at most (2 m_P + T_end m_Q) max|f| <= 2 missed max|f| (plus the
    early-stop slack tau), the bound the coarse check relies on; and the tile
    histogram bound dominates the exact lost mass."""
    sc, cam, A = _proposal_scene()
    rng = np.random.default_rng(5)
    bn = rng.integers(0, 64, cam.H * cam.W)
    bf = np.minimum(63, bn + rng.integers(-1, 6, cam.H * cam.W))
    bins = np.stack([bn, bf], 1)
    f = oracle.render(sc.octree, A, cam)
    r = oracle.render_interval(sc.octree, A, cam, bins)
    fmax = np.abs(sc.octree.features).max()
    err = np.abs(r["F"] - f["F"]).max(-1)
    assert np.all(err <= (2 * r["missed"] + 2 * oracle.TAU_DEFAULT) * fmax + 1e-12)
    assert (r["missed"] > 1e-3).mean() > 0.005  # the draw does skip mass somewhere
    hist = oracle.tau_hist(sc.octree, A, cam)
    bound = oracle.coarse_bound(hist, bins, 1.0 - r["A"], cam)
    assert np.all(bound >= r["missed"] - 1e-12)


def test_tau_hist_brute_force():
    """Each voxel adds sigma (dmax - dmin) to the bins its distance range
    overlaps, in every tile whose pixel centres its box covers."""
    sc, cam, A = _proposal_scene()
    hist = oracle.tau_hist(sc.octree, A, cam, 8, 4)
    vb = oracle.voxel_bounds(sc.octree, A, cam)
    tile, vid = oracle.tile_pairs(sc.octree, A, cam, 8, 4)
    D = (cam.far - cam.near) / 64
    ref = np.zeros_like(hist)
    for t, i in zip(tile, vid):
        b0 = int(np.clip(np.floor((vb[i, 5] - cam.near) / D), 0, 63))
        b1 = int(np.clip(np.floor((vb[i, 6] - cam.near) / D), 0, 63))
        ref[t, b0:b1 + 1] += sc.octree.density[i] * (vb[i, 6] - vb[i, 5])
    np.testing.assert_allclose(hist, ref, rtol=1e-12, atol=1e-15)


def test_labels_brute_force_and_label_bins_pass_check():
    """Labels (min t1, max t0 over hits with weight > 1e-6, transmittance
    after the last) recomputed from the ordered hit lists; the label bins
    keep every significant hit, pass the coarse check in every tile, and the
    learned-skip render with them equals the plain render within the
    lost-mass bound."""
    sc, cam, A = _proposal_scene()
    full = oracle.render(sc.octree, A, cam, hits=True)
    r = oracle.render_interval(sc.octree, A, cam, None, labels=True)
    lab = r["labels"].reshape(-1, 3)
    sig = sc.octree.density.astype(np.float64)
    off = full["hit_off"]
    for p in range(cam.H * cam.W):
        lo, hi, Ts, opt = np.inf, -np.inf, 1.0, 0.0
        for k in range(off[p], off[p + 1]):
            i, t0, t1 = full["hit_id"][k], full["hit_t0"][k], full["hit_t1"][k]
            w = math.exp(-opt) * (1.0 - math.exp(-sig[i] * (t1 - t0)))
            opt += sig[i] * (t1 - t0)
            if w > oracle.LABEL_WMIN:
                lo, hi, Ts = min(lo, t1), max(hi, t0), math.exp(-opt)
            if math.exp(-opt) < oracle.TAU_DEFAULT:
                break
        np.testing.assert_allclose(lab[p], [lo, hi, Ts], rtol=0, atol=1e-14)
    hist = oracle.tau_hist(sc.octree, A, cam)
    bins = oracle.label_bins(r["labels"], hist, cam)
    D = (cam.far - cam.near) / 64
    has = np.isfinite(lab[:, 0])
    assert has.sum() > 100
    assert np.all(cam.near + bins[has, 0] * D <= lab[has, 0])
    assert np.all(cam.near + (bins[has, 1] + 1) * D > lab[has, 1])
    s = oracle.skip_render(sc.octree, A, cam, bins)
    assert not s["fallback"].any() and s["bound"].max() <= oracle.MISSED_MAX
    fmax = np.abs(sc.octree.features).max()
    assert np.abs(s["F"] - full["F"]).max() <= 2 * oracle.MISSED_MAX * fmax


def test_tile_union_bins_cases():
    """Union of a tile's non-empty intervals, margin and clamping; a tile of
    empty intervals stays empty; pixels take their tile's interval."""
    cam = sg.orbit_camera(np.zeros(3), 16, 4)  # two 8 x 4 tiles
    b = np.zeros((4, 16, 2), np.int32)
    b[..., 0], b[..., 1] = 30, 31          # tile 0: all (30, 31) ...
    b[1, 3] = (27, 29)                      # ... one pixel reaches lower
    b[2, 5] = (40, 10)                      # ... an empty one is ignored
    b[:, 8:] = (5, 4)                       # tile 1: all empty
    u = oracle.tile_union_bins(b, cam).reshape(4, 16, 2)
    assert np.all(u[:, :8] == (27, 31)) and np.all(u[:, 8:, 1] < u[:, 8:, 0])
    u2 = oracle.tile_union_bins(b, cam, margin=30).reshape(4, 16, 2)
    assert np.all(u2[:, :8] == (0, 61))
    b[..., 0], b[..., 1] = 62, 63
    assert np.all(oracle.tile_union_bins(b, cam, margin=2).reshape(4, 16, 2) == (60, 63))


# ---------------------------------------------------------------------------
# Sec. 3.1 "Hybrid Rendering": the depth buffer
# ---------------------------------------------------------------------------

def test_depth_single_voxel_front_face():
    # The centre ray of an axis-aligned cube, seen from distance D along an
    # axis, enters it at D - h/2; along a diagonal through the centre the
    # entry is at D - h / (2 max_a |d_a|).
    oc = make_octree([[7, 8, 9]], dens=[5.0], C=2)
    c = voxel_center(oc, 0)
    for direction in [(0, 0, 1), (1, 0, 0), (1, 1, 1), (0.3, -0.5, 1.0)]:
        d = np.asarray(direction, float) / np.linalg.norm(direction)
        cam = axis_camera(c, direction, dist=1.2)
        r = oracle.depth(oc, identity_A(1), cam, 1.0)
        half = 0.5 * oc.h / np.max(np.abs(d))
        np.testing.assert_allclose(r["depth"][0, 0], 1.2 - half, rtol=1e-12)
        np.testing.assert_allclose(r["chord"][0, 0], 2 * half, rtol=1e-12)
    # denser threshold than the voxel: no depth
    assert np.isinf(oracle.depth(oc, identity_A(1), cam, 5.0)["depth"][0, 0])


def test_depth_skips_thin_voxels_and_ignores_the_stop():
    # Three voxels stacked along the ray, densities 1, 50, 9: with threshold 2
    # the depth is the second voxel's front face even where an opaque first
    # voxel would have stopped the composite (tau = 1: stop after the first hit).
    oc = make_octree([[5, 5, 5], [5, 5, 6], [5, 5, 7]], dens=[1.0, 50.0, 9.0], C=1)
    c0 = voxel_center(oc, 0)
    cam = axis_camera(c0, (0, 0, 1), dist=1.0)
    r = oracle.depth(oc, identity_A(3), cam, 2.0)
    np.testing.assert_allclose(r["depth"][0, 0], 1.0 + 0.5 * oc.h, rtol=1e-12)
    assert oracle.render(oc, identity_A(3), cam, tau=1.0)["nused"][0, 0] == 1
    np.testing.assert_allclose(oracle.depth(oc, identity_A(3), cam, 0.5)["depth"][0, 0], 1.0 - 0.5 * oc.h,
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.depth(oc, identity_A(3), cam, 20.0)["depth"][0, 0], 1.0 + 0.5 * oc.h,
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.depth(oc, identity_A(3), cam, 50.0)["depth"][0, 0], np.inf)
    # the near plane clips the entry: the depth is where the ray enters [near, far]
    cam = axis_camera(c0, (0, 0, 1), dist=1.0, near=1.0)
    np.testing.assert_allclose(oracle.depth(oc, identity_A(3), cam, 0.5)["depth"][0, 0], 1.0, rtol=1e-12)


def test_depth_is_first_dense_hit_of_the_brute_force_lists():
    # Brute force: the first entry of each pixel's full hit list (every voxel
    # tested) whose density exceeds the threshold; raising the threshold never
    # brings the depth closer.
    sc = sg.preset("mini")
    cam = sg.orbit_camera(sc.centroid, 24, 16, az_deg=30.0, fov_deg=8.0)
    pose = sg.random_pose(4)
    _, A, _ = oracle.pose_transforms(sc, pose)
    dens = sc.octree.density.astype(np.float64)
    thr = float(np.median(dens))
    r = oracle.depth(sc.octree, A, cam, thr)
    n_some = 0
    for y in range(cam.H):
        for x in range(cam.W):
            b = oracle.pixel_brute(sc.octree, A, cam, x, y, tau=0.0)
            want = np.inf
            for i, t0 in zip(b["ids"], b["t0"]):
                if dens[i] > thr:
                    want = t0
                    break
            n_some += np.isfinite(want)
            np.testing.assert_allclose(r["depth"][y, x], want, rtol=1e-12)
    assert n_some > 20
    r2 = oracle.depth(sc.octree, A, cam, 2 * thr)
    assert np.all(r2["depth"] >= r["depth"])
    assert np.all(r["depth"][np.isfinite(r["depth"])] >= cam.near)


# ---------------------------------------------------------------------------
# Eq. 2: view-dependent features (spherical harmonics)
# ---------------------------------------------------------------------------

def _real_sh_scipy(L, d):
    """Real orthonormal SH from scipy's complex ones (which carry the
    Condon-Shortley phase): sqrt(2) (-1)^m Re / Im of Y_l^|m|."""
    sp = pytest.importorskip("scipy.special")
    th = np.arccos(np.clip(d[:, 2], -1, 1))
    ph = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi)
    out = np.zeros((d.shape[0], (L + 1) ** 2))
    for l in range(L + 1):
        for m in range(-l, l + 1):
            y = sp.sph_harm_y(l, abs(m), th, ph)
            if m < 0:
                v = math.sqrt(2) * (-1) ** m * y.imag
            elif m == 0:
                v = y.real
            else:
                v = math.sqrt(2) * (-1) ** m * y.real
            out[:, l * l + l + m] = v
    return out


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = np.concatenate([d, [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0]]])
    for L in (0, 1, 3, 6, 9):
        np.testing.assert_allclose(oracle.sh_basis(L, d), _real_sh_scipy(L, d), atol=1e-11)
    # degree 1 in closed form: sqrt(3 / 4pi) (y, z, x)
    c1 = math.sqrt(3.0 / (4 * math.pi))
    np.testing.assert_allclose(oracle.sh_basis(1, d)[:, 1:], c1 * d[:, [1, 2, 0]], atol=1e-14)
    with pytest.raises(ValueError):
        oracle.sh_basis(10, d[:1])


def test_sh_basis_orthonormal_on_the_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of
    # degree <= 7 harmonics exactly: the Gram matrix is the identity.
    L = 7
    x, wx = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(L, d)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye((L + 1) ** 2), atol=1e-12)


def test_polar_rotation_factors():
    rng = np.random.default_rng(3)
    for k in range(5):
        Q = oracle.rodrigues(rng.standard_normal(3))
        M = rng.standard_normal((3, 3))
        S = M @ M.T + 0.5 * np.eye(3)  # symmetric positive definite
        for lin in (Q, 2.5 * Q, Q @ S):
            A = np.concatenate([lin, rng.standard_normal((3, 1))], 1)
            np.testing.assert_allclose(oracle.polar_rotation(A)[0], Q, atol=1e-12)
    # a blend of two rotations: orthonormal, det +1, and R^T A_lin symmetric positive definite
    R1, R2 = oracle.rodrigues([0.3, -0.2, 0.5]), oracle.rodrigues([-0.4, 0.1, 0.2])
    lin = 0.7 * R1 + 0.3 * R2
    R = oracle.polar_rotation(np.concatenate([lin, np.zeros((3, 1))], 1))[0]
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    assert abs(np.linalg.det(R) - 1) < 1e-13
    P = R.T @ lin
    np.testing.assert_allclose(P, P.T, atol=1e-13)
    assert np.all(np.linalg.eigvalsh(0.5 * (P + P.T)) > 0)


def test_render_sh_degree_zero_is_the_plain_render():
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 32, 24, az_deg=70.0, fov_deg=10.0)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(2))
    rng = np.random.default_rng(1)
    k0 = rng.standard_normal((oc.n, 1, 5))
    r = oracle.render_sh(oc, A, cam, 0, k0)
    y00 = 0.5 / math.sqrt(math.pi)
    p = oracle.render(oc, A, cam, features=k0[:, 0, :] * y00)
    assert (p["A"] > 0).sum() > 50
    np.testing.assert_allclose(r["A"], p["A"], atol=1e-14)
    np.testing.assert_allclose(r["F"], p["F"], atol=1e-13)


def test_render_sh_single_voxel_closed_form():
    # One voxel under a rigid transform [Q | t], seen along direction d through
    # its centre: S = sum_h k_h Y_h(Q^T d), weighted by its alpha.
    oc = make_octree([[6, 7, 8]], dens=[4.0], C=2)
    Q = oracle.rodrigues([0.3, 0.9, -0.4])
    t = np.array([0.02, -0.05, 0.04])
    A = np.zeros((1, 3, 4))
    A[0, :, :3], A[0, :, 3] = Q, t
    cw = Q @ voxel_center(oc, 0) + t
    L = 3
    k = np.random.default_rng(5).standard_normal((1, (L + 1) ** 2, 2))
    for direction in [(0, 0, 1), (0.4, -0.3, 1.0), (-1, 0.2, 0.1)]:
        d = np.asarray(direction, float) / np.linalg.norm(direction)
        cam = axis_camera(cw, direction, dist=1.1)
        r = oracle.render_sh(oc, A, cam, L, k)
        dl = Q.T @ d
        chord = oc.h / np.max(np.abs(dl))
        a = 1 - math.exp(-4.0 * chord)
        S = _real_sh_scipy(L, dl[None, :])[0] @ k[0]
        np.testing.assert_allclose(r["F"][0, 0], a * S, rtol=1e-10, atol=1e-13)


def test_render_sh_rigid_joint_equals_moved_camera():
    # All voxels bound to one joint (a rigid G_j): the canonical ray direction
    # R_j^T d is the direction seen by the camera world_to_cam * G_j looking at
    # the unposed animal, so the two renders agree.
    sc = sg.preset("mini")
    oc = sc.octree
    w = np.zeros_like(oc.weights)
    w[:, 0] = 1.0
    jidx = np.full_like(oc.joint_idx, 4)
    oc1 = sg.Octree(oc.depth, oc.origin, oc.extent, oc.ijk, jidx, w, oc.features, oc.density, oc.sdf)
    sc1 = sg.Scene(oc1, sc.skeleton, sc.centroid, sc.scale, sc.bones, sc.capsules)
    G, A, _ = oracle.pose_transforms(sc1, sg.random_pose(7))
    cam = _cam64(sg.orbit_camera(sc.centroid, 40, 30, az_deg=-25, fov_deg=10.0))
    L = 4
    k = np.random.default_rng(8).standard_normal((oc.n, (L + 1) ** 2, 3))
    r1 = oracle.render_sh(oc1, A, cam, L, k)
    M, Gj = cam.world_to_cam, G[4]
    M2 = np.concatenate([M[:, :3] @ Gj[:, :3], (M[:, :3] @ Gj[:, 3] + M[:, 3])[:, None]], 1)
    cam2 = sg.Camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, M2, cam.near, cam.far)
    r2 = oracle.render_sh(oc1, identity_A(oc.n), cam2, L, k)
    assert (r1["A"] > 0).sum() > 50
    np.testing.assert_allclose(r1["A"], r2["A"], atol=1e-10)
    np.testing.assert_allclose(r1["F"], r2["F"], atol=1e-9)


# ---------------------------------------------------------------------------
# remaining entry points: the tiny network, the whole frame, ray directions,
# sampled pixels
# ---------------------------------------------------------------------------

def test_tiny_net_matches_torch_and_shade_dispatches():
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    layers = sg.tiny_net_weights(4, cin=5, mid=7, cout=4)
    x = np.random.default_rng(2).standard_normal((11, 13, 5))
    t = torch.from_numpy(x).permute(2, 0, 1)[None]
    for k, (w, b) in enumerate(layers):
        t = Fn.conv2d(t, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                      torch.from_numpy(b.astype(np.float64)), padding=1)
        t = torch.sigmoid(t) if k == 2 else torch.relu(t)
    ref = t[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(oracle.shade_tiny(x, layers), ref, atol=1e-12)
    np.testing.assert_array_equal(oracle.shade(x, layers), oracle.shade_tiny(x, layers))
    ul = sg.unet_weights(3, cin=5, ch=(4, 6, 8, 10))
    xu = np.random.default_rng(3).standard_normal((16, 24, 5))
    np.testing.assert_array_equal(oracle.shade(xu, ul), oracle.shade_unet(xu, ul))


def test_render_frame_is_pose_render_and_shade():
    sc = sg.preset("mini")
    cam = sg.orbit_camera(sc.centroid, 24, 16, az_deg=10.0, fov_deg=10.0)
    pose = sg.random_pose(6)
    layers = sg.tiny_net_weights(1, cin=sc.octree.C, mid=6)
    out = oracle.render_frame(sc, pose, cam, layers)
    G, A, det = oracle.pose_transforms(sc, pose)
    r = oracle.render(sc.octree, A, cam)
    np.testing.assert_array_equal(out["F"], r["F"])
    np.testing.assert_array_equal(out["A"], r["A"])
    np.testing.assert_array_equal(out["rgba"], oracle.shade(r["F"], layers))
    np.testing.assert_array_equal(out["G"], G)


def test_ray_dirs_equal_pixel_rays():
    cam = sg.orbit_camera(np.array([0.1, 0.2, -0.3]), 7, 5, az_deg=33.0, elev_deg=-20.0)
    D = oracle.ray_dirs(cam)
    for y in range(cam.H):
        for x in range(cam.W):
            _, d = oracle.pixel_ray(cam, x, y)
            np.testing.assert_allclose(D[y, x], d, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(D, axis=2), 1.0, atol=1e-14)


def test_sampled_pixels_equal_the_full_render():
    # pixels() tests every voxel for each sampled pixel; render() only the
    # candidates of the projected boxes: the same F and A wherever sampled.
    sc = sg.preset("mini")
    cam = sg.orbit_camera(sc.centroid, 32, 24, az_deg=140.0, fov_deg=10.0)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(9))
    full = oracle.render(sc.octree, A, cam)
    rng = np.random.default_rng(4)
    px, py = rng.integers(0, cam.W, 60), rng.integers(0, cam.H, 60)
    cov = np.argwhere(full["A"] > 0)
    px = np.concatenate([px, cov[:40, 1]])
    py = np.concatenate([py, cov[:40, 0]])
    o = oracle.pixels(sc.octree, A, cam, px, py)
    np.testing.assert_allclose(o["F"], full["F"][py, px], atol=1e-14)
    np.testing.assert_allclose(o["A"], full["A"][py, px], atol=1e-14)
    assert np.all(o["nhit"] == full["nhit"][py, px])


def test_render_sh_is_linear_and_its_coefficient_gradient():
    # F is linear in the coefficients: F(a k1 + b k2) = a F(k1) + b F(k2), and
    # the gradient of <gF, F> is exact under a central difference; at degree
    # 0 it is Y_00 times the plain render's feature gradient.
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 16, 12, az_deg=40.0, fov_deg=8.0)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(5))
    rng = np.random.default_rng(11)
    L, C = 2, 3
    k1 = rng.standard_normal((oc.n, 9, C))
    k2 = rng.standard_normal((oc.n, 9, C))
    F1 = oracle.render_sh(oc, A, cam, L, k1)["F"]
    F2 = oracle.render_sh(oc, A, cam, L, k2)["F"]
    F12 = oracle.render_sh(oc, A, cam, L, 0.7 * k1 - 1.3 * k2)["F"]
    np.testing.assert_allclose(F12, 0.7 * F1 - 1.3 * F2, atol=1e-13)
    gF = rng.standard_normal((cam.H, cam.W, C))
    g = oracle.render_sh_backward(oc, A, cam, L, gF)
    hit = np.argwhere(np.abs(g).sum((1, 2)) > 0)[:, 0]
    assert len(hit) > 20
    eps = 1e-3
    for i in hit[:: max(1, len(hit) // 6)][:6]:
        for h, c in [(0, 0), (4, 1), (8, 2)]:
            kp, km = k1.copy(), k1.copy()
            kp[i, h, c] += eps
            km[i, h, c] -= eps
            fd = (np.sum(gF * oracle.render_sh(oc, A, cam, L, kp)["F"]) -
                  np.sum(gF * oracle.render_sh(oc, A, cam, L, km)["F"])) / (2 * eps)
            np.testing.assert_allclose(g[i, h, c], fd, rtol=1e-7, atol=1e-10)
    g0 = oracle.render_sh_backward(oc, A, cam, 0, gF)
    gfeat, _, _ = oracle.render_backward(oc, A, cam, gF, np.zeros((cam.H, cam.W)), features=np.zeros((oc.n, C)))
    np.testing.assert_allclose(g0[:, 0, :], gfeat * (0.5 / math.sqrt(math.pi)), atol=1e-13)


# ---------------------------------------------------------------------------
# The paper's per-frame index: warped centres snapped to the leaf lattice
# ---------------------------------------------------------------------------

def _snap_brute(oc, A):
    """Python loop: lattice cell of each warped centre, survivors by dict."""
    h = oc.extent / (1 << oc.depth)
    org = oc.origin.astype(np.float64)
    A = np.asarray(A, np.float64).reshape(-1, 3, 4)
    cells, owner = [], {}
    for i in range(oc.n):
        if np.linalg.det(A[i, :, :3]) < 1e-3:
            cells.append(None)
            continue
        pc = org + (oc.ijk[i].astype(np.float64) + 0.5) * h
        p = A[i, :, :3] @ pc + A[i, :, 3]
        c = tuple(int(math.floor(v)) for v in (p - org) / h)
        cells.append(c)
        owner.setdefault(c, i)  # ids ascend: the first is the smallest
    win = np.array([-1 if c is None else owner[c] for c in cells])
    return cells, win, len(owner)


def test_grid_snap_matches_brute_force_under_a_pose():
    sc = sg.preset("mini")
    oc = sc.octree
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(9))
    A = np.asarray(A, np.float64).reshape(-1, 3, 4).copy()
    A[7, :, :3] *= 0.05  # det 1.25e-4 < 1e-3: not placed
    g = oracle.grid_snap(oc, A)
    cells, win, nc = _snap_brute(oc, A)
    np.testing.assert_array_equal(g["winner"], win)
    assert g["n_cells"] == nc and g["winner"][7] == -1
    for i in range(oc.n):
        if cells[i] is not None:
            assert tuple(g["cell"][i]) == cells[i]
    assert nc < int(np.sum(win >= 0))  # the pose makes some voxels collide


def test_grid_at_identity_is_the_voxel_render():
    # with every A_i = I each centre lands in its own leaf: no collision, the
    # cells are the canonical cubes and the two renders are the same numbers
    sc = sg.preset("tiny")
    oc = sc.octree
    A = identity_A(oc.n)
    g = oracle.grid_snap(oc, A)
    np.testing.assert_array_equal(g["winner"], np.arange(oc.n))
    np.testing.assert_array_equal(g["cell"], oc.ijk.astype(np.int64))
    cam = sg.orbit_camera(sc.centroid, 64, 48, az_deg=30.0, fov_deg=10.0)
    r = oracle.render(oc, A, cam)
    q = oracle.render_grid(oc, A, cam)
    assert q["n_cells"] == oc.n and np.count_nonzero(r["A"]) > 200
    np.testing.assert_array_equal(q["F"], r["F"])
    np.testing.assert_array_equal(q["A"], r["A"])
    np.testing.assert_array_equal(q["nhit"], r["nhit"])
    assert oracle.vrt_loss(oc, A) == 0.0


def test_grid_render_is_the_voxel_render_of_the_survivors_moved_to_their_cells():
    # under any pose: the survivors, each translated from its canonical cube
    # onto its cell, rendered by the exact voxel path
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 40, 32, az_deg=75.0, fov_deg=8.0)
    _, A, _ = oracle.pose_transforms(sc, sg.random_pose(4))
    g = oracle.grid_snap(oc, A)
    keep = np.flatnonzero(g["winner"] == np.arange(oc.n))
    h = oc.extent / (1 << oc.depth)
    At = identity_A(keep.size)
    At[:, :, 3] = (g["cell"][keep] - oc.ijk[keep].astype(np.int64)) * h
    r = oracle.render(oc.subset(keep), At, cam)
    q = oracle.render_grid(oc, A, cam)
    assert q["n_cells"] == keep.size and np.count_nonzero(q["A"]) > 100
    np.testing.assert_allclose(q["F"], r["F"], atol=1e-10)
    np.testing.assert_allclose(q["A"], r["A"], atol=1e-10)
    np.testing.assert_array_equal(q["nhit"], r["nhit"])


def test_grid_collision_keeps_the_smallest_id():
    # voxel 3 is moved onto voxel 1's leaf: both centres share one cell, voxel
    # 1 survives, the picture is the scene without voxel 3, and the
    # regularisation term is |f_1 - f_3|_1 over the placed voxels
    ijk = [(4, 4, 4), (6, 4, 4), (8, 4, 4), (10, 8, 4)]
    oc = make_octree(ijk, depth=4, extent=1.0, C=3, seed=5)
    h = 1.0 / 16
    A = identity_A(4)
    A[3, :, 3] = (np.array([6, 4, 4]) - np.array([10, 8, 4])) * h + 0.3 * h  # inside the same leaf
    g = oracle.grid_snap(oc, A)
    np.testing.assert_array_equal(g["winner"], [0, 1, 2, 1])
    assert g["n_cells"] == 3
    f = oc.features.astype(np.float64)
    assert math.isclose(oracle.vrt_loss(oc, A, lam=2.0), 2.0 * np.abs(f[1] - f[3]).sum() / 4, rel_tol=1e-14)
    cam = axis_camera(oc.centers()[1], (0.2, 0.1, 1.0), dist=1.0, W=9, H=9, f=60.0, near=0.05, far=3.0)
    keep = np.array([0, 1, 2])
    r = oracle.render(oc.subset(keep), identity_A(3), cam)
    q = oracle.render_grid(oc, A, cam)
    assert np.count_nonzero(q["A"]) > 0
    np.testing.assert_array_equal(q["F"], r["F"])
    np.testing.assert_array_equal(q["A"], r["A"])


# ---------------------------------------------------------------------------
# The two-branch shading network (Sec. 3.1 "Neural Shading", Fig. 4)
# ---------------------------------------------------------------------------

def _torch_unet(torch, t, layers, levels):
    """The U-Net written recursively with torch's FP64 ops."""
    import torch.nn.functional as Fn
    L = iter(layers)

    def conv(z, act):
        w, b = next(L)
        y = Fn.conv2d(z, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                      torch.from_numpy(b.astype(np.float64)), padding=w.shape[1] // 2)
        return torch.relu(y) if act else torch.sigmoid(y)

    def level(z, l):
        e = conv(conv(z, True), True)
        if l == levels - 1:
            return e
        below = level(Fn.max_pool2d(e, 2), l + 1)
        up = Fn.interpolate(below, scale_factor=2, mode="nearest")
        return conv(conv(torch.cat([up, e], 1), True), True)

    return conv(level(t, 0), False)


def test_two_branch_net_matches_torch_and_its_structure():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    F = rng.standard_normal((16, 24, 5))
    A = rng.uniform(0, 1, (16, 24))
    rgb, alpha = sg.two_branch_weights(2, cin=5, rgb_ch=(4, 6, 8, 10), alpha_ch=(3, 5))
    assert [w.shape for w, _ in sg.unet_weights(3, cin=5, ch=(4, 6, 8, 10))] == \
        [(co, k, k, ci) for co, ci, k in [(4, 5, 3), (4, 4, 3), (6, 4, 3), (6, 6, 3), (8, 6, 3), (8, 8, 3),
                                          (10, 8, 3), (10, 10, 3), (8, 18, 3), (8, 8, 3), (6, 14, 3),
                                          (6, 6, 3), (4, 10, 3), (4, 4, 3), (4, 4, 1)]]
    got = oracle.shade_two_branch(F, A, rgb, alpha)
    assert got.shape == (16, 24, 4)
    tF = torch.from_numpy(F).permute(2, 0, 1)[None]
    I_f = _torch_unet(torch, tF, rgb, 4)
    a = _torch_unet(torch, torch.cat([torch.from_numpy(A)[None, None], I_f], 1), alpha, 2)
    ref = torch.cat([I_f, a], 1)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(got, ref, atol=1e-12)
    # the appearance branch does not see A; the opacity branch does
    got2 = oracle.shade_two_branch(F, 1.0 - A, rgb, alpha)
    np.testing.assert_array_equal(got2[..., :3], got[..., :3])
    assert np.abs(got2[..., 3] - got[..., 3]).max() > 1e-6
    # an opacity branch with a zero head returns sigmoid of the head's bias
    alpha0 = [(w, b) for w, b in alpha[:-1]] + [(np.zeros_like(alpha[-1][0]), np.array([0.3], np.float32))]
    np.testing.assert_allclose(oracle.shade_two_branch(F, A, rgb, alpha0)[..., 3],
                               1.0 / (1.0 + math.exp(-float(np.float32(0.3)))), atol=1e-15)
