"""The seeded synthetic inputs (stand-ins for the paper's CGI animals) have
the shapes and statistics the workloads state (CPU only)."""
import math

import numpy as np

import scenegen as sg


def test_presets_hit_their_voxel_targets_and_are_deterministic():
    for name, target, depth in [("tiny", 20000, 8), ("diff", 200000, 9)]:
        sc = sg.preset(name)
        oc = sc.octree
        assert oc.depth == depth
        assert abs(oc.n - target) <= 0.05 * target, (name, oc.n)
        assert np.all(oc.ijk < (1 << depth))
        again = sg.make_octree(depth, target, oc.C, sg.PRESETS[name]["band"], 0,
                               fur_shell=sg.PRESETS[name]["fur_shell"])
        np.testing.assert_array_equal(again.octree.ijk, oc.ijk)
        np.testing.assert_array_equal(again.octree.features, oc.features)
        np.testing.assert_array_equal(again.octree.density, oc.density)


def test_voxels_lie_in_the_sdf_band_with_the_stated_densities():
    oc = sg.preset("tiny").octree
    lo, hi = sg.PRESETS["tiny"]["band"]
    h = oc.extent / (1 << oc.depth)
    # each voxel's centre is within half a diagonal of the band
    assert np.all(oc.sdf >= lo - math.sqrt(3) * h) and np.all(oc.sdf <= hi + math.sqrt(3) * h)
    # features N(0, 0.5^2); density softplus(N(0, 1)) * 20 / m (no shell in this preset)
    assert abs(float(oc.features.std()) - 0.5) < 0.01 and abs(float(oc.features.mean())) < 0.01
    assert np.all(oc.density > 0)
    sp = np.log1p(np.exp(np.random.default_rng(0).standard_normal(200000))) * 20.0
    assert abs(float(np.median(oc.density)) - float(np.median(sp))) < 0.5


def test_skinning_weights_are_a_partition_of_unity_over_valid_joints():
    sc = sg.preset("tiny")
    oc = sc.octree
    J = sc.skeleton.parent.shape[0]
    assert J == 24 and sc.skeleton.parent[0] == -1 and np.all(sc.skeleton.parent[1:] < np.arange(1, J))
    assert np.all(oc.joint_idx < J)
    assert np.all(oc.weights >= 0)
    np.testing.assert_allclose(oc.weights.sum(1), 1.0, atol=1e-6)
    # the top weight is the nearest bone's (weights sorted by distance)
    assert np.all(oc.weights[:, 0] >= oc.weights[:, 1] - 1e-7)


def test_walk_cycle_is_periodic_and_within_its_amplitudes():
    p0, p60 = sg.walk_pose(0), sg.walk_pose(60)
    np.testing.assert_array_equal(p0.axis_angle, p60.axis_angle)
    amax = max(float(np.abs(sg.walk_pose(f).axis_angle).max()) for f in range(60))
    assert amax <= math.radians(25.0) + 1e-6
    q = sg.random_pose(3)
    assert np.all(np.linalg.norm(q.axis_angle, axis=1) <= math.radians(30.0) + 1e-6)


def test_orbit_camera_looks_at_its_target():
    t = np.array([0.1, -0.2, 0.3])
    cam = sg.orbit_camera(t, 64, 48, az_deg=70.0, elev_deg=10.0, dist=2.0)
    M = cam.world_to_cam.astype(np.float64)
    np.testing.assert_allclose(M[:, :3] @ M[:, :3].T, np.eye(3), atol=1e-6)
    pc = M[:, :3] @ t + M[:, 3]
    np.testing.assert_allclose(pc[:2], 0.0, atol=1e-6)  # on the optical axis
    np.testing.assert_allclose(pc[2], 2.0, atol=1e-5)   # at the orbit distance, in front
    assert abs(cam.fy - 0.5 * cam.H / math.tan(math.radians(20.0))) < 1e-3  # 40 degree vertical fov
