"""GPU parity of the rendering path (FK, LBS, binning, sort, composite)
against the FP64 oracle, called through the C ABI."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import (compare_hit_lists, render_maps, renderer, set_cam, set_pose, tiny_setup)

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-4  # max-abs on F, A and RGBA for the FP32 form


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fk_and_lbs_match_oracle():
    sc, cam, pose = tiny_setup(pose_seed=3)
    r = renderer(sc)
    set_pose(r, pose)
    G_or, A_or, det = oracle.pose_transforms(sc, pose)
    G = r.debug_buffer(0, np.float32).reshape(-1, 3, 4)
    np.testing.assert_allclose(G, G_or, atol=2e-6)
    geo = r.debug_buffer(2, np.float32).reshape(-1, 4, 4)
    c = sc.octree.centers()
    cw = np.einsum("nab,nb->na", A_or[:, :, :3], c) + A_or[:, :, 3]
    np.testing.assert_allclose(geo[:, 0, :3], cw, atol=2e-6)
    h2 = 0.5 * sc.octree.h
    for a in range(3):
        np.testing.assert_allclose(geo[:, 1 + a, :3], A_or[:, :, a] * h2, atol=1e-7)
    rec = r.debug_buffer(1, np.float32).reshape(-1, 4, 4)
    Binv = rec[:, :3, :3].astype(np.float64)
    prod = np.einsum("nab,nbc->nac", Binv, A_or[:, :, :3]) * sc.octree.h
    np.testing.assert_allclose(prod, np.broadcast_to(np.eye(3), prod.shape), atol=2e-5)
    np.testing.assert_array_equal(rec[:, 3, 0], sc.octree.density)


TS, TSY = 8, 4  # screen tile


def _check_tile_order(r, n, cam):
    """The instance list is exactly the stable sort of the (tile << depth_bits
    | depth quantum, voxel id) pairs emitted in voxel order from the rectangles
    and quanta the projection recorded, and the tile ranges delimit it.
    Returns keys, vals, depth_bits and the tile counts."""
    st = r.sync_status()
    keys = r.debug_buffer(5, np.uint32)
    vals = r.debug_buffer(6, np.uint32)
    assert st["instances"] == len(keys) and st["overflow_inst"] == 0
    rect = r.debug_buffer(3, np.int16).reshape(-1, 4).astype(np.int64)
    q = r.debug_buffer(4, np.uint32).astype(np.uint64)
    tw, th = (cam.W + TS - 1) // TS, (cam.H + TSY - 1) // TSY
    tb = max(1, int(np.ceil(np.log2(tw * th))))
    db = min(32 - tb, 20)
    vis = np.nonzero((rect[:, 0] <= rect[:, 2]) & (rect[:, 1] <= rect[:, 3]))[0]
    tx0, ty0 = rect[vis, 0] // TS, rect[vis, 1] // TSY
    nx, ny = rect[vis, 2] // TS - tx0 + 1, rect[vis, 3] // TSY - ty0 + 1
    per = nx * ny  # instances of each visible voxel, emitted row by row
    idx = np.repeat(np.arange(len(vis)), per)
    k = np.arange(per.sum()) - np.repeat(np.cumsum(per) - per, per)
    t = ((ty0[idx] + k // nx[idx]) * tw + tx0[idx] + k % nx[idx]).astype(np.uint64)
    ek = (t << np.uint64(db)) | q[vis[idx]]
    ev = vis[idx].astype(np.uint64)
    order = np.lexsort((ev, ek))
    np.testing.assert_array_equal(keys, ek[order].astype(np.uint32))
    np.testing.assert_array_equal(vals, ev[order].astype(np.uint32))
    rng_ = r.debug_buffer(7, np.uint32).reshape(-1, 2)[: tw * th]
    tiles = (keys >> db).astype(np.int64)
    counts = np.bincount(tiles, minlength=tw * th)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    np.testing.assert_array_equal(rng_[:, 0], starts)
    np.testing.assert_array_equal(rng_[:, 1], starts + counts)
    return keys, vals, db, counts


@pytest.mark.parametrize("az,pose_seed", [(0.0, 1), (135.0, 2)])
def test_tile_lists_sorted_and_cover_oracle(az, pose_seed):
    sc, cam, pose = tiny_setup(az=az, pose_seed=pose_seed)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    render_maps(r, 0, cam, sc.octree.C)
    # 1. the sort: exactly the stable sort of the emitted (key, voxel) pairs
    keys, vals, db, _ = _check_tile_order(r, sc.octree.n, cam)
    tw, th = (cam.W + TS - 1) // TS, (cam.H + TSY - 1) // TSY
    # 2. the tiles: a superset of the oracle's coverage, extras only at bbox edges
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    ot, ov = oracle.tile_pairs(sc.octree, A_or, cam, TS, TSY)
    gpu_pairs = set(zip((keys >> db).tolist(), vals.tolist()))
    or_pairs = set(zip(ot.tolist(), ov.tolist()))
    assert or_pairs <= gpu_pairs
    vb = oracle.voxel_bounds(sc.octree, A_or, cam)
    for (t, i) in gpu_pairs - or_pairs:
        ok, u0, u1, v0, v1, d0, d1 = vb[i]
        tx, ty = t % tw, t // tw
        xs = np.arange(tx * TS, min(tx * TS + TS, cam.W)) + 0.5
        ys = np.arange(ty * TSY, min(ty * TSY + TSY, cam.H)) + 0.5
        e = 1e-2
        assert ok and np.any((xs >= u0 - e) & (xs <= u1 + e)) and np.any((ys >= v0 - e) & (ys <= v1 + e))


# Views chosen so that the binning takes each of its paths: the ~20k-voxel
# scene at 512^2 (8192 tiles: a tile scan of eight blocks chained by
# look-back; buckets of a few entries, warp sort, and of hundreds, block
# sort with the entries in registers), and the 1M-voxel scene at 1024^2
# seen from the side (buckets of up to ~8.6k entries: staged in global
# memory past 8192).
@pytest.mark.parametrize("preset,res,az,min_bucket", [("tiny", 512, 60.0, 257), ("paper", 1024, 90.0, 8193)])
def test_bucket_sort_regimes(preset, res, az, min_bucket):
    sc = sg.preset(preset)
    cam = sg.orbit_camera(sc.centroid, res, res, az_deg=az)
    pose = sg.walk_pose(5, 60)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    render_maps(r, 0, cam, sc.octree.C)
    _, _, _, counts = _check_tile_order(r, sc.octree.n, cam)
    assert counts.max() >= min_bucket  # the regime this view is meant to reach


@pytest.mark.parametrize("az,pose_seed", [(0.0, 1), (80.0, 4), (215.0, 7)])
def test_hit_lists_and_maps_match_oracle(az, pose_seed):
    sc, cam, pose = tiny_setup(az=az, pose_seed=pose_seed)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    cap = 96
    g = r.debug_hits(0, cap)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(sc.octree, A_or, cam, hits=True)
    assert (o["nhit"] > 0).sum() > 150
    assert np.abs(g["F"] - o["F"]).max() < TOL_F32
    assert np.abs(g["A"] - o["A"]).max() < TOL_F32
    bad = []
    for p in np.nonzero(o["nhit"].ravel() + g["count"].ravel())[0]:
        y, x = divmod(int(p), cam.W)
        s, e = o["hit_off"][p], o["hit_off"][p + 1]
        n = g["count"][y, x]
        assert n <= cap
        msg = compare_hit_lists(o["hit_id"][s:e], o["hit_t0"][s:e], o["hit_t1"][s:e], g["ids"][y, x, :n].astype(np.int64),
                                g["t0"][y, x, :n].astype(np.float64), g["t1"][y, x, :n].astype(np.float64))
        if msg:
            bad.append((x, y, msg))
    assert not bad, bad[:5]
    assert r.sync_status()["overflow_order"] == 0


def test_render_f32_device_and_host_outputs():
    import torch
    sc, cam, pose = tiny_setup(az=30.0, pose_seed=5)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, sc.octree.C)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(sc.octree, A_or, cam)
    assert np.abs(F - o["F"]).max() < TOL_F32 and np.abs(A - o["A"]).max() < TOL_F32
    # host outputs: the library copies back and synchronises
    Fh = np.zeros((cam.H, cam.W, sc.octree.C), np.float32)
    Ah = np.zeros((cam.H, cam.W), np.float32)
    r.render_feature_maps(0, Fh, Ah, "f32")
    np.testing.assert_array_equal(Fh, F)
    np.testing.assert_array_equal(Ah, A)
    # bf16 output of the same render: rounding of F only
    Fb, Ab = render_maps(r, 0, cam, sc.octree.C, "bf16")
    assert np.abs(Fb - F).max() <= np.abs(F).max() * 2 ** -8
    np.testing.assert_array_equal(Ab, A)
    del torch


def _stop_case(dens_scale, tau, tol):
    sc, cam, pose = tiny_setup(az=20.0, pose_seed=6)
    oc = sc.octree
    dens = oc.density * np.float32(dens_scale)
    oc2 = sg.Octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, oc.features, dens, oc.sdf)
    sc2 = sg.Scene(oc2, sc.skeleton, sc.centroid, sc.scale, sc.bones, sc.capsules)
    r = renderer(sc2, tau=tau)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    g = r.debug_hits(0, 96)
    _, A_or, _ = oracle.pose_transforms(sc2, pose)
    o = oracle.render(oc2, A_or, cam, tau=tau, hits=True)
    stopped = o["nused"] < o["nhit"]
    assert stopped.sum() > 20
    # exclude pixels whose transmittance passes within 1e-3 tau of tau
    near = np.zeros((cam.H, cam.W), bool)
    for p in np.nonzero(o["nhit"].ravel())[0]:
        s, e = o["hit_off"][p], o["hit_off"][p + 1]
        T = np.exp(-np.cumsum(dens[o["hit_id"][s:e]].astype(np.float64) * (o["hit_t1"][s:e] - o["hit_t0"][s:e])))
        near.flat[p] = np.any(np.abs(T - tau) < 1e-3 * tau)
    ok = ~near
    assert np.abs(g["F"] - o["F"])[ok].max() < tol
    assert np.abs(g["A"] - o["A"])[ok].max() < tol
    assert np.array_equal(g["count"][ok & stopped], o["nused"][ok & stopped])
    # the split walk (segments of 32 entries): a stop inside a later segment
    # sends the tile to the plain walk, so the stop rule holds exactly
    r.set_config(tau=tau, segment=32)
    F, A = render_maps(r, 0, cam, oc.C)
    st = r.sync_status()
    assert np.abs(F - o["F"])[ok].max() < tol
    assert np.abs(A - o["A"])[ok].max() < tol
    return st


def test_early_stop_matches_oracle():
    # tau = 0.7 fires inside the animal at the workload's densities: FP32 tolerance
    st = _stop_case(1.0, 0.7, TOL_F32)
    assert st["fallback_tiles"] > 0


def test_early_stop_opaque_voxels():
    # sigma x 60 (up to ~3000 / m) with tau = 1e-4: the FP32 ray parameter carries
    # ~2e-7 m of rounding at 2 m, i.e. up to sigma * 2e-7 * 4 ~ 3e-3 of alpha per
    # hit; the bound below is that per-hit figure times max|f|.
    st = _stop_case(60.0, 1e-4, 3e-3 * 2.0)
    assert st["fallback_tiles"] > 0


@pytest.mark.parametrize("segment,az,pose_seed", [(32, 80.0, 4), (96, 215.0, 7)])
def test_split_walk_matches_oracle(segment, az, pose_seed):
    """Tiles walked in segments by separate warps and merged front to back
    (F = F_0 + T_0 F_1 + ...) against the oracle, and against one segment
    per tile (the same sum, grouped differently)."""
    sc, cam, pose = tiny_setup(az=az, pose_seed=pose_seed)
    r = renderer(sc, segment=segment, profile=True)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, sc.octree.C)
    kt = r.kernel_times(reset=True)
    assert kt["composite_merge"][0] == 1 and kt["composite"][0] == 1
    rg = r.debug_buffer(7, np.uint32).reshape(-1, 2)[: ((cam.W + 7) // 8) * ((cam.H + 3) // 4)]
    assert (rg[:, 1] - rg[:, 0]).max() >= 4 * segment  # some tiles split in four or more
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(sc.octree, A_or, cam)
    assert np.abs(F - o["F"]).max() < TOL_F32 and np.abs(A - o["A"]).max() < TOL_F32
    r.set_config(segment=1 << 24)
    F1, A1 = render_maps(r, 0, cam, sc.octree.C)
    assert np.abs(F - F1).max() < 1e-6 and np.abs(A - A1).max() < 1e-6
    assert r.sync_status()["fallback_tiles"] == 0


def test_bf16_and_f16_feature_storage():
    sc, cam, pose = tiny_setup(az=60.0, pose_seed=8)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.render(sc.octree, A_or, cam)
    fmax = np.abs(sc.octree.features).max()
    for storage, rel in (("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)):
        r = renderer(sc, storage=storage)
        set_pose(r, pose)
        set_cam(r, 0, cam)
        F, A = render_maps(r, 0, cam, sc.octree.C)
        # F error <= sum_i w_i |f_i - rn(f_i)| <= A * max|f| * rel (+ FP32 rounding)
        bound = o["A"][..., None] * fmax * rel + TOL_F32
        assert np.all(np.abs(F - o["F"]) <= bound)
        assert np.abs(A - o["A"]).max() < TOL_F32


def test_degenerate_blends_are_dropped_and_counted():
    sc = sg.preset("mini")
    oc = sc.octree
    rng = np.random.default_rng(0)
    pick = rng.uniform(size=oc.n) < 0.1
    w = oc.weights.copy()
    jidx = oc.joint_idx.copy()
    w[pick] = [0.5, 0.5, 0.0, 0.0]
    jidx[pick] = [1, 2, 0, 0]
    oc2 = sg.Octree(oc.depth, oc.origin, oc.extent, oc.ijk, jidx, w, oc.features, oc.density, oc.sdf)
    sc2 = sg.Scene(oc2, sc.skeleton, sc.centroid, sc.scale, sc.bones, sc.capsules)
    aa = np.zeros((24, 3), np.float32)
    aa[2] = [0.0, np.pi, 0.0]  # spine2 turned half a turn relative to spine1
    pose = sg.Pose(aa, np.zeros(3, np.float32), np.zeros(3, np.float32))
    _, A_or, det = oracle.pose_transforms(sc2, pose)
    r = renderer(sc2)
    set_pose(r, pose)
    cam = sg.orbit_camera(sc.centroid, 64, 64)
    set_cam(r, 0, cam)
    g = r.debug_hits(0, 128)
    st = r.sync_status(raise_on_overflow=False)
    assert st["degenerate"] == int((det < 1e-3).sum()) >= int(pick.sum())
    o = oracle.render(oc2, A_or, cam, hits=True)
    assert st["overflow_order"] == 0
    # The half-turn folds voxels onto each other: coincident voxels enter at the
    # same t0 to FP32 precision, and their order (hence F) is then decided by
    # rounding.  Hit sets must agree everywhere; F and A are compared on the
    # pixels without such near-ties.
    tied = np.zeros((cam.H, cam.W), bool)
    for p in np.nonzero(o["nhit"].ravel() + g["count"].ravel())[0]:
        y, x = divmod(int(p), cam.W)
        s, e = o["hit_off"][p], o["hit_off"][p + 1]
        n = g["count"][y, x]
        msg = compare_hit_lists(o["hit_id"][s:e], o["hit_t0"][s:e], o["hit_t1"][s:e],
                                g["ids"][y, x, :n].astype(np.int64), g["t0"][y, x, :n].astype(np.float64),
                                g["t1"][y, x, :n].astype(np.float64))
        assert msg is None, (x, y, msg)
        t0, ch = o["hit_t0"][s:e], o["hit_t1"][s:e] - o["hit_t0"][s:e]
        big = ch >= 1e-5
        tied.flat[p] = bool(np.any(np.diff(np.sort(t0[big])) < 1e-6))
    ok = ~tied
    assert ok.sum() > 0.5 * ok.size and tied.sum() > 0
    assert np.abs(g["F"] - o["F"])[ok].max() < TOL_F32
    assert np.abs(g["A"] - o["A"])[ok].max() < TOL_F32


def test_invalid_arguments_raise():
    import paper_2202_05628_gb300 as art
    sc = sg.preset("mini")
    r = art.Renderer()
    with pytest.raises(art.ArtemisError):
        r.set_pose(np.zeros((24, 3)), np.zeros(3), np.zeros(3))  # before load
    oc = sc.octree
    with pytest.raises(art.ArtemisError):
        r.load_octree(oc.depth, oc.origin, oc.extent, oc.ijk, oc.joint_idx, oc.weights, oc.features[:, :3],
                      oc.density)  # C = 3
    bad_ijk = oc.ijk.copy()
    bad_ijk[0, 0] = 1 << oc.depth
    with pytest.raises(art.ArtemisError):
        r.load_octree(oc.depth, oc.origin, oc.extent, bad_ijk, oc.joint_idx, oc.weights, oc.features, oc.density)
    with pytest.raises(art.ArtemisError):
        r.load_skeleton(np.array([-1, 2, 0]), np.zeros((3, 3)))
    r2 = renderer(sc)
    r2.load_skeleton(sc.skeleton.parent[:4], sc.skeleton.rest[:4])  # J=4 < joint indices
    with pytest.raises(art.ArtemisError):
        set_pose(r2, sg.rest_pose(4))
    with pytest.raises(art.ArtemisError):
        r2.set_camera(0, 64, 64, 100.0, 100.0, 32.0, 32.0, np.eye(3, 4), 2.0, 1.0)  # near > far


def test_instance_overflow_is_reported():
    sc, cam, pose = tiny_setup()
    r = renderer(sc, instance_cap=1000)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    render_maps(r, 0, cam, sc.octree.C)
    st = r.sync_status(raise_on_overflow=False)
    assert st["status"] == 4 and st["overflow_inst"] > 0
    assert r.sync_status()["overflow_inst"] == 0  # cleared


@pytest.mark.parametrize("n,bits", [(0, 32), (1, 32), (4095, 32), (4097, 16), (100003, 24), (262144 * 3 + 17, 32),
                                    (50000, 8)])
def test_sort_pairs_matches_stable_sort(n, bits):
    import torch
    import paper_2202_05628_gb300 as art
    rng = np.random.default_rng(n)
    k = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        k[: n // 3] = k[n // 3: 2 * (n // 3)]  # many equal keys: stability matters
    v = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(k.view(np.int32)).cuda()
    vt = torch.from_numpy(v.view(np.int32)).cuda()
    r = art.Renderer()
    r.sort_pairs(kt, vt, bits)
    torch.cuda.synchronize()
    mask = np.uint64((1 << bits) - 1)
    order = np.argsort(k.astype(np.uint64) & mask, kind="stable")
    np.testing.assert_array_equal(kt.cpu().numpy().view(np.uint32), k[order])
    np.testing.assert_array_equal(vt.cpu().numpy().view(np.uint32), v[order])


@pytest.mark.parametrize("az,pose_seed,q", [(30.0, 2, 0.5), (200.0, 6, 0.9)])
def test_depth_buffer_matches_oracle(az, pose_seed, q):
    """Depth buffer (Sec. 3.1 "Hybrid Rendering") against the oracle: the same
    pixels have a voxel denser than the threshold and their depths agree to
    FP32 rounding; a first dense hit that grazes its voxel (chord < 1e-5 m)
    may be decided either way by that rounding."""
    import torch
    sc, _, pose = tiny_setup(az=az, pose_seed=pose_seed)
    cam = sg.orbit_camera(sc.centroid, 128, 96, az_deg=az, fov_deg=12.0)
    r = renderer(sc)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    thr = float(np.quantile(sc.octree.density, q))
    D = torch.empty((cam.H, cam.W), dtype=torch.float32, device="cuda")
    r.render_depth(0, thr, D)
    g = D.cpu().numpy().astype(np.float64)
    h = np.zeros((cam.H, cam.W), np.float32)
    r.render_depth(0, thr, h)  # host output
    np.testing.assert_array_equal(h, g.astype(np.float32))
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    o = oracle.depth(sc.octree, A_or, cam, thr)
    fin_o, fin_g = np.isfinite(o["depth"]), np.isfinite(g)
    assert fin_o.sum() > 200
    both = fin_o & fin_g
    dz = np.zeros_like(g)
    dz[both] = np.abs(g[both] - o["depth"][both])  # (inf - inf is not a difference)
    close = (fin_o == fin_g) & (dz <= 1e-5)
    graze = fin_o & (o["chord"] < 1e-5)
    bad = ~close & ~graze
    assert bad.sum() <= max(2, int(0.005 * fin_o.sum())), (bad.sum(), fin_o.sum())
    with pytest.raises(RuntimeError):
        r.render_depth(0, -1.0, D)


def test_reorder_buffer_overflow_is_walked_exactly():
    """40 coincident copies of one voxel (each its own features and density)
    enter every ray through them at the same distance, so more hits pend
    than a pixel's 16-entry reorder buffer holds.  The tile is walked again
    by the exact walk (all hits collected and sorted by entry distance, chord,
    list position = voxel id for equal depth keys), which gives the oracle's
    composite (its ties also by voxel id): no out-of-order release remains,
    in the single-view walk, with short segments, and for a batch of views."""
    import torch
    depth, extent = 4, 1.0
    ijk = np.array([[8, 8, 8]] * 40 + [[8, 8, 9], [9, 8, 8], [7, 8, 8], [8, 9, 8]], np.uint16)
    n = ijk.shape[0]
    rng = np.random.default_rng(17)
    f = rng.standard_normal((n, 8)).astype(np.float32)
    sigma = rng.uniform(1.0, 3.0, n).astype(np.float32)
    jidx = np.zeros((n, 4), np.uint8)
    w = np.zeros((n, 4), np.float32)
    w[:, 0] = 1.0
    oc = sg.Octree(depth, np.array([-0.5, -0.5, -0.5], np.float32), extent, ijk, jidx, w, f, sigma,
                   np.zeros(n, np.float32))
    skel = sg.Skeleton(np.array([-1, 0], np.int32), np.array([[0, 0, 0], [0.1, 0, 0]], np.float32))
    sc = sg.Scene(oc, skel, np.zeros(3), 1.0, None, None)
    centre = oc.centers()[0].astype(np.float64)
    eye = centre + np.array([0.07, 0.11, -1.0])
    cam = sg.Camera(24, 16, 120.0, 120.0, 12.0, 8.0, sg.look_at(eye, centre), 0.1, 3.0)
    o = oracle.render(oc, oracle.pose_transforms(sc, sg.rest_pose(2))[1], cam, hits=True)
    assert o["nhit"].max() >= 40 and (o["nhit"] >= 17).sum() >= 20
    for segment in (256, 32):
        r = renderer(sc, segment=segment)
        set_pose(r, sg.rest_pose(2))
        set_cam(r, 0, cam)
        F, A = render_maps(r, 0, cam, 8)
        st = r.sync_status()
        assert st["overflow_order"] == 0 and st["exact_tiles"] >= 1, st
        np.testing.assert_allclose(F, o["F"], atol=1e-4)
        np.testing.assert_allclose(A, o["A"], atol=1e-4)
        set_cam(r, 1, cam)
        Fs = [torch.zeros((cam.H, cam.W, 8), device="cuda") for _ in range(2)]
        As = [torch.zeros((cam.H, cam.W), device="cuda") for _ in range(2)]
        r.render_views([0, 1], Fs, As)
        st = r.sync_status()
        assert st["overflow_order"] == 0 and st["exact_tiles"] >= 2, st
        for k in range(2):
            np.testing.assert_allclose(Fs[k].cpu().numpy(), o["F"], atol=1e-4)
            np.testing.assert_allclose(As[k].cpu().numpy(), o["A"], atol=1e-4)
