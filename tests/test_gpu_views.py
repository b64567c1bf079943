"""Several views of one pose in one pass (art_render_views: one tile space
over the views, one scan, scatter, sort and composite walk), against the
single-view render of each view and against the FP64 oracle, through the C
ABI."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from helpers import order_ambiguous, render_maps, renderer, set_cam, set_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cams(sc):
    # a stereo pair (6.4 cm baseline) and a third view of another, ragged size
    return [sg.orbit_camera(sc.centroid, 128, 96, az_deg=60.0, fov_deg=14.0, shift_x=s) for s in (-0.032, 0.032)] + \
           [sg.orbit_camera(sc.centroid, 100, 70, az_deg=200.0, fov_deg=12.0)]


def _batch(r, cams, C, F_dtype="f32", views=None):
    import torch
    dt = torch.float32 if F_dtype == "f32" else torch.bfloat16
    views = list(range(len(cams))) if views is None else views
    Fs = [torch.full((c.H, c.W, C), 7.0, dtype=dt, device="cuda") for c in cams]  # stale values must be overwritten
    As = [torch.full((c.H, c.W), 7.0, dtype=torch.float32, device="cuda") for c in cams]
    r.render_views(views, Fs, As, F_dtype)
    torch.cuda.synchronize()
    return [F.float().cpu().numpy() for F in Fs], [A.cpu().numpy() for A in As]


def test_views_in_one_pass_match_single_views_and_oracle():
    sc = sg.preset("tiny")
    oc = sc.octree
    pose = sg.random_pose(6)
    cams = _cams(sc)
    r = renderer(sc, profile=True)
    set_pose(r, pose)
    singles, inst = [], 0
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
        singles.append(render_maps(r, v, cam, oc.C))
        inst += r.sync_status()["instances"]
    r.kernel_times(reset=True)
    Fs, As = _batch(r, cams, oc.C)
    st = r.sync_status()
    kt = r.kernel_times()
    assert st["instances"] == inst  # the same instances, in one tile space
    assert kt["bin_scan"][0] == 1 and kt["tile_sort"][0] == 1 and kt["composite"][0] == 1, kt
    assert kt["project"][0] == len(cams) and kt["bin_emit"][0] == len(cams), kt
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    for v, cam in enumerate(cams):
        F1, A1 = singles[v]
        # the same sums, regrouped by other segment cuts
        assert np.abs(Fs[v] - F1).max() < 1e-6 and np.abs(As[v] - A1).max() < 1e-6, v
        o = oracle.render(oc, A_or, cam, hits=True)
        keep = ~order_ambiguous(o, oc, cam.H, cam.W)
        assert (o["A"] > 0).sum() > 200
        assert np.abs(Fs[v] - o["F"])[keep].max() < 1e-4, v
        assert np.abs(As[v] - o["A"])[keep].max() < 1e-4, v


def test_views_bf16_output_and_a_subset_in_another_order():
    sc = sg.preset("tiny")
    oc = sc.octree
    pose = sg.random_pose(8)
    cams = _cams(sc)
    r = renderer(sc, storage="bf16")
    set_pose(r, pose)
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
    Fs, As = _batch(r, [cams[2], cams[0]], oc.C, "bf16", views=[2, 0])
    for F, A, v in zip(Fs, As, (2, 0)):
        F1, A1 = render_maps(r, v, cams[v], oc.C, "bf16")
        assert np.abs(F - F1).max() <= 2.0 ** -7 * max(1.0, np.abs(F1).max())  # one BF16 rounding of the output
        assert np.abs(A - A1).max() < 1e-6


def test_views_with_learned_skip_render_view_by_view():
    import paper_2202_05628_gb300 as art
    from paper_2202_05628_gb300 import proposal as prop
    sc = sg.preset("tiny")
    oc = sc.octree
    pose = sg.random_pose(2)
    cams = _cams(sc)[:2]
    r = renderer(sc)
    rng = np.random.default_rng(0)
    r.load_proposal((0.05 * rng.standard_normal(art.PROPOSAL_PARAMS)).astype(np.float32))
    r.set_config(skip=1, max_missed=1e-3, margin=1)
    set_pose(r, pose)
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
    Fs, As = _batch(r, cams, oc.C)
    for v, cam in enumerate(cams):
        F1, A1 = render_maps(r, v, cam, oc.C)
        np.testing.assert_array_equal(Fs[v], F1)
        np.testing.assert_array_equal(As[v], A1)
    del prop


def test_views_refuse_bad_arguments():
    import torch
    import paper_2202_05628_gb300 as art
    sc = sg.preset("mini")
    r = renderer(sc)
    cam = sg.orbit_camera(sc.centroid, 32, 32)
    set_cam(r, 0, cam)
    set_pose(r, sg.random_pose(1))
    F = torch.zeros((32, 32, sc.octree.C), device="cuda")
    with pytest.raises(art.ArtemisError):
        r.render_views([0, 0], [F, F])  # a view twice
    with pytest.raises(art.ArtemisError):
        r.render_views([0, 3], [F, F])  # a view never set
    with pytest.raises(art.ArtemisError):
        r.render_views([0], [np.zeros((32, 32, sc.octree.C), np.float32)])  # host output


def test_views_stereo_1080p_fullsize_sampled():
    """The 1M-voxel octree, the stereo pair of 1920x1080 views in one pass
    (FP32 features): sampled pixels within 1e-4 of the oracle (brute force
    over every voxel), order-ambiguous ones left out."""
    import torch
    sc = sg.preset("paper")
    oc = sc.octree
    pose = sg.walk_pose(29, 60)
    cams = [sg.orbit_camera(sc.centroid, 1920, 1080, az_deg=300.0, shift_x=s) for s in (-0.032, 0.032)]
    r = renderer(sc)
    set_pose(r, pose)
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
    Fs = [torch.zeros((c.H, c.W, oc.C), device="cuda") for c in cams]
    As = [torch.zeros((c.H, c.W), device="cuda") for c in cams]
    r.render_views([0, 1], Fs, As)
    st = r.sync_status()
    assert st["overflow_inst"] == 0 and st["overflow_order"] == 0
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    rng = np.random.default_rng(31)
    for v, cam in enumerate(cams):
        F, A = Fs[v].cpu().numpy(), As[v].cpu().numpy()
        cov = np.flatnonzero(A.reshape(-1) > 0)
        bg = np.flatnonzero(A.reshape(-1) <= 0)
        pick = np.concatenate([rng.choice(cov, 192, replace=False), rng.choice(bg, 32, replace=False)])
        px, py = pick % cam.W, pick // cam.W
        o = oracle.pixels(oc, A_or, cam, px, py, tie_eps=1e-6)
        keep = o["tie"] <= 1e-5
        assert keep.mean() >= 0.9
        dF = np.abs(F[py, px] - o["F"]).max(1)
        dA = np.abs(A[py, px] - o["A"])
        print(f"stereo 1080p eye {v}: max |dF| {dF[keep].max():.3e}, max |dA| {dA[keep].max():.3e} "
              f"over {int(keep.sum())} pixels ({int((~keep).sum())} order-ambiguous left out)")
        assert dF[keep].max() <= 1e-4 and dA[keep].max() <= 1e-4
