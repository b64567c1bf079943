"""The paper's per-frame index on the GPU (art_config.index = ART_INDEX_GRID,
Sec. 3.1 "Dynamic Volume Rendering"): warped centres snapped to the leaf
lattice, the smallest id surviving a cell, the occupied cells rendered as
axis-aligned leaf boxes; against the FP64 oracle's orc_grid_snap /
orc_render_grid, through the C ABI.

A warped centre within 1e-4 h of a cell face (4x the FP32 error of the
library's warped centres at these sizes) has its cell decided by rounding:
such voxels, the cells they may land in and the pixels that see those cells
are left out; everything else must agree exactly (cells, survivors) or
within 1e-4 (F, A; order-ambiguous pixels left out as for the exact boxes)."""
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


def _gpu_cells(r, oc):
    """Survivor flags and lattice cells from the library's rewritten records."""
    rec = r.debug_buffer(1, np.float32)[:oc.n * 16].reshape(oc.n, 16)
    alive = rec[:, 13] != 0.0
    cw = rec[:, [3, 7, 11]].astype(np.float64)
    h = oc.extent / (1 << oc.depth)
    cell = np.floor((cw - np.asarray(oc.origin, np.float64)) / h).astype(np.int64)
    return alive, cell


def _contested(oc, A, eps=1e-4):
    """Voxels whose FP64 warped centre lies within eps h of a cell face, and
    every cell such a voxel may land in."""
    h = oc.extent / (1 << oc.depth)
    org = np.asarray(oc.origin, np.float64)
    pc = org + (oc.ijk.astype(np.float64) + 0.5) * h
    A = np.asarray(A).reshape(-1, 3, 4)
    p = np.einsum("nij,nj->ni", A[:, :, :3], pc) + A[:, :, 3]
    u = (p - org) / h
    fr = u - np.floor(u)
    near = np.minimum(fr, 1.0 - fr) < eps
    amb = np.flatnonzero(near.any(1))
    cells = set()
    for i in amb:
        base = np.floor(u[i]).astype(np.int64)
        opts = [[0, -1 if fr[i, a] < 0.5 else 1] if near[i, a] else [0] for a in range(3)]
        for dx in opts[0]:
            for dy in opts[1]:
                for dz in opts[2]:
                    cells.add((base[0] + dx, base[1] + dy, base[2] + dz))
    return amb, cells


def _cell_pixels(cells, oc, cam):
    """Pixels whose centre may see one of the cells (projected corner boxes grown by a pixel)."""
    h = oc.extent / (1 << oc.depth)
    org = np.asarray(oc.origin, np.float64)
    M = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    out = np.zeros((cam.H, cam.W), bool)
    for c in cells:
        lo = org + np.asarray(c, np.float64) * h
        corners = lo + h * np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float64)
        X = corners @ M[:, :3].T + M[:, 3]
        if np.any(X[:, 2] <= 1e-6):
            continue
        u = cam.fx * X[:, 0] / X[:, 2] + cam.cx
        v = cam.fy * X[:, 1] / X[:, 2] + cam.cy
        x0, x1 = int(np.floor(u.min() - 1.5)), int(np.ceil(u.max() + 0.5))
        y0, y1 = int(np.floor(v.min() - 1.5)), int(np.ceil(v.max() + 0.5))
        out[max(y0, 0):max(min(y1, cam.H - 1) + 1, 0), max(x0, 0):max(min(x1, cam.W - 1) + 1, 0)] = True
    return out


def _cells_octree(oc, cell, winner):
    """The survivors placed on their cells as an axis-aligned octree (identity
    transforms): the oracle's hit lists of the index render."""
    surv = np.flatnonzero(winner == np.arange(oc.n))
    c = cell[surv]
    cmin = c.min(0)
    h = oc.extent / (1 << oc.depth)
    ijk = (c - cmin).astype(np.uint16)
    origin = (np.asarray(oc.origin, np.float64) + cmin * h).astype(np.float64)
    m = surv.size
    w = np.zeros((m, 4), np.float32)
    w[:, 0] = 1.0
    return sg.Octree(oc.depth, origin, oc.extent, ijk, np.zeros((m, 4), np.uint8), w, oc.features[surv],
                     oc.density[surv], np.zeros(m, np.float32)), surv


def test_grid_index_at_rest_is_the_voxel_render():
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 128, 96, az_deg=25.0, fov_deg=14.0)
    r = renderer(sc)
    r.set_config(index=1)
    set_pose(r, sg.rest_pose())
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, oc.C)
    st = r.sync_status()
    assert st["grid_cells"] == oc.n  # every voxel in its own leaf
    _, A_or, _ = oracle.pose_transforms(sc, sg.rest_pose())
    og = oracle.render_grid(oc, A_or, cam)
    o = oracle.render(oc, A_or, cam, hits=True)
    keep = ~order_ambiguous(o, oc, cam.H, cam.W)
    assert (og["A"] > 0).sum() > 500
    assert np.abs(F - og["F"])[keep].max() < 1e-4 and np.abs(A - og["A"])[keep].max() < 1e-4


@pytest.mark.parametrize("pose_seed,az", [(3, 60.0), (9, 210.0)])
def test_grid_index_under_pose_matches_oracle(pose_seed, az):
    sc = sg.preset("tiny")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 128, 96, az_deg=az, fov_deg=14.0)
    pose = sg.random_pose(pose_seed)
    r = renderer(sc)
    r.set_config(index=1)
    set_pose(r, pose)
    set_cam(r, 0, cam)
    F, A = render_maps(r, 0, cam, oc.C)
    st = r.sync_status()
    alive, gcell = _gpu_cells(r, oc)
    _, A_or, _ = oracle.pose_transforms(sc, pose)
    snap = oracle.grid_snap(oc, A_or)
    cell, winner = snap["cell"], snap["winner"]
    amb, cells = _contested(oc, A_or)
    cell_t = [tuple(c) for c in cell]
    free = np.array([tuple(c) not in cells for c in cell_t]) & (winner >= 0)
    free[amb] = False
    assert free.mean() > 0.9
    # survivors and their cells: exact outside the contested cells
    o_alive = winner == np.arange(oc.n)
    np.testing.assert_array_equal(alive[free], o_alive[free])
    np.testing.assert_array_equal(gcell[free & o_alive], cell[free & o_alive])
    collided = int((winner >= 0).sum() - o_alive.sum())
    assert collided > 0  # the pose makes voxels collide
    assert abs(st["grid_cells"] - int(o_alive.sum())) <= len(cells)
    # F, A against the oracle's index render
    og = oracle.render_grid(oc, A_or, cam)
    co, _ = _cells_octree(oc, cell, winner)
    ID = np.zeros((co.n, 3, 4))
    ID[:, 0, 0] = ID[:, 1, 1] = ID[:, 2, 2] = 1.0
    oh = oracle.render(co, ID, cam, hits=True)
    np.testing.assert_allclose(oh["F"], og["F"], atol=1e-12)  # the same render (pinned on the CPU)
    keep = ~order_ambiguous(oh, co, cam.H, cam.W) & ~_cell_pixels(cells, oc, cam)
    assert keep.sum() > 0.8 * cam.H * cam.W and (og["A"][keep] > 0).sum() > 300
    assert np.abs(F - og["F"])[keep].max() < 1e-4
    assert np.abs(A - og["A"])[keep].max() < 1e-4


def test_grid_index_refuses_the_backward_and_switches_back():
    import torch
    import paper_2202_05628_gb300 as art
    sc = sg.preset("mini")
    oc = sc.octree
    cam = sg.orbit_camera(sc.centroid, 64, 64, fov_deg=20.0)
    r = renderer(sc)
    set_cam(r, 0, cam)
    pose = sg.random_pose(4)
    set_pose(r, pose)
    F0, A0 = render_maps(r, 0, cam, oc.C)
    r.set_config(index=1)
    set_pose(r, pose)
    Fg = torch.zeros((64, 64, oc.C), device="cuda")
    Ag = torch.zeros((64, 64), device="cuda")
    r.render_feature_maps(0, Fg, Ag)
    with pytest.raises(art.ArtemisError):
        r.render_backward(0, Fg, Ag, Fg, Ag, torch.zeros((oc.n, oc.C), device="cuda"),
                          torch.zeros(oc.n, device="cuda"), torch.zeros((oc.n, 4), device="cuda"))
    r.set_config(index=0)
    set_pose(r, pose)
    F1, A1 = render_maps(r, 0, cam, oc.C)
    np.testing.assert_array_equal(F1, F0)
    np.testing.assert_array_equal(A1, A0)
