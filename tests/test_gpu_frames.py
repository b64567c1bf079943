"""Frames queued with art_render_frame_async (two in flight, RGBA copied to
pinned host buffers on a second stream) against art_render_frame, and the
refusal of a device output buffer."""
import numpy as np
import pytest

import scenegen as sg
from helpers import renderer, set_cam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _frame_renderer(sc, cams):
    import paper_2202_05628_gb300 as art
    oc = sc.octree
    r = renderer(sc)
    r.load_shader(art.ART_NET_TINY, oc.C, [32], 4, art.flat_params(sg.tiny_net_weights(0, cin=oc.C)), "f32")
    for v, cam in enumerate(cams):
        set_cam(r, v, cam)
    return r


def test_async_frames_equal_synchronous_frames():
    """Five frames over two views (the third and later wait for the oldest
    frame's slot): each host buffer holds its own frame, equal to the
    synchronous call's."""
    import torch
    import paper_2202_05628_gb300 as art
    sc = sg.preset("tiny")
    cams = [sg.orbit_camera(sc.centroid, 96, 80, az_deg=a) for a in (20.0, 150.0)]
    poses = [sg.random_pose(40 + k) for k in range(5)]
    r = _frame_renderer(sc, cams)
    want = []
    for k, p in enumerate(poses):
        out = np.zeros((80, 96, 4), np.float32)
        r.render_frame(k % 2, p.axis_angle, p.R, p.T, out)
        want.append(out)
    pinned = [(torch.from_numpy(p.axis_angle).pin_memory(), torch.from_numpy(p.R).pin_memory(),
               torch.from_numpy(p.T).pin_memory()) for p in poses]
    outs = [torch.full((80, 96, 4), -1.0, dtype=torch.float32, pin_memory=True) for _ in poses]
    for k in range(len(poses)):
        r.render_frame_async(k % 2, *pinned[k], outs[k])
    r.wait_frames()
    for k in range(len(poses)):
        got = outs[k].numpy()
        assert np.abs(got - want[k]).max() <= 1e-6, k
    assert r.sync_status()["overflow_order"] == 0
    # a device buffer is refused (art_render_frame takes those)
    dev = torch.empty((80, 96, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(art.ArtemisError) as ex:
        r.render_frame_async(0, *pinned[0], dev)
    assert ex.value.status == 1
    r.wait_frames()
    r.close()
