"""Host side of the learned ray-interval proposal's training code (CPU only):
its ray encoding and network equal the oracle's definitions, the weights
file round-trips, and the committed weights load."""
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2202_05628_gb300", "weights", "proposal_quadruped_1m_1024.bin")


@pytest.fixture(scope="module")
def prop():
    # the package loads its library on import: build it first (a no-op when current)
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_2202_05628_gb300 import proposal
    return proposal


def test_encoding_equals_the_oracle_inputs(prop):
    cam = sg.orbit_camera(np.array([0.05, 0.1, -0.02]), 24, 16, az_deg=70.0, elev_deg=-5.0)
    pose = sg.random_pose(4)
    x = prop.encode(pose.axis_angle, cam, device="cpu").double().numpy()
    ref = oracle.proposal_inputs(pose.axis_angle, cam)
    assert x.shape == ref.shape == (cam.H * cam.W, 107)
    # pose and direction columns to FP32 rounding; the Fourier columns form
    # their argument 2^k pi u in FP32, off by up to 2^7 pi u 2^-24 ~ 2.4e-5
    np.testing.assert_allclose(x[:, :75], ref[:, :75], atol=2e-6)
    np.testing.assert_allclose(x[:, 75:], ref[:, 75:], atol=4e-5)
    # a subset of pixels encodes as the same rows
    pix = np.array([0, 5, 17, cam.H * cam.W - 1])
    xs = prop.encode_rays(pose.axis_angle, cam, pix, device="cpu").double().numpy()
    np.testing.assert_array_equal(xs, x[pix])


def test_network_equals_the_oracle_mlp(prop):
    p = prop.init_params(7)
    p[64 * 107:64 * 107 + 64] = np.random.default_rng(1).standard_normal(64).astype(np.float32) * 0.1  # a bias
    x = np.random.default_rng(2).standard_normal((50, 107)).astype(np.float32)
    with torch.no_grad():
        y = prop._module(p, "cpu")(torch.from_numpy(x)).double().numpy()
    ref = oracle.proposal_mlp(x.astype(np.float64), p.astype(np.float64))
    np.testing.assert_allclose(y, ref, atol=1e-4 * max(1.0, float(np.abs(ref).max())))
    np.testing.assert_array_equal(prop._flat(prop._module(p, "cpu")), p)


def test_weights_file_round_trip_and_checks(prop, tmp_path):
    p = prop.init_params(3)
    f = tmp_path / "w.bin"
    prop.save(str(f), p, "tiny quadruped")
    q, meta = prop.load(str(f))
    np.testing.assert_array_equal(p, q)
    assert meta == "tiny quadruped"
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTPROP!" + bytes(16))
    with pytest.raises(ValueError):
        prop.load(str(bad))


def test_committed_weights_load(prop):
    if not os.path.exists(WEIGHTS):
        pytest.skip("trained proposal weights missing")
    p, meta = prop.load(WEIGHTS)
    assert p.size == prop.N_PARAMS == 27712 and np.all(np.isfinite(p))
    assert meta  # the file records how it was trained
