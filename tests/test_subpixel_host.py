"""CPU check of the sub-pixel reading of the level-0 decoder convolution
that the BF16 tensor-core network runs (and that the GPU test's emulation
follows): conv3x3 over [up2(d) | e] equals a convolution of e plus, per
output phase, a convolution of the low-resolution d with summed weights
(Sec. 3.1 "Neural Shading": nearest upsampling, concatenation, 3x3
convolution)."""
import numpy as np
import pytest

from helpers import subpixel_cat_conv


@pytest.mark.parametrize("h,w,cu,cs", [(4, 6, 8, 4), (5, 3, 3, 2)])
def test_subpixel_form_equals_concatenated_convolution(h, w, cu, cs):
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    rng = np.random.default_rng(h * 10 + w)
    d = torch.from_numpy(rng.standard_normal((1, cu, h, w)))
    e = torch.from_numpy(rng.standard_normal((1, cs, 2 * h, 2 * w)))
    wt = rng.standard_normal((7, 3, 3, cu + cs)).astype(np.float32)
    b = rng.standard_normal(7).astype(np.float32)
    x = torch.cat([Fn.interpolate(d, scale_factor=2, mode="nearest"), e], 1)
    ref = torch.relu(Fn.conv2d(x, torch.from_numpy(wt.astype(np.float64)).permute(0, 3, 1, 2),
                               torch.from_numpy(b.astype(np.float64)), padding=1))
    got = subpixel_cat_conv(d, e, (wt, b), bf16=False)
    assert got.shape == ref.shape
    assert float((got - ref).abs().max()) < 1e-12


def test_subpixel_form_with_bf16_taps_stays_within_bf16_error():
    """With the skip weights and the summed taps rounded to BF16 the result
    moves by about one BF16 rounding of the weights (2^-9 relative), not
    more."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    rng = np.random.default_rng(3)
    d = torch.from_numpy(rng.standard_normal((1, 16, 6, 6)))
    e = torch.from_numpy(rng.standard_normal((1, 8, 12, 12)))
    wt = rng.standard_normal((5, 3, 3, 24)).astype(np.float32)
    b = np.zeros(5, np.float32)
    exact = subpixel_cat_conv(d, e, (wt, b), bf16=False)
    got = subpixel_cat_conv(d, e, (wt, b), bf16=True)
    x = torch.cat([Fn.interpolate(d, scale_factor=2, mode="nearest"), e], 1).abs()
    bound = 2.0 ** -8 * Fn.conv2d(x, torch.from_numpy(np.abs(wt).astype(np.float64)).permute(0, 3, 1, 2), padding=1)
    assert bool(((got - exact).abs() <= bound + 1e-12).all())
