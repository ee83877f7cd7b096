"""Pins of the FP64 convolution oracle (used to check the surrogate's tensor-core kernels):
against torch's CPU conv3d in float64 (a library special case), and the adjoint identities."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dil", [1, 2, 3])
def test_conv3d_matches_library_convolution(dil):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(dil)
    x = rng.standard_normal((2, 3, 7, 6, 9))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = oracle.conv3d_fwd(x, w, b, dil)
    ref = torch.nn.functional.conv3d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b),
                                     padding=dil, dilation=dil).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dil", [1, 2])
def test_conv3d_gradients_are_adjoints(dil):
    """<gy, conv(dx)> = <gx, dx> (linearity in x), <gy, conv_w(dw)> = <gw, dw>, and the bias
    gradient is the sum of gy: exact identities of a linear map."""
    rng = np.random.default_rng(10 + dil)
    x = rng.standard_normal((2, 3, 6, 5, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    gy = rng.standard_normal((2, 4, 6, 5, 7))
    gx, gw, gb = oracle.conv3d_bwd(x, w, gy, dil)
    dx = rng.standard_normal(x.shape)
    lhs = np.sum(gy * oracle.conv3d_fwd(dx, w, None, dil))
    assert abs(lhs - np.sum(gx * dx)) <= 1e-10 * np.abs(lhs)
    dw = rng.standard_normal(w.shape)
    lhs = np.sum(gy * oracle.conv3d_fwd(x, dw, None, dil))
    assert abs(lhs - np.sum(gw * dw)) <= 1e-10 * np.abs(lhs)
    np.testing.assert_allclose(gb, gy.sum(axis=(0, 2, 3, 4)), rtol=1e-12)
