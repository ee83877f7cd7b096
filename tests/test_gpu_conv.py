"""Tensor-core 3-D convolution (tcgen05) against the FP64 convolution oracle.

Inputs and weights are rounded to bf16 first, so both sides see identical operands; the GPU
accumulates in FP32. Bars: relative L2 <= 1e-4 for the FP32 channel-0 output, <= 1e-2 for
outputs rounded to bf16 (bf16 keeps 8 significant bits)."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2511_09389_gb300 import build, _native
    build.build()
    assert torch.cuda.is_available()
    return torch, _native.load()


def bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def to_c32(torch, lib, x):
    B, C, D, H, W = x.shape
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    out = torch.empty(B * D * H * W * 32, dtype=torch.bfloat16, device="cuda")
    assert lib.rt_c32_from_f32(xt.data_ptr(), B, C, D, H, W, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    return out


def from_c32(torch, lib, buf, B, C, D, H, W):
    out = torch.empty(B * C * D * H * W, dtype=torch.float32, device="cuda")
    assert lib.rt_c32_to_f32(buf.data_ptr(), B, C, D, H, W, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(B, C, D, H, W).astype(np.float64)


def pack(torch, lib, w, transpose):
    co, ci = w.shape[:2]
    wt = torch.from_numpy(np.ascontiguousarray(w.reshape(co, ci, 27), np.float32)).cuda()
    packed = torch.empty(27 * 32 * 32, dtype=torch.bfloat16, device="cuda")
    assert lib.rt_conv3d_pack_weights(wt.data_ptr(), ci, co, int(transpose), packed.data_ptr(), None) == 0
    torch.cuda.synchronize()
    return packed


def conv_gpu(torch, lib, xc, shape, c_in, packed, bias, c_out, dil, act, slope=0.1, mask=None, f32=False):
    B, D, H, W = shape
    y = torch.full((B * D * H * W * 32,), float("nan"), dtype=torch.bfloat16, device="cuda")
    yf = torch.zeros(B * D * H * W, dtype=torch.float32, device="cuda") if f32 else None
    bt = torch.from_numpy(np.asarray(bias, np.float32)).cuda() if bias is not None else None
    st = lib.rt_conv3d_forward(xc.data_ptr(), B, D, H, W, c_in, packed.data_ptr(),
                               bt.data_ptr() if bt is not None else None, c_out, dil, act, slope,
                               mask.data_ptr() if mask is not None else None, y.data_ptr(),
                               yf.data_ptr() if yf is not None else None, None)
    assert st == 0, lib.rt_last_error()
    code = ctypes.c_int()
    assert lib.rt_device_status(ctypes.byref(code)) == 0, code.value
    # every channel is written: the ones beyond c_out as exact zeros
    pad = y.view(B * D * H * W, 32)[:, c_out:].float().cpu().numpy()
    assert np.all(pad == 0.0)
    return y, yf


@pytest.mark.parametrize("c_in,c_out,dil,act", [(2, 32, 1, 1), (32, 32, 1, 1), (32, 32, 2, 1), (32, 32, 4, 0),
                                                (32, 1, 1, 0), (16, 16, 3, 1), (5, 7, 1, 0)])
def test_conv_forward_matches_oracle(env, c_in, c_out, dil, act):
    torch, lib = env
    rng = np.random.default_rng(c_in * 100 + c_out + dil)
    B, D, H, W = 2, 5, 6, 64
    x = bf16_round(rng.standard_normal((B, c_in, D, H, W)))
    w = bf16_round(rng.standard_normal((c_out, c_in, 3, 3, 3)) / np.sqrt(27 * c_in))
    b = rng.standard_normal(c_out).astype(np.float32).astype(np.float64)
    ref = oracle.conv3d_fwd(x, w, b, dil)
    if act:
        ref = np.where(ref > 0, ref, 0.1 * ref)
    y, yf = conv_gpu(torch, lib, to_c32(torch, lib, x), (B, D, H, W), c_in, pack(torch, lib, w, False), b, c_out,
                     dil, act, f32=True)
    torch.cuda.synchronize()
    assert rel(yf.cpu().numpy().reshape(B, D, H, W), ref[:, 0]) <= 1e-4
    assert rel(from_c32(torch, lib, y, B, c_out, D, H, W), ref) <= 1e-2


def test_conv_masked_output(env):
    """Outputs where a second activation is <= 0 are scaled by the slope (LeakyReLU derivative)."""
    torch, lib = env
    rng = np.random.default_rng(5)
    B, D, H, W, c = 1, 4, 4, 64, 32
    x = bf16_round(rng.standard_normal((B, c, D, H, W)))
    w = bf16_round(rng.standard_normal((c, c, 3, 3, 3)) / np.sqrt(27 * c))
    m = bf16_round(rng.standard_normal((B, c, D, H, W)))
    ref = oracle.conv3d_fwd(x, w, None, 1)
    ref = np.where(m > 0, ref, 0.2 * ref)
    y, _ = conv_gpu(torch, lib, to_c32(torch, lib, x), (B, D, H, W), c, pack(torch, lib, w, False), None, c, 1, 0,
                    slope=0.2, mask=to_c32(torch, lib, m))
    assert rel(from_c32(torch, lib, y, B, c, D, H, W), ref) <= 1e-2


@pytest.mark.parametrize("c_in,c_out,dil", [(32, 32, 1), (32, 32, 2), (32, 1, 1), (2, 32, 1)])
def test_conv_data_gradient_matches_oracle(env, c_in, c_out, dil):
    """dL/dx = the convolution of dL/dy with flipped, transposed weights."""
    torch, lib = env
    rng = np.random.default_rng(7 * c_out + dil)
    B, D, H, W = 2, 4, 4, 64
    x = bf16_round(rng.standard_normal((B, c_in, D, H, W)))
    w = bf16_round(rng.standard_normal((c_out, c_in, 3, 3, 3)) / np.sqrt(27 * c_in))
    gy = bf16_round(rng.standard_normal((B, c_out, D, H, W)))
    gx, _, _ = oracle.conv3d_bwd(x, w, gy, dil)
    y, _ = conv_gpu(torch, lib, to_c32(torch, lib, gy), (B, D, H, W), c_out, pack(torch, lib, w, True), None, c_in,
                    dil, 0)
    assert rel(from_c32(torch, lib, y, B, c_in, D, H, W), gx) <= 1e-2


def test_c32_round_trip(env):
    torch, lib = env
    x = bf16_round(np.random.default_rng(1).standard_normal((3, 19, 2, 4, 64)))
    buf = to_c32(torch, lib, x)
    assert np.array_equal(from_c32(torch, lib, buf, 3, 19, 2, 4, 64), x)
    # layout: channel c of voxel v at element v * 32 + c, channels >= 19 zero
    raw = buf.view(3, 2 * 4 * 64, 32).float().cpu().numpy()
    assert np.array_equal(raw[:, :, :19], x.reshape(3, 19, -1).transpose(0, 2, 1))
    assert np.all(raw[:, :, 19:] == 0.0)


@pytest.mark.parametrize("c_in,c_out,dil", [(32, 32, 1), (32, 32, 4), (2, 32, 1), (32, 1, 2), (9, 5, 1)])
def test_conv_weight_and_bias_gradients_match_oracle(env, c_in, c_out, dil):
    """dL/dw and dL/db, summed over the batch and every voxel, on the tensor cores."""
    torch, lib = env
    rng = np.random.default_rng(31 * c_in + c_out + dil)
    B, D, H, W = 2, 6, 4, 64
    x = bf16_round(rng.standard_normal((B, c_in, D, H, W)))
    gy = bf16_round(rng.standard_normal((B, c_out, D, H, W)))
    w = np.zeros((c_out, c_in, 3, 3, 3))
    _, gw, gb = oracle.conv3d_bwd(x, w, gy, dil)
    dw = torch.zeros(c_out * c_in * 27, dtype=torch.float32, device="cuda")
    db = torch.zeros(c_out, dtype=torch.float32, device="cuda")
    xc, gc = to_c32(torch, lib, x), to_c32(torch, lib, gy)      # keep both alive until the kernel ran
    st = lib.rt_conv3d_weight_grad(xc.data_ptr(), gc.data_ptr(), B, D, H, W, c_in, c_out, dil, dw.data_ptr(),
                                   db.data_ptr(), None)
    assert st == 0, lib.rt_last_error()
    code = ctypes.c_int()
    assert lib.rt_device_status(ctypes.byref(code)) == 0, code.value
    assert rel(dw.cpu().numpy().reshape(gw.shape), gw) <= 1e-4
    assert rel(db.cpu().numpy(), gb) <= 1e-4


@pytest.mark.parametrize("shape,c_in,c_out,dil", [((3, 20, 4, 64), 32, 32, 1), ((2, 19, 6, 64), 32, 32, 2),
                                                  ((1, 27, 2, 64), 7, 32, 3), ((2, 9, 8, 64), 32, 3, 4)])
def test_conv_weight_gradient_across_chain_segments(env, shape, c_in, c_out, dil):
    """The weight gradient walks chains of outputs along z in segments of at most eight: depths
    with several segments per chain (and a ragged last one), every residue of the dilation, more
    items than the dZ ring and input stages hold, against the FP64 oracle."""
    torch, lib = env
    B, D, H, W = shape
    rng = np.random.default_rng(7 * D + dil)
    x = bf16_round(rng.standard_normal((B, c_in, D, H, W)))
    gy = bf16_round(rng.standard_normal((B, c_out, D, H, W)))
    _, gw, gb = oracle.conv3d_bwd(x, np.zeros((c_out, c_in, 3, 3, 3)), gy, dil)
    dw = torch.zeros(c_out * c_in * 27, dtype=torch.float32, device="cuda")
    db = torch.zeros(c_out, dtype=torch.float32, device="cuda")
    xc, gc = to_c32(torch, lib, x), to_c32(torch, lib, gy)
    st = lib.rt_conv3d_weight_grad(xc.data_ptr(), gc.data_ptr(), B, D, H, W, c_in, c_out, dil, dw.data_ptr(),
                                   db.data_ptr(), None)
    assert st == 0, lib.rt_last_error()
    code = ctypes.c_int()
    assert lib.rt_device_status(ctypes.byref(code)) == 0, code.value
    assert rel(dw.cpu().numpy().reshape(gw.shape), gw) <= 1e-4
    assert rel(db.cpu().numpy(), gb) <= 1e-4
