"""The convolutional surrogate, trained by the library's own kernels.

- Parameter gradients of the whole network (loss -> five tensor-core convolution layers)
  against an FP64 CPU reference built from the convolution oracle, with bf16 rounding applied
  where the GPU path stores bf16 (features, activations, back-propagated gradients, weights).
- Training reduces the loss on march-generated fields; the error estimate, its calibration and
  the fallback to the plain march behave as specified.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_network_gradients_match_fp64_reference(env):
    torch = env
    from paper_2511_09389_gb300 import surrogate as S
    rng = np.random.default_rng(0)
    B, D, H, W = 2, 4, 4, 64
    kappa = (0.05 * np.exp(0.7 * rng.standard_normal((B, D, H, W)))).astype(np.float32)
    j = np.abs(rng.standard_normal((B, D, H, W))).astype(np.float32)
    field = (np.exp(2 * rng.standard_normal((B, D, H, W)))).astype(np.float32)
    model = S.Surrogate(seed=3)
    model.mu, model.sigma = -1.0, 2.0
    kt, jt, ft = (torch.from_numpy(a).cuda() for a in (kappa, j, field))
    fmax = S.field_max(model.lib, ft, model.device)
    pred = model.forward(kt, jt, keep=True)
    model.loss_and_backward(pred, ft, fmax)
    torch.cuda.synchronize()
    g_gpu = model.grads.cpu().numpy().astype(np.float64)
    P = model.params.cpu().numpy().astype(np.float64)

    # FP64 reference on the same rounded operands
    feats = np.stack([np.log(np.maximum(kappa, 1e-30).astype(np.float64) * 20.0), np.log1p(j.astype(np.float64))], 1)
    a = bf16(feats)
    acts = [a]
    Ws = []
    for l, (ci, co, dil, act) in enumerate(S.LAYERS):
        wo, wn, bo, bn = model.shapes[l]
        w = bf16(P[wo:wo + wn]).reshape(co, ci, 3, 3, 3)
        Ws.append(w)
        z = oracle.conv3d_fwd(a, w, P[bo:bo + bn], dil)
        if act:
            a = bf16(np.where(z > 0, z, S.SLOPE * z))
            acts.append(a)
        else:
            pred_ref = z[:, 0]
    np.testing.assert_allclose(pred.cpu().numpy(), pred_ref, rtol=2e-2, atol=2e-2 * np.abs(pred_ref).max())
    eps = S.EPS_REL * field.reshape(B, -1).max(1).astype(np.float64)
    T = (np.log(field + eps[:, None, None, None]) - model.mu) / model.sigma
    g = bf16((2.0 * (pred.cpu().numpy().astype(np.float64) - T) / T.size)[:, None])
    for l in range(len(S.LAYERS) - 1, -1, -1):
        ci, co, dil, _ = S.LAYERS[l]
        wo, wn, bo, bn = model.shapes[l]
        gx, gw, gb = oracle.conv3d_bwd(acts[l], Ws[l], g, dil)
        assert rel(g_gpu[wo:wo + wn], gw.ravel()) <= 1e-2, (l, rel(g_gpu[wo:wo + wn], gw.ravel()))
        assert rel(g_gpu[bo:bo + bn], gb) <= 1e-2, (l, rel(g_gpu[bo:bo + bn], gb))
        if l > 0:
            g = bf16(np.where(acts[l] > 0, gx, S.SLOPE * gx))


def test_training_reduces_loss_and_fallback_is_the_march(env):
    torch = env
    from paper_2511_09389_gb300 import surrogate as S
    from paper_2511_09389_gb300.api import Grid
    grid = Grid((64, 64, 64), 1)
    train = S.Dataset(range(48), grid, num_rays=768)
    model = S.Surrogate(seed=1)
    losses = S.train(model, train, epochs=4, batch=16, lr=3e-3)
    assert all(math.isfinite(x) for x in losses)
    assert losses[-1] < 0.7 * losses[0], losses
    errs, est = S.fit_estimator(model, train, batch=16)
    assert np.all(np.isfinite(est)) and errs.shape == (48,)
    # with no field inside the bound the threshold is -inf: everything falls back to the march
    held = S.Dataset(range(1000, 1016), grid, num_rays=768)
    model.est_threshold = -math.inf
    out = S.evaluate(model, grid, held, batch=16)
    assert out["fallback_fraction"] == 1.0
    assert out["fields"] == 16 and out["plain_fields_per_s"] > 0
