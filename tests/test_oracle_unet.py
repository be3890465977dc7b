"""Pins of the U-Net oracle (oracle/unet.py): each layer against PyTorch's CPU routines (a library
computation independent of the oracle's code), the whole network's explicit backward against central
finite differences, the parameter count of the specified architecture, and the sample encoding."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet


def _t(a):
    return torch.tensor(a, dtype=torch.float64)


@pytest.mark.parametrize("k", [3, 1])
def test_conv3d_forward_and_backward_match_torch(k):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 6, 5, 4))
    w = rng.standard_normal((5, 3, k, k, k))
    b = rng.standard_normal(5)
    y = unet.conv3d(x, w, b)
    xt, wt, bt = _t(x).requires_grad_(), _t(w).requires_grad_(), _t(b).requires_grad_()
    yt = F.conv3d(xt, wt, bt, padding=k // 2)
    assert np.abs(y - yt.detach().numpy()).max() < 1e-12
    gy = rng.standard_normal(y.shape)
    yt.backward(_t(gy))
    gx, gw, gb = unet.conv3d_backward(x, w, gy)
    assert np.abs(gx - xt.grad.numpy()).max() < 1e-11
    assert np.abs(gw - wt.grad.numpy()).max() < 1e-10
    assert np.abs(gb - bt.grad.numpy()).max() < 1e-11


def test_pool_and_upsample_match_torch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 6, 8))
    y, arg = unet.maxpool2(x)
    assert np.array_equal(y, F.max_pool3d(_t(x), 2).numpy())
    xt = _t(x).requires_grad_()
    yt = F.max_pool3d(xt, 2)
    gy = rng.standard_normal(y.shape)
    yt.backward(_t(gy))
    assert np.array_equal(unet.maxpool2_backward(arg, gy, x.shape), xt.grad.numpy())
    u = unet.upsample2(y)
    assert np.array_equal(u, F.interpolate(_t(y), scale_factor=2, mode="nearest").numpy())
    yt2 = _t(y).requires_grad_()
    ut = F.interpolate(yt2, scale_factor=2, mode="nearest")
    gu = rng.standard_normal(u.shape)
    ut.backward(_t(gu))
    assert np.abs(unet.upsample2_backward(gu) - yt2.grad.numpy()).max() < 1e-12


def test_parameter_count_of_the_specified_network():
    """4 levels 16/32/64/64, 6 inputs, 4 outputs: sum over the 13 convolutions of
    c_in * c_out * 27 + c_out, plus the 1x1x1 head 16 * 4 + 4 = 908,708."""
    assert unet.UNet().n_params() == 908708


def test_network_gradient_by_central_differences():
    """2 levels, 4 and 8 channels, 8^3 input: dL/dtheta and dL/dx of L = sum(G * out) from the explicit
    backward agree with central differences (FP64, relative 1e-6) on sampled entries."""
    net = unet.UNet(channels=(4, 8), seed=3)
    rng = np.random.default_rng(4)
    for v in net.params.values():          # non-zero biases so their gradients are exercised too
        if v.ndim == 1:
            v[:] = 0.1 * rng.standard_normal(v.shape)
    x = rng.standard_normal((1, 6, 8, 8, 8))
    out, cache = net.forward(x)
    G = rng.standard_normal(out.shape)
    grads, gx = net.backward(cache, G)

    def loss():
        return float((net.forward(x)[0] * G).sum())

    eps = 1e-6
    for name in ["enc0.0.w", "enc1.1.w", "dec0.0.w", "dec0.1.b", "head.w", "head.b", "enc1.0.b"]:
        p = net.params[name]
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss()
            flat[idx] = old - eps
            lm = loss()
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)
    flatx = x.reshape(-1)
    for idx in rng.choice(flatx.size, size=6, replace=False):
        old = flatx[idx]
        flatx[idx] = old + eps
        lp = loss()
        flatx[idx] = old - eps
        lm = loss()
        flatx[idx] = old
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gx.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_sample_encoding_is_scale_free_and_round_trips():
    rng = np.random.default_rng(5)
    shape = (4, 6, 8)
    n = int(np.prod(shape))
    mask = (rng.random(shape) > 0.3).astype(np.uint8)
    xs = rng.standard_normal(4 * n)
    xns = xs + 0.1 * rng.standard_normal(4 * n)
    f, U, P = unet.features(mask, xs, 10.0)
    assert f.shape == (1, 6) + shape and np.all(f[0, 5] == 1.0)
    assert np.isclose(np.abs(f[0, 1:4]).max(), 1.0) and np.isclose(np.abs(f[0, 4]).max(), 1.0)
    f2, _, _ = unet.features(mask, 3.0 * xs, 10.0)
    assert np.allclose(f, f2, rtol=1e-15, atol=0)
    t = unet.targets(xns, xs, shape, U, P)
    assert np.allclose(unet.proposal(t, xs, shape, U, P), xns, rtol=1e-14, atol=1e-14)


def test_adam_matches_torch():
    rng = np.random.default_rng(6)
    p0 = {"a": rng.standard_normal((3, 4)), "b": rng.standard_normal(5)}
    params = {k: v.copy() for k, v in p0.items()}
    opt = unet.Adam(params, lr=1e-2)
    tp = {k: _t(v).requires_grad_() for k, v in p0.items()}
    topt = torch.optim.Adam(list(tp.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(5):
        grads = {k: rng.standard_normal(v.shape) for k, v in p0.items()}
        opt.step(params, grads)
        topt.zero_grad()
        for k in tp:
            tp[k].grad = _t(grads[k])
        topt.step()
    for k in params:
        assert np.abs(params[k] - tp[k].detach().numpy()).max() < 1e-12


def test_masked_mse_gradient_and_a_small_fit():
    """The loss gradient by central differences, then 60 Adam steps of a 2-level network on one
    8^3 sample lower the masked loss by at least 10x."""
    rng = np.random.default_rng(7)
    out = rng.standard_normal((1, 4, 4, 4, 4))
    tgt = rng.standard_normal(out.shape)
    wgt = (rng.random((1, 1, 4, 4, 4)) > 0.3).astype(np.float64)
    L, g = unet.masked_mse(out, tgt, wgt)
    e = 1e-6
    for idx in [(0, 1, 2, 3, 1), (0, 3, 0, 0, 2)]:
        o2 = out.copy(); o2[idx] += e
        o3 = out.copy(); o3[idx] -= e
        fd = (unet.masked_mse(o2, tgt, wgt)[0] - unet.masked_mse(o3, tgt, wgt)[0]) / (2 * e)
        assert abs(fd - g[idx]) < 1e-8
    net = unet.UNet(channels=(4, 8), seed=8)
    x = rng.standard_normal((1, 6, 8, 8, 8))
    t = 0.1 * rng.standard_normal((1, 4, 8, 8, 8))
    w = np.ones((1, 1, 8, 8, 8))
    opt = unet.Adam(net.params, lr=3e-3)
    first = None
    for _ in range(60):
        out, cache = net.forward(x)
        L, gout = unet.masked_mse(out, t, w)
        first = L if first is None else first
        grads, _ = net.backward(cache, gout)
        opt.step(net.params, grads)
    assert L < 0.1 * first, (first, L)
