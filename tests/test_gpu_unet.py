"""The learned initial guess on the GPU (include/pns_unet.h) against the NumPy oracle of the network
(oracle/unet.py, pinned against torch's conv3d, max-pool, upsampling and Adam and by central
differences): forward, parameter gradients of the masked MSE loss, one Adam step, the sample encodings,
and a short fit.

The library keeps activations and working weights in BF16 and accumulates in FP32, so it is compared with
the oracle run in FP64 on the same (FP32 master) weights.  Bars, from the arithmetic: each of the <= 9
stacked layers rounds its input and weights to BF16 (relative 2^-9 per factor) and its output again, so
the network output carries a few 1e-3 of relative error and the gradients about 1e-2; the bars are 3e-2
(output) and 6e-2 (gradients, relative L2 over each parameter tensor), where a wrong tap order, a
transposed weight, a missing bias or a dropped skip connection leaves an O(1) error."""
import numpy as np
import pytest

from oracle import unet as ou

pytestmark = pytest.mark.gpu


def _net(channels, shape, batch, seed=0):
    from paper_2510_22077_gb300 import pns
    ref = ou.UNet(channels=channels, in_ch=6, out_ch=4, seed=seed)
    # non-zero biases so that a dropped bias shows
    rng = np.random.default_rng(seed + 100)
    for k in ref.params:
        if k.endswith(".b"):
            ref.params[k] = 0.05 * rng.standard_normal(ref.params[k].shape)
    net = pns.UNet(channels=channels, in_ch=6, out_ch=4, batch=batch, shape=shape, seed=seed)
    names = pns.unet_param_names(len(channels))
    assert sorted(names) == sorted(ref.params)
    flat = np.concatenate([ref.params[n].ravel() for n in names]).astype(np.float32)
    assert flat.size == net.num_params() == ref.n_params()
    net.set_params(flat)
    # the oracle works on the FP32 values the library holds
    for n in names:
        ref.params[n] = ref.params[n].astype(np.float32).astype(np.float64)
    return ref, net, names


def _sample(batch, shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((batch, 6) + shape)
    x[:, 0] = rng.random((batch,) + shape) > 0.4        # a void mask channel
    t = 0.3 * rng.standard_normal((batch, 4) + shape)
    w = x[:, :1].copy()
    return x, t, w


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("channels,shape,batch", [((8,), (8, 8, 8), 2), ((8, 16), (8, 8, 16), 2),
                                                  ((16, 32, 64, 64), (16, 16, 16), 1)])
def test_forward_and_gradients_match_oracle(channels, shape, batch):
    ref, net, names = _net(channels, shape, batch)
    x, t, w = _sample(batch, shape, seed=3)
    out_o, cache = ref.forward(x)
    out_g = net.forward(_dev(x)).cpu().numpy()
    e_out = _rel(out_g, out_o)
    L_o, g_o = ou.masked_mse(out_o, t, w)
    # the library's loss gradient, then its backward, on its own output
    L_g, gout = net.mse(_dev(out_g), _dev(t), _dev(w))
    L_ref_on_gpu_out, g_ref = ou.masked_mse(out_g.astype(np.float64), t, w)
    assert abs(L_g - L_ref_on_gpu_out) <= 1e-5 * L_ref_on_gpu_out
    assert _rel(gout.cpu().numpy(), g_ref) < 1e-5
    net.backward(gout)
    grads_o, _ = ref.backward(cache, g_o)
    gg = net.get_grads()
    off = 0
    worst = 0.0
    lines = []
    for n in names:
        sz = ref.params[n].size
        e = _rel(gg[off:off + sz], grads_o[n].ravel())
        lines.append(f"{n}: {e:.2e}")
        worst = max(worst, e)
        off += sz
    print(f"U-Net {channels} {shape} x{batch}: output rel err {e_out:.2e}; gradient rel err worst {worst:.2e} "
          f"({', '.join(lines)})")
    assert e_out < 3e-2
    assert worst < 6e-2


def test_adam_step_matches_oracle():
    ref, net, names = _net((8, 16), (8, 8, 8), 1)
    x, t, w = _sample(1, (8, 8, 8), seed=5)
    p0 = net.get_params().astype(np.float64)
    out = net.forward(_dev(x))
    _, gout = net.mse(out, _dev(t), _dev(w))
    net.backward(gout)
    g = net.get_grads().astype(np.float64)
    net.adam(lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    # the oracle's Adam on the library's own gradients
    P = {"p": p0.copy()}
    opt = ou.Adam(P, lr=1e-3)
    opt.step(P, {"p": g})
    assert _rel(p1 - p0, P["p"] - p0) < 1e-4


def test_training_reduces_the_loss():
    ref, net, names = _net((8, 16), (8, 8, 8), 2)
    x, t, w = _sample(2, (8, 8, 8), seed=7)
    X, T, W = _dev(x), _dev(t), _dev(w)
    losses = [net.train_step(X, T, W, lr=3e-3) for _ in range(60)]
    print(f"fit: loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    assert losses[-1] < 0.5 * losses[0]


def test_encodings_match_oracle():
    import torch
    from paper_2510_22077_gb300 import inputs, pns
    w = inputs.make_workload("tiny3d", n=8, seed=1)
    shape = w.mask.shape
    nc = int(np.prod(shape))
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(4 * nc)
    xn = xs + 0.1 * rng.standard_normal(4 * nc)
    net = pns.UNet(channels=(8,), batch=1, shape=shape)
    mask = torch.as_tensor(w.mask.astype(np.uint8)).cuda()
    f = torch.zeros((1, 6) + shape, dtype=torch.float32, device="cuda")
    tt = torch.zeros((1, 4) + shape, dtype=torch.float32, device="cuda")
    ww = torch.zeros((1, 1) + shape, dtype=torch.float32, device="cuda")
    xs_d = torch.as_tensor(xs).cuda()
    sc = net.features(mask, xs_d, 12.5, f)
    f_o, U, P = ou.features(w.mask, xs, 12.5)
    assert abs(sc[0] - U) <= 1e-15 * U and abs(sc[1] - P) <= 1e-15 * P
    assert _rel(f.cpu().numpy(), f_o) < 1e-6
    net.targets(mask, torch.as_tensor(xn).cuda(), xs_d, sc, tt, ww)
    assert _rel(tt.cpu().numpy(), ou.targets(xn, xs, shape, U, P)) < 1e-6
    assert np.array_equal(ww.cpu().numpy()[0, 0], w.mask.astype(np.float32))
    xo = torch.zeros(4 * nc, dtype=torch.float64, device="cuda")
    net.proposal(tt, xs_d, sc, xo)
    assert _rel(xo.cpu().numpy(), ou.proposal(tt.cpu().numpy().astype(np.float64), xs, shape, U, P)) < 1e-12
