"""The learned initial guess on the GPU (include/pns_unet.h) against the NumPy oracle of the network
(oracle/unet.py, pinned against torch's conv3d, max-pool, upsampling and Adam and by central
differences): forward, parameter gradients of the masked MSE loss, one Adam step, the sample encodings,
and a short fit.

The library keeps activations, working weights and back-propagated gradients in BF16 and accumulates in
FP32.  Two comparisons:
* against the oracle in FP64 on the same (FP32 master) weights -- the output to 3e-2 relative L2 and
  every gradient tensor to 0.15 (BF16 rounding of every stored tensor, compounded through up to 2L + 6
  layers of back-propagation, with ReLU masks flipping where a pre-activation rounds across zero);
* against the oracle's layer functions run in FP64 with the library's BF16 roundings applied at the same
  points (inputs, weights, every stored activation and gradient) -- 3e-3 on the output and 1e-2 on each
  gradient tensor: what remains is the FP32 accumulation order, through the elements whose BF16 rounding
  or ReLU mask it flips (measured: up to 1.8e-3 and 4.1e-3 on the 4-level network, 20x closer than to the
  FP64 oracle); a wrong tap order, a transposed weight, a missing bias or a dropped skip connection leaves
  an O(1) error in either."""
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


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def emulated(ref, x, t, w):
    """Forward and parameter gradients of the network with the library's BF16 roundings: inputs and weights
    rounded, each convolution accumulated in high precision, biased, rectified and rounded; the head output
    unrounded; the output gradient rounded; data gradients masked by (input > 0) and rounded; the upsampling
    gradient summed and rounded; the pooling gradient added to the skip gradient and rounded."""
    P = {k: (bf16(v) if k.endswith(".w") else v) for k, v in ref.params.items()}
    L = ref.L
    conv = lambda n, a: ou.conv3d(a, P[n + ".w"], ref.params[n + ".b"])
    act = lambda n, a: bf16(np.maximum(conv(n, a), 0.0))
    inp, e0, e1, args, shapes = [bf16(x)], [], [], [], []
    for l in range(L):
        e0.append(act(f"enc{l}.0", inp[l]))
        e1.append(act(f"enc{l}.1", e0[l]))
        if l < L - 1:
            p_, a_ = ou.maxpool2(e1[l])
            args.append(a_)
            shapes.append(e1[l].shape)
            inp.append(p_)
    h = {L - 1: e1[L - 1]}
    cat, d0 = {}, {}
    for l in range(L - 2, -1, -1):
        cat[l] = np.concatenate([ou.upsample2(h[l + 1]), e1[l]], axis=1)
        d0[l] = act(f"dec{l}.0", cat[l])
        h[l] = act(f"dec{l}.1", d0[l])
    out = conv("head", h[0])
    _, gout = ou.masked_mse(out, t, w)
    grads = {}

    def back(n, xin, g, want_dx):
        gx, gw, gb = ou.conv3d_backward(xin, P[n + ".w"], g)
        grads[n + ".w"], grads[n + ".b"] = gw, gb
        return bf16(gx * (xin > 0)) if want_dx else None

    g = back("head", h[0], bf16(gout), True)          # gradient of the pre-activation of h[0]
    g_skip = {}
    for l in range(0, L - 1):
        g = back(f"dec{l}.1", d0[l], g, True)
        gc = back(f"dec{l}.0", cat[l], g, True)
        cu = h[l + 1].shape[1]
        g_skip[l] = gc[:, cu:]
        g = bf16(ou.upsample2_backward(gc[:, :cu]))  # gradient of the pre-activation of h[l + 1]
    g_e1 = {L - 1: g}
    for l in range(L - 1, -1, -1):
        g0 = back(f"enc{l}.1", e0[l], g_e1[l], True)
        gp = back(f"enc{l}.0", inp[l], g0, l > 0)
        if l > 0:
            g_e1[l - 1] = bf16(g_skip[l - 1] + ou.maxpool2_backward(args[l - 1], gp, shapes[l - 1]))
    return out, grads


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
    out_e, grads_e = emulated(ref, x, t, w)
    e_out_e = _rel(out_g, out_e)
    off = 0
    worst_e = 0.0
    for n in names:
        sz = ref.params[n].size
        worst_e = max(worst_e, _rel(gg[off:off + sz], grads_e[n].ravel()))
        off += sz
    print(f"U-Net {channels} {shape} x{batch}: output rel err {e_out:.2e} (FP64 oracle), {e_out_e:.2e} (BF16-rounded "
          f"oracle); gradient rel err worst {worst:.2e} (FP64), {worst_e:.2e} (BF16-rounded) ({', '.join(lines)})")
    assert e_out < 3e-2 and e_out_e < 3e-3
    assert worst < 0.15 and worst_e < 1e-2


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
