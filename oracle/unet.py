"""3D U-Net of the learned Newton initial guess: plain NumPy forward and explicit backward (FP64 by
default).  Test infrastructure.

The network maps the solid mask, the Stokes solution and the Reynolds number of an image to a
correction of the Stokes solution towards the Navier-Stokes solution; Newton then starts from the
corrected state, and keeps the plain Stokes guess when the proposal's residual is not smaller.  The
paper has no such network (it only notes that the initial guess is Newton's weak point, Sec. 9.4); the
architecture is the one this build specifies:

* levels L (default 4) with channels c_0..c_{L-1} (default 16, 32, 64, 64);
* encoder level l: two 3x3x3 convolutions (zero padding 1, bias) each followed by ReLU; between
  levels a 2x2x2 max-pool;
* decoder level l < L-1: nearest 2x upsampling of level l+1's output, concatenated (upsampled first,
  skip second) with the encoder output of level l, then two 3x3x3 convolutions with ReLU;
* head: a 1x1x1 convolution to the output channels, no activation.

Arrays are (N, C, D, H, W).  Max-pool ties go to the first element in (dz, dy, dx) order.

Input encoding (`features`): 6 channels -- void mask, Stokes u_x, u_y, u_z (face arrays in the low-face
convention, image-shaped), Stokes p, log10 Re -- velocities divided by U = max |u_Stokes|, pressure by
P = max |p_Stokes| (or 1 when zero).  Target encoding (`targets`): the NS - Stokes difference with the
same scales, 4 channels.  Both are readings of this build.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------------------------
# layers
# ----------------------------------------------------------------------------------------------
def conv3d(x, w, b):
    """y[n, o] = b[o] + sum_{c, dz, dy, dx} w[o, c, dz, dy, dx] x_pad[n, c, z+dz, y+dy, x+dx]; kernel 3 with
    zero padding 1, or kernel 1 with no padding."""
    k = w.shape[2]
    p = k // 2
    N, C, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p), (p, p)))
    y = np.zeros((N, w.shape[0], D, H, W), dtype=x.dtype)
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                y += np.einsum("oc,nczyx->nozyx", w[:, :, dz, dy, dx], xp[:, :, dz:dz + D, dy:dy + H, dx:dx + W])
    return y + b[None, :, None, None, None]


def conv3d_backward(x, w, gy):
    """Gradients of conv3d with respect to x, w and b, given gy = dL/dy."""
    k = w.shape[2]
    p = k // 2
    N, C, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p), (p, p)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                win = (slice(None), slice(None), slice(dz, dz + D), slice(dy, dy + H), slice(dx, dx + W))
                gw[:, :, dz, dy, dx] = np.einsum("nozyx,nczyx->oc", gy, xp[win])
                gxp[win] += np.einsum("oc,nozyx->nczyx", w[:, :, dz, dy, dx], gy)
    gx = gxp[:, :, p:p + D, p:p + H, p:p + W]
    gb = gy.sum(axis=(0, 2, 3, 4))
    return gx, gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, gy):
    return gy * (x > 0.0)


def maxpool2(x):
    """2x2x2 max-pool; returns the output and the argmax (0..7 in (dz, dy, dx) order, first on ties)."""
    N, C, D, H, W = x.shape
    v = x.reshape(N, C, D // 2, 2, H // 2, 2, W // 2, 2).transpose(0, 1, 2, 4, 6, 3, 5, 7)
    v = v.reshape(N, C, D // 2, H // 2, W // 2, 8)
    arg = np.argmax(v, axis=-1)
    return np.take_along_axis(v, arg[..., None], axis=-1)[..., 0], arg


def maxpool2_backward(arg, gy, shape):
    N, C, D, H, W = shape
    g = np.zeros((N, C, D // 2, H // 2, W // 2, 8), dtype=gy.dtype)
    np.put_along_axis(g, arg[..., None], gy[..., None], axis=-1)
    g = g.reshape(N, C, D // 2, H // 2, W // 2, 2, 2, 2).transpose(0, 1, 2, 5, 3, 6, 4, 7)
    return g.reshape(shape)


def upsample2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)


def upsample2_backward(gy):
    N, C, D, H, W = gy.shape
    return gy.reshape(N, C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(3, 5, 7))


# ----------------------------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------------------------
class UNet:
    def __init__(self, channels=(16, 32, 64, 64), in_ch=6, out_ch=4, seed=0, dtype=np.float64):
        self.ch = tuple(channels)
        self.L = len(channels)
        rng = np.random.default_rng(seed)
        self.params = {}

        def conv(name, ci, co, k=3):
            std = np.sqrt(2.0 / (ci * k ** 3))          # He initialisation for ReLU layers
            self.params[name + ".w"] = (std * rng.standard_normal((co, ci, k, k, k))).astype(dtype)
            self.params[name + ".b"] = np.zeros(co, dtype)

        prev = in_ch
        for l, c in enumerate(self.ch):
            conv(f"enc{l}.0", prev, c)
            conv(f"enc{l}.1", c, c)
            prev = c
        for l in range(self.L - 2, -1, -1):
            conv(f"dec{l}.0", self.ch[l + 1] + self.ch[l], self.ch[l])
            conv(f"dec{l}.1", self.ch[l], self.ch[l])
        conv("head", self.ch[0], out_ch, k=1)

    def n_params(self):
        return int(sum(v.size for v in self.params.values()))

    def _conv(self, name, x, cache):
        y = conv3d(x, self.params[name + ".w"], self.params[name + ".b"])
        cache.append(("conv", name, x))
        return y

    def _conv_relu(self, name, x, cache):
        y = self._conv(name, x, cache)
        cache.append(("relu", y))
        return relu(y)

    def forward(self, x):
        """Returns (output, cache for backward)."""
        cache = []
        skips = []
        h = x
        for l in range(self.L):
            h = self._conv_relu(f"enc{l}.0", h, cache)
            h = self._conv_relu(f"enc{l}.1", h, cache)
            if l < self.L - 1:
                skips.append(h)
                shape = h.shape
                h, arg = maxpool2(h)
                cache.append(("pool", arg, shape, l))
        for l in range(self.L - 2, -1, -1):
            up = upsample2(h)
            cache.append(("cat", up.shape[1]))
            h = np.concatenate([up, skips[l]], axis=1)
            h = self._conv_relu(f"dec{l}.0", h, cache)
            h = self._conv_relu(f"dec{l}.1", h, cache)
        out = self._conv("head", h, cache)
        return out, cache

    def backward(self, cache, gout):
        """Gradients of a scalar loss with respect to every parameter and to the input, given
        gout = dL/d(output).  Returns (grads dict, dL/dx)."""
        grads = {k: np.zeros_like(v) for k, v in self.params.items()}
        g = gout
        skip_grads = {}
        dec_levels = list(range(self.L - 2, -1, -1))
        n_cat = len(dec_levels)
        for item in reversed(cache):
            kind = item[0]
            if kind == "conv":
                _, name, x = item
                gx, gw, gb = conv3d_backward(x, self.params[name + ".w"], g)
                grads[name + ".w"] += gw
                grads[name + ".b"] += gb
                g = gx
            elif kind == "relu":
                g = relu_backward(item[1], g)
            elif kind == "cat":
                n_cat -= 1
                c_up = item[1]
                skip_grads[dec_levels[n_cat]] = g[:, c_up:]
                g = upsample2_backward(g[:, :c_up])
            elif kind == "pool":
                _, arg, shape, lvl = item
                # the pooled tensor was also the skip of this encoder level
                g = maxpool2_backward(arg, g, shape) + skip_grads.pop(lvl)
        return grads, g


# ----------------------------------------------------------------------------------------------
# encoding of samples
# ----------------------------------------------------------------------------------------------
def _split(x, shape):
    nz, ny, nx = shape
    n = nz * ny * nx
    return [x[k * n:(k + 1) * n].reshape(shape) for k in range(4)]


def features(mask, x_stokes, re):
    """6-channel input (1, 6, nz, ny, nx) of a 3D image from its Stokes solution (full layout)."""
    shape = mask.shape
    u, v, w, p = _split(np.asarray(x_stokes, np.float64), shape)
    U = max(float(np.abs(np.concatenate([u.ravel(), v.ravel(), w.ravel()])).max()), 1e-300)
    P = float(np.abs(p).max()) or 1.0
    f = np.stack([np.asarray(mask, np.float64), u / U, v / U, w / U, p / P,
                  np.full(shape, np.log10(re))])
    return f[None], U, P


def targets(x_ns, x_stokes, shape, U, P):
    """4-channel target (1, 4, nz, ny, nx): (NS - Stokes) / (U, U, U, P)."""
    d = _split(np.asarray(x_ns, np.float64) - np.asarray(x_stokes, np.float64), shape)
    return np.stack([d[0] / U, d[1] / U, d[2] / U, d[3] / P])[None]


def proposal(out, x_stokes, shape, U, P):
    """Full-layout initial iterate from the network output: Stokes + decoded correction (entries that
    are not unknowns are left for the caller to zero)."""
    o = out[0]
    corr = np.concatenate([(o[0] * U).ravel(), (o[1] * U).ravel(), (o[2] * U).ravel(), (o[3] * P).ravel()])
    return np.asarray(x_stokes, np.float64) + corr


# ----------------------------------------------------------------------------------------------
# training
# ----------------------------------------------------------------------------------------------
def masked_mse(out, target, weight):
    """L = sum(weight * (out - target)^2) / sum(weight) over every channel; returns (L, dL/dout).
    `weight` (N, 1, D, H, W) restricts the loss to the cells that carry unknowns (1 on void, 0 solid)."""
    w = np.broadcast_to(weight, out.shape)
    den = float(w.sum())
    d = out - target
    return float((w * d * d).sum() / den), 2.0 * w * d / den


class Adam:
    """Adam (Kingma & Ba, 2015) with the bias-corrected moments:
    m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,  theta <- theta - lr m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g * g
            params[k] -= self.lr * (self.m[k] / c1) / (np.sqrt(self.v[k] / c2) + self.eps)
