"""The learned Newton initial guess, end to end on the GPU: solver-generated samples, training of the 3D
U-Net (pns.UNet: BF16 tensor-core kernels, Adam on FP32 master weights), and the guarded initial iterate.

Every numerical step runs in libpns (the solver of include/pns.h and the network of include/pns_unet.h);
this module only sequences the calls.

* Samples: seeded synthetic images (sphere packs with porosity U[0.30, 0.45] and thresholded Gaussian
  fields with porosity U[0.20, 0.40], alternating, or sphere packs only), Re drawn uniformly in
  [re_min, re_max], mu from the
  Kozeny-Carman estimate; the Stokes solution (the method's own initial iterate) and the Navier-Stokes
  solution by gPLMM Newton-FGMRES.  Inputs are the encoded (mask, Stokes, log10 Re) channels, targets the
  scaled NS - Stokes difference, the loss weight the void mask.  Images whose solve fails (an iteration
  cap, a singular closure block of the labelling) are skipped and counted.
* Training: minibatches of `batch` samples, masked MSE, Adam.  The network learns the targets scaled by
  one gain per channel (the reciprocal of the channel's RMS over the void cells of the training set), so
  that every channel is O(1); the proposal divides the gains out again.
* Guarded start: the network proposes x_p = Stokes + decoded correction; Newton starts from x_p only if
  ||r(x_p)|| < ||r(x_Stokes)|| (the Newton residual judges the proposal), else from the Stokes solution.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, pns


def _image(kind, seed, n):
    rng = np.random.default_rng(seed)
    if kind == "spheres":
        phi = float(rng.uniform(0.30, 0.45))
        target = max(8, int(round(200 * (n / 96) ** 3)))
        return inputs.make_workload("spheres", seed=seed, n=n, porosity=phi, target=target), phi
    phi = float(rng.uniform(0.20, 0.40))
    target = max(8, int(round(200 * (n / 96) ** 3)))
    return inputs.make_workload("grf", seed=seed, n=n, porosity=phi, target=target), phi


def solve_pair(w, re, precision="fp32", newton_tol=1e-8):
    """Stokes and Navier-Stokes solutions of an image at Reynolds number ~re (device FP64 full layout).
    Returns (solver, x_stokes, x_ns, stats) or None when a solve fails."""
    import torch
    mu = inputs.mu_kozeny_carman(w.mask, re)
    try:
        S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant="gplmm", precision=precision,
                       newton_tol=newton_tol, max_newton=15, max_fgmres=600)
    except pns.PnsError:
        return None
    try:
        xs, _ = S.pns_stokes_solve()
        x = xs.clone()
        S.pns_build_precond(xs)
        st = S.pns_newton_solve(x, check=False)
    except pns.PnsError:
        S.close()
        return None
    if st["status"] != "PNS_OK" or not torch.isfinite(x).all():
        S.close()
        return None
    return S, xs, x, st


class Dataset:
    """Encoded samples held on the device: x (M, 6, n, n, n), t (M, 4, ...), w (M, 1, ...), FP32."""

    def __init__(self, net: pns.UNet, n_samples, n=64, seed0=1000, re_min=1.0, re_max=100.0, log=None,
                 kinds=("spheres", "grf")):
        import torch
        self.n = n
        self.x = torch.zeros((n_samples, 6, n, n, n), dtype=torch.float32, device="cuda")
        self.t = torch.zeros((n_samples, 4, n, n, n), dtype=torch.float32, device="cuda")
        self.w = torch.zeros((n_samples, 1, n, n, n), dtype=torch.float32, device="cuda")
        self.meta = []
        self.skipped = 0
        t0 = time.time()
        k = 0
        seed = seed0
        while k < n_samples and seed < seed0 + 4 * n_samples:
            kind = kinds[seed % len(kinds)]
            re = float(np.random.default_rng(seed + 7).uniform(re_min, re_max))
            seed += 1
            try:
                w, phi = _image(kind, seed - 1, n)
            except (ValueError, ZeroDivisionError):
                w = None
            # an image without a void path along x (possible for a small Gaussian field) has no flow
            r = solve_pair(w, re) if w is not None and w.mask.any() else None
            if r is None:
                self.skipped += 1
                continue
            S, xs, xn, st = r
            mask = torch.as_tensor(w.mask.astype(np.uint8)).cuda()
            sc = net.features(mask, xs, re, self.x, k)
            net.targets(mask, xn, xs, sc, self.t, self.w, k)
            self.meta.append({"kind": kind, "seed": seed - 1, "phi": phi, "re": re, "newton_its": st["newton_its"]})
            S.close()
            k += 1
            if log:
                log(f"sample {k}/{n_samples} ({kind}, Re {re:.1f}, newton {st['newton_its']}) "
                    f"{time.time() - t0:.0f} s")
        self.m = k
        # per-channel gains: the targets are trained at unit RMS over the void cells
        self.gain = torch.ones(4, dtype=torch.float32, device="cuda")
        if k:
            wsum = self.w[:k].sum()
            for c in range(4):
                rms = torch.sqrt((self.w[:k, 0] * self.t[:k, c] ** 2).sum() / wsum)
                if float(rms) > 0:
                    self.gain[c] = 1.0 / rms
            self.t[:k] *= self.gain.view(1, 4, 1, 1, 1)
        self.seconds = time.time() - t0


def train(net: pns.UNet, data: Dataset, epochs=20, batch=4, lr=1e-3, seed=0, log=None):
    """Adam on minibatches of the dataset; returns the mean loss of each epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(data.m)
        ls = []
        for b0 in range(0, data.m - batch + 1, batch):
            idx = order[b0:b0 + batch]
            import torch
            ii = torch.as_tensor(idx, device="cuda")
            ls.append(net.train_step(data.x[ii].contiguous(), data.t[ii].contiguous(), data.w[ii].contiguous(), lr))
        hist.append(float(np.mean(ls)) if ls else float("nan"))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4e}")
    return hist


def guarded_start(S: pns.Solver, net: pns.UNet, mask, re, xs, gain=None):
    """The initial Newton iterate: the network's proposal if its Newton residual is below the Stokes
    solution's, else the Stokes solution.  `gain` (4 channels) is the target scaling the network was trained
    with.  Returns (x0, used_network, ||r(x_p)|| / ||r(x_s)||)."""
    import torch
    nz, ny, nx = mask.shape
    f = torch.zeros((1, 6, nz, ny, nx), dtype=torch.float32, device="cuda")
    m = torch.as_tensor(mask.astype(np.uint8)).cuda()
    sc = net.features(m, xs, re, f)
    out = net.forward(f)
    if gain is not None:
        out = (out / gain.view(1, 4, 1, 1, 1)).contiguous()
    xp = torch.zeros_like(xs)
    net.proposal(out, xs, sc, xp)
    rp = float(S.pns_residual(xp).norm())
    rs = float(S.pns_residual(xs).norm())
    if rp < rs:
        return xp, True, rp / rs
    return xs.clone(), False, rp / rs


def compare_on(w, re, net: pns.UNet, precision="fp32", gain=None):
    """Newton from the Stokes solution and from the guarded learned start on one image: Newton iterations,
    FGMRES iterations and the time of each (CUDA events on the solver's stream; the Stokes solve and the
    network inference are counted in the learned path's time, the Stokes solve in both)."""
    import torch
    mu = inputs.mu_kozeny_carman(w.mask, re)
    out = {}
    for mode in ("stokes", "learned"):
        S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant="gplmm", precision=precision)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(S.stream)
        xs, _ = S.pns_stokes_solve()
        ratio, used = None, False
        if mode == "learned":
            x, used, ratio = guarded_start(S, net, w.mask, re, xs, gain)
        else:
            x = xs.clone()
        S.pns_build_precond(x)
        st = S.pns_newton_solve(x, check=False)
        e1.record(S.stream)
        torch.cuda.synchronize()
        out[mode] = {"ms": e0.elapsed_time(e1), "status": st["status"], "newton_its": st["newton_its"],
                     "fgmres_its": st["fgmres_its"], "used_network": used, "residual_ratio": ratio}
        S.close()
    return out
