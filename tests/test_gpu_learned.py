"""The learned Newton initial guess end to end on the GPU, at a small scale: solver-generated samples
(32^3 sphere packs, Re in [1, 100]), training of the U-Net with the library's kernels,
and Newton from the guarded learned start against Newton from the Stokes solution on the same image.

Checks: the training loss falls; the guarded start never has a larger Newton residual than the Stokes
solution (the network's proposal is used only when its residual is smaller); both starts reach the 1e-8
Newton tolerance.  What the network gains (Newton and FGMRES iterations, time) is printed; the benchmark's
learned mode measures it at scale."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_start_end_to_end():
    import torch
    from paper_2510_22077_gb300 import learned, pns
    n = 32
    net = pns.UNet(channels=(16, 32, 64, 64), in_ch=6, out_ch=4, batch=4, shape=(n, n, n), seed=0)
    data = learned.Dataset(net, 8, n=n, seed0=1000, kinds=("spheres",))
    assert data.m == 8
    hist = learned.train(net, data, epochs=150, batch=4, lr=2e-3)
    print(f"samples {data.m} (skipped {data.skipped}) in {data.seconds:.1f} s; loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert hist[-1] < 0.5 * hist[0]
    # guarded start on a training image and on a held-out image
    for seed in (data.meta[0]["seed"], 9000):
        kind = "spheres" if seed % 2 == 0 else "grf"
        w, _ = learned._image(kind, seed, n)
        re = float(np.random.default_rng(seed + 7).uniform(1.0, 100.0))
        r = learned.compare_on(w, re, net, gain=data.gain)
        print(f"image seed {seed} ({kind}, Re {re:.1f}): stokes start newton {r['stokes']['newton_its']} fgmres "
              f"{r['stokes']['fgmres_its']} {r['stokes']['ms']:.0f} ms; learned start (used: "
              f"{r['learned']['used_network']}, residual ratio {r['learned']['residual_ratio']:.3f}) newton "
              f"{r['learned']['newton_its']} fgmres {r['learned']['fgmres_its']} {r['learned']['ms']:.0f} ms")
        assert r["stokes"]["status"] == "PNS_OK" and r["learned"]["status"] == "PNS_OK"
        assert r["learned"]["used_network"] == (r["learned"]["residual_ratio"] < 1.0)
    net.close()
    torch.cuda.synchronize()
