"""Writes tests/golden/spheres96_<variant>_apply.json: sampled entries of z = M^{-1} v computed by the
FP64 oracle (oracle/ only) on the 96^3 sphere pack of the benchmark, for the GPU parity tests at full
size (the oracle's build takes minutes, too slow for a test).

Workload: inputs.make_workload("spheres", seed=0, n=96), rho = b_x = 1, mu = Kozeny-Carman for Re = 1.
Variants:
  aplmm_s  build matrix = the Stokes operator (no linearisation state);
  gplmm    build matrix = the modified Jacobian of Eq. 27 at the wind inputs.synthetic_wind(shape,
           seed=31), zeroed off the unknowns.
v is standard normal on the unknowns (numpy default_rng(21), in the order of the oracle's unknown list)
and zero elsewhere.  M is applied with the build matrix in its residual updates (Eqs. 4a, 24).

Sampled outputs (default_rng(22)), each tagged with a group so that a test can report its error per
group: 0-9 = the decile of the size of the unknown's primary grid (all 209 grids contribute up to 12
unknowns each), 10 = 800 unknowns of the largest primary grid, 11 = unknowns on interface faces or in
interface cells (in no primary grid), 12 = 600 unknowns covered by a dual grid.  Takes several minutes
and a few GB of host memory; run one process per variant:
    python tests/golden/make_spheres96_applies.py aplmm_s
    python tests/golden/make_spheres96_applies.py gplmm"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, mac  # noqa: E402
from paper_2510_22077_gb300 import inputs  # noqa: E402

WIND_SEED = 31


def sample(pb, rng):
    """Stratified output indices and their groups (see the module docstring)."""
    m = pb.g, pb.maps
    prim = [np.asarray(P) for P in pb.maps.prim_unknowns]
    sizes = np.array([len(P) for P in prim])
    edges = np.quantile(sizes, np.linspace(0, 1, 11))
    idx, grp = [], []
    for P, n in zip(prim, sizes):
        dec = int(min(9, np.searchsorted(edges, n, side="right") - 1))
        pick = rng.choice(P, size=min(12, len(P)), replace=False)
        idx += pick.tolist()
        grp += [dec] * len(pick)
    big = prim[int(np.argmax(sizes))]
    pick = rng.choice(big, size=min(800, len(big)), replace=False)
    idx += pick.tolist()
    grp += [10] * len(pick)
    in_prim = np.zeros(pb.g.nfull, bool)
    for P in prim:
        in_prim[P] = True
    rest = np.asarray(pb.g.unknown)[~in_prim[pb.g.unknown]]
    pick = rng.choice(rest, size=min(600, len(rest)), replace=False)
    idx += pick.tolist()
    grp += [11] * len(pick)
    dual = np.unique(np.concatenate([np.asarray(D) for D in pb.maps.dual_unknowns]))
    pick = rng.choice(dual, size=min(600, len(dual)), replace=False)
    idx += pick.tolist()
    grp += [12] * len(pick)
    # unique indices, first group kept
    seen, out_i, out_g = set(), [], []
    for i, gq in zip(idx, grp):
        if i not in seen:
            seen.add(i)
            out_i.append(int(i))
            out_g.append(int(gq))
    del m
    return out_i, out_g, [float(e) for e in edges]


def main(variant):
    t0 = time.time()
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)), w.periodic)
    g = pb.g
    v = np.zeros(g.nfull)
    v[g.unknown] = np.random.default_rng(21).standard_normal(len(g.unknown))
    x_lin = None
    if variant == "gplmm":
        x_lin = inputs.synthetic_wind(w.mask.shape, seed=WIND_SEED)
        keep = np.zeros(g.nfull, bool)
        keep[g.unknown] = True
        x_lin[~keep] = 0.0
    M, A_b = pb.preconditioner(variant, x_lin)
    z = M.apply(v, A_b)
    idx, grp, edges = sample(pb, np.random.default_rng(22))
    out = {"workload": "spheres n=96 seed=0, rho=1, b=(1,0,0), mu=Kozeny-Carman(Re=1)", "mu": mu,
           "variant": variant, "wind_seed": WIND_SEED if variant == "gplmm" else None, "v_seed": 21,
           "sample_seed": 22, "n_unknowns": int(len(g.unknown)), "norm_v": float(np.linalg.norm(v)),
           "norm_z": float(np.linalg.norm(z)), "size_decile_edges": edges, "idx": idx, "group": grp,
           "z": [float(z[i]) for i in idx], "seconds": time.time() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"spheres96_{variant}_apply.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["n_unknowns"], len(idx), out["norm_z"], out["seconds"])


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "aplmm_s")
