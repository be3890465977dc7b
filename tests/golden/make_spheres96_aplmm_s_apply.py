"""Writes tests/golden/spheres96_aplmm_s_apply.json: sampled entries of z = M^{-1} v computed by the FP64
oracle (oracle/ only) for the aPLMM_S preconditioner on the 96^3 sphere pack of the benchmark.

Workload: inputs.make_workload("spheres", seed=0, n=96), rho = b_x = 1, mu = Kozeny-Carman for Re = 1.
aPLMM_S's build matrix is the Stokes operator, so no linearisation state is involved.  v is standard
normal on the unknowns (numpy default_rng(21), in the order of the oracle's unknown list) and zero
elsewhere.  Stored: 4000 sampled unknown indices (default_rng(22)), z there, and the norms of v and z.
Takes a few minutes and a few GB of host memory."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, mac  # noqa: E402
from paper_2510_22077_gb300 import inputs  # noqa: E402


def main():
    t0 = time.time()
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)), w.periodic)
    g = pb.g
    v = np.zeros(g.nfull)
    v[g.unknown] = np.random.default_rng(21).standard_normal(len(g.unknown))
    M, A_b = pb.preconditioner("aplmm_s", None)
    z = M.apply(v, A_b)
    idx = np.sort(np.random.default_rng(22).choice(g.unknown, size=4000, replace=False))
    out = {"workload": "spheres n=96 seed=0, rho=1, b=(1,0,0), mu=Kozeny-Carman(Re=1)", "mu": mu,
           "variant": "aplmm_s", "v_seed": 21, "sample_seed": 22, "n_unknowns": int(len(g.unknown)),
           "norm_v": float(np.linalg.norm(v)), "norm_z": float(np.linalg.norm(z)),
           "idx": [int(i) for i in idx], "z": [float(x) for x in z[idx]],
           "seconds": time.time() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spheres96_aplmm_s_apply.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["n_unknowns"], out["norm_z"], out["seconds"])


if __name__ == "__main__":
    main()
