"""Writes tests/golden/spheres96_dilation.json: the FP64 oracle's (oracle/ only) iteration counts on the
benchmark's workload -- the 96^3 sphere pack, rho = b_x = 1, mu = Kozeny-Carman for Re = 1 -- with dual
grids built without dilation (n_dilate = 0), in the steps and with the tolerances of
make_spheres96_solve.py (which uses the default n_dilate = 1): the aPLMM_S Stokes iterate, then gPLMM
built at it and Newton-FGMRES to ||r|| / ||r(0)|| < 1e-8 with the FGMRES tolerance 1e-9 ||r(0)||.
Stores the FGMRES counts, the Newton residual history and the dual grids' coverage of the unknowns.

Takes about a quarter of an hour on a few cores."""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

from make_spheres96_solve import stokes_fgmres  # noqa: E402
from oracle import krylov, mac  # noqa: E402
from paper_2510_22077_gb300 import inputs  # noqa: E402


def main(n_dilate=0):
    t0 = time.time()
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)), w.periodic, n_dilate=n_dilate)
    g = pb.g
    cover = np.zeros(g.nfull, bool)
    for u in pb.maps.dual_unknowns:
        cover[u] = True
    xs, its_s = stokes_fgmres(pb)
    M, A_b = pb.preconditioner("gplmm", xs)
    x, st = krylov.newton(pb, xs, variant="gplmm", tol=1e-8, inner_tol=1e-9, precond=(M, A_b))
    out = {"workload": "spheres n=96 seed=0, rho=1, b=(1,0,0), mu=Kozeny-Carman(Re=1)", "mu": mu,
           "n_dilate": n_dilate, "n_unknowns": int(len(g.unknown)),
           "dual_coverage": float(cover.sum()) / len(g.unknown),
           "dual_overlap": float(sum(len(u) for u in pb.maps.dual_unknowns)) / len(g.unknown),
           "stokes_fgmres_its": [int(i) for i in its_s], "newton_its": st["newton_its"],
           "newton_fgmres_its": [int(i) for i in st["fgmres_its"]], "res_hist": [float(r) for r in st["res_hist"]],
           "seconds": time.time() - t0}
    path = os.path.join(HERE, "spheres96_dilation.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
