"""Writes tests/golden/spheres96_solve.json: the FP64 oracle's (oracle/ only) solve of the benchmark's
workload -- the 96^3 sphere pack, rho = b_x = 1, mu = Kozeny-Carman for Re = 1 -- in the benchmark's
steps, with the benchmark's tolerances, then refined:

1. Stokes initial iterate: FGMRES on the Stokes system (inertia dropped, rho b kept) with the aPLMM_S
   preconditioner, from zero, to ||A x - b|| < 1e-9 ||r(0)||, as a Newton solve of the linear system
   until ||r(x)|| / ||r(0)|| < 1e-8 (Sec. 4: the Stokes solution is the initial Newton iterate).
2. gPLMM built at that iterate (wind = its velocity), Newton-FGMRES to ||r|| / ||r(0)|| < 1e-8 with the
   FGMRES tolerance 1e-9 ||r(0)|| (Sec. 8): the FGMRES iteration counts of both solves are stored.
3. Newton continued from there with the same preconditioner to 1e-12 (FGMRES tolerance 1e-13), and
   sampled entries of that converged state stored (default_rng(41), 20000 unknowns) with its norm.

Takes tens of minutes on one core and several GB of host memory."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, mac  # noqa: E402
from paper_2510_22077_gb300 import inputs  # noqa: E402


def stokes_fgmres(pb, tol=1e-8, inner_tol=1e-9):
    """Newton on the (linear) Stokes residual r_s(x) = A_s x + r(0) with FGMRES and aPLMM_S, from zero:
    returns (x, FGMRES iterations per step)."""
    g = pb.g
    M, A_s = pb.preconditioner("aplmm_s", None)
    r_zero = pb.residual(np.zeros(g.nfull))      # -rho b on the face unknowns, 0 on the cells
    x = np.zeros(g.nfull)
    its = []
    for _ in range(3):
        r = A_s @ x + r_zero
        if np.linalg.norm(r) / pb.r0 < tol:
            break
        dx, n_it, _ = krylov.fgmres(lambda v: A_s @ v, lambda v: M.apply(v, A_s), -r, inner_tol * pb.r0)
        its.append(n_it)
        x = x + dx
    return x, its


def main():
    t0 = time.time()
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)), w.periodic)
    g = pb.g
    xs, its_s = stokes_fgmres(pb)
    t_stokes = time.time() - t0
    print("stokes", its_s, t_stokes, flush=True)
    t1 = time.time()
    M, A_b = pb.preconditioner("gplmm", xs)
    x, st = krylov.newton(pb, xs, variant="gplmm", tol=1e-8, inner_tol=1e-9, precond=(M, A_b))
    t_newton = time.time() - t1
    print("newton", st, t_newton, flush=True)
    x2, st2 = krylov.newton(pb, x, variant="gplmm", tol=1e-12, inner_tol=1e-13, precond=(M, A_b))
    print("refined", st2, flush=True)
    idx = np.sort(np.random.default_rng(41).choice(g.unknown, size=20000, replace=False))
    out = {"workload": "spheres n=96 seed=0, rho=1, b=(1,0,0), mu=Kozeny-Carman(Re=1)", "mu": mu,
           "n_unknowns": int(len(g.unknown)),
           "stokes_fgmres_its": its_s, "newton_its": st["newton_its"], "newton_fgmres_its": st["fgmres_its"],
           "res_hist": st["res_hist"], "refined_res_hist": st2["res_hist"], "refined_fgmres_its": st2["fgmres_its"],
           "norm_x": float(np.linalg.norm(x2)), "sample_seed": 41, "idx": [int(i) for i in idx],
           "x": [float(x2[i]) for i in idx], "seconds_stokes": t_stokes, "seconds_newton": t_newton,
           "seconds": time.time() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spheres96_solve.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["seconds"])


if __name__ == "__main__":
    main()
