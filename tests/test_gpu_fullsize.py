"""Parity at the full size of the benchmarked workload (96^3 sphere pack, 1.15 M unknowns): the FP64
residual and Jacobian apply element by element against the oracle, the converged solve judged by the
oracle's own residual function (a property that holds at any size), and the converged velocity and
pressure against the oracle's own Newton-FGMRES solve of the same workload on sampled unknowns (stored by
tests/golden/make_spheres96_solve.py, which calls only the oracle; both solved to 1e-12)."""
import json
import os

import numpy as np
import pytest

from gpu_util import problem, random_vector, rel, solver, to_dev
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    return w, mu


def test_residual_and_jacobian_full_size(c2):
    w, mu = c2
    pb = problem(w, mu=mu)
    S = solver(w, mu=mu)
    x = random_vector(pb, seed=3)
    v = random_vector(pb, seed=5)
    assert rel(S.pns_residual(to_dev(x)).cpu().numpy(), pb.residual(x)) < 1e-13
    assert rel(S.pns_jacobian_apply(to_dev(x), to_dev(v)).cpu().numpy(), pb.jacobian(x) @ v) < 1e-13
    S.close()


def test_converged_solve_full_size_by_the_oracle_residual(c2):
    """The bench's solve (Stokes guess, gPLMM, FP32 local inverses, Newton to 1e-8): the oracle's
    residual of the returned state is below 1e-8 of its reference norm."""
    w, mu = c2
    pb = problem(w, mu=mu)
    S = solver(w, mu=mu, variant="gplmm", precision="fp32")
    x, _ = S.pns_stokes_solve()
    S.pns_build_precond(x)
    st = S.pns_newton_solve(x)
    assert st["status"] == "PNS_OK"
    xh = x.cpu().numpy()
    r = np.linalg.norm(pb.residual(xh)) / pb.r0
    print(f"96^3 solve: newton {st['newton_its']} fgmres {st['fgmres_its']} oracle residual {r:.2e}")
    assert r < 1e-8, (r, st)
    S.close()


def test_converged_solution_full_size_matches_oracle_solve(c2):
    """The benchmark's solve (Stokes iterate by aPLMM_S, gPLMM built there, FP32 local inverses) taken to
    ||r|| / ||r(0)|| < 1e-12: its velocity and pressure on 20,000 sampled unknowns match the oracle's solve
    to 1e-8 relative L2, and the FGMRES iteration counts at the benchmark's tolerances equal the oracle's."""
    w, mu = c2
    ref = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spheres96_solve.json")))
    assert abs(mu - ref["mu"]) <= 1e-15 * mu
    S = solver(w, mu=mu, variant="gplmm", precision="fp32")
    x, sst = S.pns_stokes_solve()
    S.pns_build_precond(x)
    st = S.pns_newton_solve(x)
    its = [sst["fgmres_its_total"], st["fgmres_its"]]
    S.close()
    S = solver(w, mu=mu, variant="gplmm", precision="fp32", newton_tol=1e-12, inner_tol=1e-13)
    xs, _ = S.pns_stokes_solve()
    S.pns_build_precond(xs)
    x = xs.clone()
    st2 = S.pns_newton_solve(x)
    S.close()
    idx = np.asarray(ref["idx"])
    xo = np.asarray(ref["x"])
    err = rel(x.cpu().numpy()[idx], xo)
    print(f"96^3 converged solution vs oracle solve: rel L2 {err:.2e} on {len(idx)} samples; FGMRES its "
          f"{its} (oracle {ref['stokes_fgmres_its']}, {ref['newton_fgmres_its']}); refined solve "
          f"{st2['fgmres_its']}")
    assert err < 1e-8
    assert its[0] == sum(ref["stokes_fgmres_its"])
    assert all(abs(a - b) <= 2 for a, b in zip(its[1], ref["newton_fgmres_its"]))
