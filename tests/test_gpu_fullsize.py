"""Parity at the full size of the benchmarked workload (96^3 sphere pack, 1.15 M unknowns): the FP64
residual and Jacobian apply element by element against the oracle, and the converged solve judged by
the oracle's own residual function (a property that holds at any size; the oracle's direct solve is
out of reach at this size)."""
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
