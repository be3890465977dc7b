"""Backward Euler through the library over several time steps with one preconditioner build reused
(Sec. 8.2: the aPLMM_NS factors are built once and kept across steps), against the oracle's own
transient driver (oracle/krylov.transient, pinned by the tridiagonal start-up recurrence) on the 64x64
disk pack: every time level, the converged state matches to 1e-8 relative L2 with both sides solved
to 1e-11."""
import numpy as np
import pytest

from gpu_util import problem, rel, solver, to_dev

pytestmark = pytest.mark.gpu

MU, DT, STEPS = 3.87, 0.5, 3


@pytest.fixture(scope="module")
def oracle_levels(c1_workload):
    from oracle import krylov
    pb = problem(c1_workload, mu=MU, dt=DT)
    xs, stats = krylov.transient(pb, np.zeros(pb.g.nfull), STEPS, variant="aplmm_ns", tol=1e-11, inner_tol=1e-12)
    assert all(s["converged"] for s in stats)
    return xs, stats


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_transient_steps_with_reused_preconditioner(c1_workload, oracle_levels, precision):
    xs, stats = oracle_levels
    S = solver(c1_workload, mu=MU, dt=DT, variant="aplmm_ns", precision=precision, newton_tol=1e-11,
               inner_tol=1e-12)
    x_prev = S.zeros()
    S.pns_build_precond(x_prev)               # built once, at the start state, as the oracle's driver does
    its = []
    for n in range(1, STEPS + 1):
        x = x_prev.clone()
        st = S.pns_newton_solve(x, x_prev)
        err = rel(x.cpu().numpy(), xs[n])
        print(f"{precision} step {n}: newton {st['newton_its']} fgmres {st['fgmres_its']} "
              f"(oracle {stats[n - 1]['fgmres_its']}) rel L2 {err:.2e}")
        assert err < 1e-8, (n, err)
        its.append(st["fgmres_its"])
        x_prev = x
    S.close()


def test_transient_rebuild_every_step(c1_workload):
    """rebuild_every = 1: the library rebuilds the aPLMM_NS preconditioner at the initial guess of every
    time step after the first (one build per step in pns_stats.precond_builds), as the oracle's driver does
    with the same policy; every level matches the oracle's to 1e-8."""
    from oracle import krylov
    pb = problem(c1_workload, mu=MU, dt=DT)
    xs, stats = krylov.transient(pb, np.zeros(pb.g.nfull), STEPS, variant="aplmm_ns", rebuild_every=1, tol=1e-11,
                                 inner_tol=1e-12)
    S = solver(c1_workload, mu=MU, dt=DT, variant="aplmm_ns", precision="fp64", newton_tol=1e-11, inner_tol=1e-12,
               rebuild_every=1)
    x_prev = S.zeros()
    S.pns_build_precond(x_prev)
    builds = []
    for n in range(1, STEPS + 1):
        x = x_prev.clone()
        st = S.pns_newton_solve(x, x_prev)
        builds.append(st["precond_builds"])
        err = rel(x.cpu().numpy(), xs[n])
        print(f"rebuild every step, step {n}: builds {st['precond_builds']} fgmres {st['fgmres_its']} "
              f"(oracle {stats[n - 1]['fgmres_its']}) rel L2 {err:.2e}")
        assert err < 1e-8, (n, err)
        x_prev = x
    assert builds == [1, 2, 3]
    S.close()
