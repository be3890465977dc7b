"""Pins of the oracle's Newton and backward-Euler drivers (Eq. 3, Sec. 8.2) against closed forms and an
independent formulation, never against the drivers themselves:

* transient(): the start-up of channel flow under backward Euler solves, at every step, the textbook 1D
  tridiagonal system (rho/dt + mu T) u^n = rho/dt u^{n-1} + rho b; a channel split into two pores runs
  it through the full preconditioned path (interfaces, dual grids, coarse level) with the
  preconditioner built once and reused, and must reproduce the recurrence step by step.  A driver that
  rebuilt the preconditioner every step, or passed the wrong previous time level, fails here.
* newton(combine="current"): the residual updates inside M (Eqs. 4a, 24) use the Jacobian of the
  current iterate.  M applied that way is compared with the literal matrix product of Eqs. 4a and 24
  with A = J (an independent formulation), the driver is checked to hand M exactly J(x_k), and the
  converged solution is compared with a brute-force sparse Newton solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov, mac, plmm
from paper_2510_22077_gb300 import inputs


def _split_channel(nx=8, ny=6, dt=0.3, rho=1.0, mu=0.4):
    mask = inputs.channel(nx, ny)
    labels = np.where(mask > 0, 1 + (np.arange(nx)[None, None, :] >= nx // 2), 0).astype(np.int32)
    return krylov.Problem(mask, labels, mac.Params(rho, mu, (1.0, 0.0), dt=dt))


def test_transient_driver_reproduces_the_tridiagonal_startup():
    ny, nx = 6, 8
    pb = _split_channel(nx, ny)
    assert pb.maps.n_prim == 2 and pb.maps.n_iface >= 1
    builds = []
    orig = pb.preconditioner

    def counting(variant, x_lin):
        builds.append(None if x_lin is None else np.array(x_lin))
        return orig(variant, x_lin)

    pb.preconditioner = counting
    prm = pb.prm
    T = 2 * np.eye(ny) - np.eye(ny, k=1) - np.eye(ny, k=-1)
    T[0, 0] = T[-1, -1] = 3.0
    K = prm.rho / prm.dt * np.eye(ny) + prm.mu * T
    xs, stats = krylov.transient(pb, np.zeros(pb.g.nfull), 4, variant="aplmm_ns", tol=1e-13, inner_tol=1e-14)
    assert len(builds) == 1 and np.all(builds[0] == 0.0)   # built once, at the start state, and reused
    assert len(xs) == 5 and len(stats) == 4
    u1d = np.zeros(ny)
    for n in range(1, 5):
        u1d = np.linalg.solve(K, prm.rho / prm.dt * u1d + prm.rho * prm.b[0])
        ux = pb.g.split(xs[n])[0][0].reshape(ny, nx)
        assert np.abs(ux - u1d[:, None]).max() < 1e-11 * np.abs(u1d).max(), n
        assert stats[n - 1]["converged"]


def _state(pb, seed=0):
    xs = krylov.stokes_solution(pb)
    rng = np.random.default_rng(seed)
    x = xs.copy()
    x[pb.g.unknown] += 0.1 * np.abs(xs).max() * rng.standard_normal(len(pb.g.unknown))
    return x


@pytest.mark.parametrize("kind,seed,variant", [("tiny2d", 0, "gplmm"), ("tiny2d", 4, "aplmm_s"),
                                               ("tiny3d", 1, "gplmm")])
def test_current_jacobian_apply_equals_literal_form(kind, seed, variant):
    w = inputs.make_workload(kind, seed=seed)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 0.3, (1.0, 0.0, 0.0)))
    if pb.maps.n_iface == 0:
        pytest.skip("fixture has no interface")
    g = pb.g
    M, A_b = pb.preconditioner(variant, _state(pb, 0))
    J = pb.jacobian(_state(pb, 7))            # a different state: J differs from A_b
    Mlit, _, unk = plmm.literal_preconditioner(g, pb.prm, pb.maps, A_b, J)
    rng = np.random.default_rng(2)
    for _ in range(2):
        v = np.zeros(g.nfull)
        v[unk] = rng.standard_normal(len(unk))
        z = M.apply(v, J)
        zl = Mlit @ v[unk]
        assert np.linalg.norm(z[unk] - zl) / np.linalg.norm(zl) < 1e-11
        # and it differs from the build-matrix form by far more than rounding
        zb = M.apply(v, A_b)
        assert np.linalg.norm(zb[unk] - zl) / np.linalg.norm(zl) > 1e-6


def test_newton_current_hands_the_iterate_jacobian_to_m_and_converges():
    w = inputs.make_workload("tiny2d", seed=3)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 0.5, (1.0, 0.0, 0.0)))
    x0 = krylov.stokes_solution(pb)
    M, A_b = pb.preconditioner("gplmm", x0)
    seen = []

    class Spy:
        def apply(self, v, A):
            seen.append(A)
            return M.apply(v, A)

    x, st = krylov.newton(pb, x0, variant="gplmm", combine="current", tol=1e-12, inner_tol=1e-13,
                          precond=(Spy(), A_b))
    assert st["converged"] and st["newton_its"] >= 2
    xd = x0.copy()
    for _ in range(20):
        dx = pb.direct_step(xd)
        xd += dx
        if np.linalg.norm(dx) <= 1e-14 * np.linalg.norm(xd):
            break
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    # the applies of the first step received J(x_0), and none of them the build matrix
    J0 = pb.jacobian(x0)
    assert (seen[0] - J0).count_nonzero() == 0
    assert all((A - A_b).count_nonzero() > 0 for A in seen)   # never the build matrix


def test_transient_driver_passes_the_previous_level():
    """One step from a nonzero start: the backward-Euler residual at the result, with the start as the
    previous level, vanishes; with a zero previous level it does not."""
    pb = _split_channel(dt=0.2)
    xs, _ = krylov.transient(pb, np.zeros(pb.g.nfull), 2, variant="aplmm_ns", tol=1e-13, inner_tol=1e-14)
    r_ok = pb.residual(xs[2], xs[1])
    r_bad = pb.residual(xs[2], None)
    assert np.linalg.norm(r_ok) / pb.r0 < 1e-12
    assert np.linalg.norm(r_bad) / pb.r0 > 1e-3
    # the direct backward-Euler step from xs[1] lands on the same state
    g = pb.g
    x = xs[1].copy()
    for _ in range(6):
        r = pb.residual(x, xs[1])
        J = mac.restrict(g, pb.jacobian(x))
        x[g.unknown] += spla.spsolve(J.tocsc(), -r[g.unknown])
    assert np.linalg.norm(x - xs[2]) / np.linalg.norm(xs[2]) < 1e-11


@pytest.mark.parametrize("variant,every,expect", [("aplmm_ns", 2, [0, 2, 4]), ("aplmm_ns", 1, [0, 1, 2, 3, 4]),
                                                  ("aplmm_ns", 0, [0]), ("aplmm_s", 1, [0])])
def test_transient_rebuild_policy(variant, every, expect):
    """rebuild_every = k: the preconditioner is rebuilt at the initial guess of each time step that follows
    k steps solved with the current one (the previous level, which is also the step's initial iterate);
    0 keeps the start-up build; aPLMM_S (state-independent) is never rebuilt.  The states stay those of the
    tridiagonal recurrence whatever the policy (Newton converges to the same level)."""
    ny, nx = 6, 8
    pb = _split_channel(nx, ny)
    builds = []
    orig = pb.preconditioner

    def counting(v, x_lin):
        builds.append(np.array(x_lin))
        return orig(v, x_lin)

    pb.preconditioner = counting
    xs, stats = krylov.transient(pb, np.zeros(pb.g.nfull), 5, variant=variant, rebuild_every=every, tol=1e-13,
                                 inner_tol=1e-14)
    assert len(builds) == len(expect)
    for b, n in zip(builds, expect):
        assert np.array_equal(b, xs[n]), n
    prm = pb.prm
    T = 2 * np.eye(ny) - np.eye(ny, k=1) - np.eye(ny, k=-1)
    T[0, 0] = T[-1, -1] = 3.0
    K = prm.rho / prm.dt * np.eye(ny) + prm.mu * T
    u1d = np.zeros(ny)
    for n in range(1, 6):
        u1d = np.linalg.solve(K, prm.rho / prm.dt * u1d + prm.rho * prm.b[0])
        ux = pb.g.split(xs[n])[0][0].reshape(ny, nx)
        assert np.abs(ux - u1d[:, None]).max() < 1e-11 * np.abs(u1d).max(), n
