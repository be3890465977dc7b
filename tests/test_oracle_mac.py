"""Pins of the oracle's discretisation (Eq. 1, Eq. 3, Sec. 2) against closed forms, finite
differences and textbook recurrences -- never against the oracle itself."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov, mac
from paper_2510_22077_gb300 import inputs


def poiseuille(g, prm, W):
    """Plane Poiseuille flow between no-slip walls at y = 0 and y = W on the MAC grid with the
    ghost-value wall: u(y_j) = rho b / (2 mu) * (y_j (W - y_j) + h^2/4), y_j = j + 1/2, v = w = p = 0.
    The h^2/4 term is the exact discrete correction of the half-cell wall (the second difference of a
    quadratic is exact; the wall row 3 q_0 - q_1 = 2C holds with it)."""
    x = np.zeros(g.nfull)
    yj = g.coord[1] + 0.5
    ux = prm.rho * prm.b[0] / (2 * prm.mu) * (yj * (W - yj) + 0.25)
    x[g.fidx(0, np.arange(g.ncell))] = np.where(g.face_unknown[0], ux, 0.0)
    return x


@pytest.mark.parametrize("dims,periodic", [((1, 6, 8), (True, False, False)), ((4, 5, 6), (True, False, True))])
@pytest.mark.parametrize("rho", [0.5, 1.0, 7.0])
def test_poiseuille_exact(dims, periodic, rho):
    nz, ny, nx = dims
    mask = inputs.channel(nx, ny, nz)
    g = mac.Grid(mask, periodic)
    prm = mac.Params(rho, 0.3, (1.0, 0.0, 0.0))
    pins = mac.pressure_pins(g)
    x = poiseuille(g, prm, ny)
    r = mac.residual(g, prm, x, pins)
    r0 = mac.reference_norm(g, prm, pins)
    assert np.linalg.norm(r) / r0 < 1e-13
    # the inertia vanishes identically, so Newton from zero must land on it for any rho
    pb_prm = mac.Params(prm.rho, prm.mu, prm.b)
    xk = np.zeros(g.nfull)
    for _ in range(8):
        rr = mac.residual(g, pb_prm, xk, pins)
        if np.linalg.norm(rr) / r0 < 1e-14:
            break
        J = mac.restrict(g, mac.assemble(g, pb_prm, pins, "newton", state=xk))
        xk[g.unknown] += spla.spsolve(J.tocsc(), -rr[g.unknown])
    assert np.linalg.norm(xk - x) / np.linalg.norm(x) < 1e-12


def test_divergence_free_solution(c1_workload):
    w = c1_workload
    prm = mac.Params(1.0, 4.0, (1.0, 0.0))
    pb = krylov.Problem(w.mask, w.labels, prm)
    g = pb.g
    x = krylov.stokes_solution(pb)
    for _ in range(6):
        dx = pb.direct_step(x)
        x = x + dx
        if np.linalg.norm(dx) < 1e-13 * np.linalg.norm(x):
            break
    u, p = g.split(x)
    div = np.zeros(g.ncell)
    for a in range(g.dim):
        ih, uh = g.face_at(a, g.nb[a][1])
        div += np.where(uh, u[a][ih], 0.0) - u[a]
    umax = max(np.abs(ua).max() for ua in u)
    # every void cell, the pinned cell included (its row is r = p; the row sum makes it redundant)
    assert np.abs(div[g.void]).max() <= 1e-12 * umax
    assert abs(div[pb.pins[0]]) <= 1e-12 * umax


def _random_state(g, rng, sign):
    x = np.zeros(g.nfull)
    for d in range(g.dim):
        vals = sign * rng.uniform(0.5, 1.5, g.ncell)
        x[g.fidx(d, np.arange(g.ncell))] = np.where(g.face_unknown[d], vals, 0.0)
    x[g.pidx(np.arange(g.ncell))] = np.where(g.void, rng.standard_normal(g.ncell), 0.0)
    return x


@pytest.mark.parametrize("kind", ["tiny2d", "tiny3d"])
@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("dt", [0.0, 0.7])
def test_jacobian_matches_finite_differences(kind, sign, dt):
    w = inputs.make_workload(kind, seed=3)
    g = mac.Grid(w.mask)
    prm = mac.Params(1.3, 0.2, (1.0, 0.2, 0.1), dt)
    pins = mac.pressure_pins(g)
    rng = np.random.default_rng(5)
    x = _random_state(g, rng, sign)        # all |U| well away from 0: no upwind branch flips
    xp = _random_state(g, rng, 1.0) if dt > 0 else None
    v = np.zeros(g.nfull)
    v[g.unknown] = rng.standard_normal(len(g.unknown))
    J = mac.assemble(g, prm, pins, "newton", state=x)
    eps = 1e-6 * np.linalg.norm(x)
    fd = (mac.residual(g, prm, x + eps * v, pins, xp) - mac.residual(g, prm, x - eps * v, pins, xp)) / (2 * eps)
    assert np.linalg.norm(J @ v - fd) / np.linalg.norm(fd) < 1e-7


def test_oseen_matches_modified_residual(c1_workload):
    """J~_w v = r~_w(v) - r~_w(0) (the modified residual of Eq. 27 is linear), and with the wind
    equal to the state and no tags, r~_u(u, p) is the Navier-Stokes residual itself."""
    w = c1_workload
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 0.5, (1.0, 0.0)))
    g = pb.g
    rng = np.random.default_rng(1)
    x = _random_state(g, rng, 1.0)
    x[g.fidx(1, np.arange(g.ncell))] *= rng.choice([-1.0, 1.0], g.ncell)   # mixed branches
    v = np.zeros(g.nfull)
    v[g.unknown] = rng.standard_normal(len(g.unknown))
    for tags in (None, pb.maps.tags):
        Jt = mac.assemble(g, pb.prm, pb.pins, "oseen", wind=x, tags=tags)
        lhs = Jt @ v
        rhs = mac.modified_residual(g, pb.prm, v, pb.pins, x, tags) - mac.modified_residual(g, pb.prm, 0 * v, pb.pins, x, tags)
        assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13
    r_ns = mac.residual(g, pb.prm, x, pb.pins)
    r_mod = mac.modified_residual(g, pb.prm, x, pb.pins, x, None)
    assert np.linalg.norm(r_ns - r_mod) / np.linalg.norm(r_ns) < 1e-14


def test_stokes_limit_is_first_order_in_rho():
    """Body force f = rho b held fixed while rho -> 0: ||x_NS(rho) - x_Stokes|| = O(rho) (slope 1)."""
    w = inputs.make_workload("tiny2d", n=16, seed=1)
    errs, rhos = [], [1e-2, 1e-3, 1e-4, 1e-5]
    f = 0.05
    xs = None
    for rho in rhos:
        pb = krylov.Problem(w.mask, w.labels, mac.Params(rho, 0.2, (f / rho, 0.0)))
        if xs is None:
            xs = krylov.stokes_solution(pb)
        x = xs.copy()
        for _ in range(10):
            dx = pb.direct_step(x)
            x += dx
            if np.linalg.norm(dx) < 1e-15 * np.linalg.norm(x):
                break
        errs.append(np.linalg.norm(x - xs))
    slopes = np.diff(np.log10(errs)) / np.diff(np.log10(rhos))
    assert np.all(np.abs(slopes - 1.0) < 0.1), slopes


def test_stokes_residual_is_linear():
    """With no inertia (Stokes operator) the residual is affine: r(x) = r(0) + A_S x exactly, so one
    Newton step from anywhere solves it (Sec. 2)."""
    w = inputs.make_workload("tiny3d", seed=2)
    g = mac.Grid(w.mask)
    pins = mac.pressure_pins(g)
    prm = mac.Params(1e-300, 0.7, (1e299, 0.0, 0.0))   # rho b = 0.1, inertia scaled by 1e-300
    rng = np.random.default_rng(0)
    x = _random_state(g, rng, 1.0)
    A = mac.assemble(g, prm, pins, "stokes")
    lhs = mac.residual(g, prm, x, pins) - mac.residual(g, prm, 0 * x, pins)
    assert np.linalg.norm(lhs - A @ x) / np.linalg.norm(A @ x) < 1e-14


def test_transient_channel_startup_matches_tridiagonal_recurrence():
    """Start-up of channel flow under backward Euler: every step solves the 1D tridiagonal system
    (rho/dt + mu T) u^n = rho/dt u^{n-1} + rho b, T = tridiag(-1, 2, -1) with the ghost wall rows
    (3 on the wall diagonals).  Compared against numpy's dense solve of that textbook system."""
    ny, nx = 7, 5
    mask = inputs.channel(nx, ny)
    g = mac.Grid(mask)
    prm = mac.Params(1.0, 0.4, (1.0, 0.0), dt=0.3)
    pins = mac.pressure_pins(g)
    T = 2 * np.eye(ny) - np.eye(ny, k=1) - np.eye(ny, k=-1)
    T[0, 0] = T[-1, -1] = 3.0
    K = prm.rho / prm.dt * np.eye(ny) + prm.mu * T
    u1d = np.zeros(ny)
    x = np.zeros(g.nfull)
    for _ in range(4):
        u1d = np.linalg.solve(K, prm.rho / prm.dt * u1d + prm.rho * prm.b[0])
        xn = x.copy()
        for _ in range(4):
            r = mac.residual(g, prm, xn, pins, x)
            J = mac.restrict(g, mac.assemble(g, prm, pins, "newton", state=xn))
            xn[g.unknown] += spla.spsolve(J.tocsc(), -r[g.unknown])
        x = xn
        ux = g.split(x)[0][0].reshape(ny, nx)
        assert np.abs(ux - u1d[:, None]).max() < 1e-12 * np.abs(u1d).max()


def test_steady_state_is_transient_fixed_point(c1_workload):
    w = c1_workload
    prm = mac.Params(1.0, 4.0, (1.0, 0.0))
    pb = krylov.Problem(w.mask, w.labels, prm)
    x = krylov.stokes_solution(pb)
    for _ in range(5):
        x = x + pb.direct_step(x)
    pbt = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 4.0, (1.0, 0.0), dt=0.05))
    r = pbt.residual(x, x)
    assert np.linalg.norm(r) / pbt.r0 < 1e-12


def test_reynolds_calibration(c1_workload):
    w = c1_workload
    pb1 = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 1.0, (1.0, 0.0)))
    ux1 = pb1.g.split(krylov.stokes_solution(pb1))[0][0].reshape(w.mask.shape)
    mu = inputs.mu_for_reynolds(w.mask, ux1, 2.5)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0)))
    ux = pb.g.split(krylov.stokes_solution(pb))[0][0].reshape(w.mask.shape)
    assert abs(inputs.reynolds(w.mask, ux, 1.0, mu) - 2.5) < 1e-10
