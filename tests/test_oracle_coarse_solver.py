"""Pins of the coarse-scale solver (oracle/coarse_solver.py, Sec. 5, Alg. 1) and of the coarse operator
as an approximate solver."""
import numpy as np

from oracle import coarse_solver as cs
from oracle import krylov, mac, plmm
from paper_2510_22077_gb300 import inputs


def _split_channel(W=6, L=12, mu=0.5):
    lab = np.zeros((W, L), int)
    lab[:, :L // 2] = 1
    lab[:, L // 2:] = 2
    mask = (lab > 0).astype(np.uint8)[None]
    return krylov.Problem(mask, lab[None].astype(np.int32), mac.Params(1.0, mu, (1.0, 0.0)), (True, False, False))


def test_coarse_operator_reproduces_poiseuille_in_a_split_channel():
    """A straight channel cut into two pores: fully developed Poiseuille flow satisfies the closure
    (constant pressure, zero normal derivative of the velocity) exactly at the interface, so one
    application of M_G = P^ (R^ A P^)^{-1} R^ to the Stokes right-hand side is the exact solution,
    u_j = (rho b / 2 mu) (y_j (W - y_j) + 1/4), p = 0."""
    W, mu = 6, 0.5
    pb = _split_channel(W=W, mu=mu)
    g = pb.g
    A = mac.assemble(g, pb.prm, pb.pins, "stokes")
    M = plmm.Plmm(g, pb.prm, pb.maps, A)
    b = -cs.modified_residual(pb, np.zeros(g.nfull), stokes=True)
    x = M.coarse(b)
    y = np.arange(W) + 0.5
    exact = (1.0 / (2 * mu)) * (y * (W - y) + 0.25)
    u = x[:g.ncell].reshape(W, -1)
    assert np.allclose(u, exact[:, None], rtol=1e-12, atol=1e-12)
    assert np.allclose(x[2 * g.ncell:], 0.0, atol=1e-12)


def test_stokes_coarse_newton_is_one_step_of_the_coarse_operator():
    """Remark 2: without inertia, Alg. 1 converges in one Newton iteration and its solution equals
    P^ (R^ A P^)^{-1} R^ b."""
    w = inputs.make_workload("disks64", seed=0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 3.87, (1.0, 0.0, 0.0)), w.periodic)
    x, hist, M = cs.coarse_newton(pb, np.zeros(pb.g.nfull), np.zeros(pb.g.nfull), stokes=True)
    b = -cs.modified_residual(pb, np.zeros(pb.g.nfull), stokes=True)
    assert len(hist) == 2 and hist[1] < 1e-12
    assert np.linalg.norm(x - M.coarse(b)) <= 1e-12 * np.linalg.norm(x)


def test_navier_stokes_coarse_newton_converges():
    """Alg. 1 on the 64x64 disk pack at Re ~ 1 with two body-force increments: the coarse residual
    falls below 1e-6 of its start in each increment."""
    w = inputs.make_workload("disks64", seed=0)
    x, hists = cs.coarse_solver(w.mask, w.labels, 3.8746364606724244, (1.0, 0.0, 0.0), [0.5, 1.0], w.periodic)
    assert all(h[-1] < 1e-6 for h in hists), [h[-1] for h in hists]
    assert np.all(np.isfinite(x))
