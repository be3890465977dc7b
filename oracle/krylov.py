"""Right-preconditioned flexible GMRES, Newton and backward-Euler drivers (Sec. 8; Eq. 3).

* FGMRES(m) (Saad, SIAM J. Sci. Comput. 14, 1993): Arnoldi with modified Gram-Schmidt, Givens
  rotations, x0 = 0.  Stops when the Givens estimate of ||A x - b|| falls below `tol_abs`
  (Sec. 8 normalises by ||r(u=0, p=0)||, so tol_abs = 1e-9 * ||r(0)||); the true residual is
  recomputed at every restart.  Restart m = 100 (the paper does not state one).
* Newton: x <- x + dx with J(x) dx = -r(x) (Eq. 3), until ||r(x)|| / ||r(0)|| < tol, no line search.
* Backward Euler: x^n from x^{n-1} by Newton on the transient residual (Sec. 8.2, fixed dt).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import mac
from .maps import build_maps
from .plmm import Plmm


def fgmres(matvec, precond, b, tol_abs, restart=100, maxit=2000):
    """Solve A x = b.  Returns (x, iterations, final residual estimate)."""
    n = len(b)
    x = np.zeros(n)
    r = b.copy()
    beta = np.linalg.norm(r)
    its = 0
    while beta > tol_abs and its < maxit:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            its += 1
            k = j + 1
            if abs(gvec[j + 1]) <= tol_abs or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), gvec[:k])
        x = x + Z[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
    return x, its, beta


class Problem:
    """Geometry + parameters + maps of one solve."""

    def __init__(self, mask, labels, prm: mac.Params, periodic=(True, False, False), n_dilate=1, n_tag=1,
                 iface_mode="pair", rowsum="all"):
        self.g = mac.Grid(mask, periodic)
        self.prm = prm
        self.rowsum = rowsum
        self.pins = mac.pressure_pins(self.g)
        self.maps = build_maps(self.g, labels, self.pins, n_dilate, n_tag, iface_mode)
        self.r0 = mac.reference_norm(self.g, prm, self.pins)

    def residual(self, x, x_prev=None):
        return mac.residual(self.g, self.prm, x, self.pins, x_prev)

    def jacobian(self, x):
        return mac.assemble(self.g, self.prm, self.pins, "newton", state=x)

    def build_matrix(self, variant, x_lin):
        """A_b of each variant (Sec. 8.1: built before the Newton loop, not during it)."""
        if variant in ("gplmm", "ml_only"):
            return mac.assemble(self.g, self.prm, self.pins, "oseen", wind=x_lin, tags=self.maps.tags)
        if variant == "aplmm_ns":
            return mac.assemble(self.g, self.prm, self.pins, "newton", state=x_lin)
        if variant == "aplmm_s":
            return mac.assemble(self.g, self.prm, self.pins, "stokes")
        raise ValueError(variant)

    def preconditioner(self, variant, x_lin):
        A_b = self.build_matrix(variant, x_lin)
        return Plmm(self.g, self.prm, self.maps, A_b, use_coarse=(variant != "ml_only"), rowsum=self.rowsum), A_b

    def direct_step(self, x, x_prev=None):
        """Newton step with an exact sparse solve (for brute-force checks)."""
        g = self.g
        r = self.residual(x, x_prev)
        J = mac.restrict(g, self.jacobian(x))
        dx = np.zeros(g.nfull)
        dx[g.unknown] = spla.spsolve(J.tocsc(), -r[g.unknown])
        return dx


def newton(pb: Problem, x0, variant="gplmm", combine="build", tol=1e-8, inner_tol=1e-9, restart=100,
           max_newton=30, max_fgmres=2000, x_prev=None, precond=None, log=None):
    """Newton + FGMRES with a PLMM preconditioner built once at x0 (Sec. 4 and 8.1).
    combine = "build": the A of the residual updates inside M (Eqs. 4a, 24) is the build matrix A_b,
    so M is one fixed linear operator made entirely from A_b ("constructed from A set equal to the
    modified Jacobian", Sec. 4); "current": that A is the Newton Jacobian FGMRES is solving.
    Returns (x, stats dict)."""
    x = np.array(x0, dtype=np.float64)
    if precond is None:
        M, A_b = pb.preconditioner(variant, x)
    else:
        M, A_b = precond
    hist, its = [], []
    for k in range(max_newton + 1):
        r = pb.residual(x, x_prev)
        rel = np.linalg.norm(r) / pb.r0
        hist.append(rel)
        if log:
            log(k, rel)
        if rel < tol or k == max_newton:
            break
        J = pb.jacobian(x)
        A_upd = J if combine == "current" else A_b
        dx, n_it, _ = fgmres(lambda v: J @ v, lambda v: M.apply(v, A_upd), -r, inner_tol * pb.r0,
                             restart=restart, maxit=max_fgmres)
        its.append(n_it)
        x = x + dx
    return x, {"newton_its": len(its), "fgmres_its": its, "res_hist": hist, "converged": hist[-1] < tol}


def stokes_solution(pb: Problem, tol=1e-12):
    """Exact Stokes solve (rho = 0 in the inertia; the system is linear, so one Newton step)."""
    g = pb.g
    A = mac.restrict(g, mac.assemble(g, pb.prm, pb.pins, "stokes"))
    x = np.zeros(g.nfull)
    # r(0) for the Stokes operator = -rho b on faces; the transient part vanishes at x = 0
    b = -pb.residual(np.zeros(g.nfull))
    x[g.unknown] = spla.spsolve(A.tocsc(), b[g.unknown])
    return x


def transient(pb: Problem, x_start, n_steps, variant="aplmm_ns", rebuild_every=0, **kw):
    """Backward Euler from x_start (Sec. 8.2).  The preconditioner is built at x_start and reused across
    steps (factors reused); with rebuild_every = k > 0 it is rebuilt at the initial guess of every time
    step that follows k steps solved with the current one (aPLMM_S, which does not depend on the state,
    is never rebuilt).  Returns (list of states, per-step stats)."""
    assert pb.prm.transient
    M = pb.preconditioner(variant, x_start)
    xs = [np.array(x_start)]
    stats = []
    since = 0
    for _ in range(n_steps):
        if rebuild_every > 0 and since >= rebuild_every and variant != "aplmm_s":
            M = pb.preconditioner(variant, xs[-1])
            since = 0
        since += 1
        x, st = newton(pb, xs[-1], variant=variant, x_prev=xs[-1], precond=M, **kw)
        xs.append(x)
        stats.append(st)
    return xs, stats
