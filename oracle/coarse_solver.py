"""Coarse-scale solver of the steady Navier-Stokes equations (Sec. 5, Alg. 1): Newton on the coarse
unknowns only, with the prolongation P^ and restriction R^ of the gPLMM coarse level.  Test
infrastructure.

  r_c = R^ r~(x),   J_c = R^ J~(x) P^,   J_c d = -r_c,   x <- x + P^ d,   until |r_c| / |r_c^0| < tol

r~ and J~ are the Navier-Stokes residual and Newton Jacobian with the inertia removed on the tagged
faces near contact interfaces (the modified residual of Eq. 27 with the wind equal to the iterate).
P^ and R^ are built once per Reynolds increment, from the modified Jacobian J~_w with the wind w of the
previous increment (zero at the first).  The outer loop raises the Reynolds number; here it is raised
through the body force (the paper raises the inlet pressure; this build drives the flow by b).

With stokes=True the equations have no inertia: then one Newton step gives x = P^ (R^ A P^)^{-1} R^ b,
the single application of the coarse preconditioner (Remark 2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mac
from .krylov import Problem
from .plmm import Plmm


def _tag_vector(pb):
    g = pb.g
    t = np.zeros(g.nfull)
    for d in range(g.dim):
        t[d * g.ncell:(d + 1) * g.ncell] = pb.maps.tags[d]
    return t


def modified_residual(pb, x, stokes=False):
    g = pb.g
    tags = [np.ones(g.ncell, bool) for _ in range(g.dim)] if stokes else pb.maps.tags
    return mac.modified_residual(g, pb.prm, x, pb.pins, wind=x, tags=tags)


def modified_jacobian(pb, x, stokes=False):
    """Newton Jacobian on untagged face rows, inertia-free rows on tagged faces (all rows if stokes)."""
    Js = mac.assemble(pb.g, pb.prm, pb.pins, "stokes")
    if stokes:
        return Js.tocsr()
    Jn = mac.assemble(pb.g, pb.prm, pb.pins, "newton", state=x)
    T = sp.diags(_tag_vector(pb))
    return (T @ Js + (sp.identity(pb.g.nfull) - T) @ Jn).tocsr()


def back_substitute_f(pb, x, stokes=False):
    """Eq. 8: the interface-face (f) unknowns from their own rows with everything else fixed,
    x_f <- x_f - (J~_ff)^{-1} r~_f(x).  The f faces are tagged, so their rows carry no inertia and are
    linear: one solve makes them exact."""
    f = np.asarray(pb.maps.f_faces, np.int64)
    if f.size == 0:
        return x
    J = modified_jacobian(pb, x, stokes)
    r = modified_residual(pb, x, stokes)
    x = x.copy()
    x[f] -= spla.spsolve(J[f][:, f].tocsc(), r[f])
    return x


def coarse_newton(pb, x0, wind, kmax=30, tol=1e-6, stokes=False):
    """One Reynolds increment of Alg. 1.  Returns (x, relative coarse-residual history, coarse
    level).  P^ leaves the interface faces untouched (they keep x0's values)."""
    A_b = pb.build_matrix("gplmm", wind)
    M = Plmm(pb.g, pb.prm, pb.maps, A_b)
    x = np.array(x0, dtype=np.float64)
    rc = M.Rhat @ modified_residual(pb, x, stokes)
    r0 = float(np.linalg.norm(rc))
    hist = [1.0]
    if r0 == 0.0:
        return x, hist, M
    for _ in range(kmax):
        Jc = (M.Rhat @ modified_jacobian(pb, x, stokes) @ M.Phat).toarray()
        x = x + M.Phat @ np.linalg.solve(Jc, -rc)
        rc = M.Rhat @ modified_residual(pb, x, stokes)
        hist.append(float(np.linalg.norm(rc)) / r0)
        if hist[-1] < tol:
            break
    return x, hist, M


def coarse_solver(mask, labels, mu, b, scales, periodic=(True, False, False), rho=1.0, kmax=30, tol=1e-6):
    """Alg. 1: for each scale s (ascending), the body force s*b; the wind of each increment is the
    velocity of the previous one.  Returns (x, histories)."""
    x = None
    w = None
    hists = []
    for s in scales:
        pb = Problem(mask, labels, mac.Params(rho, mu, tuple(s * np.asarray(b, float)), 0.0), periodic)
        if x is None:
            x = np.zeros(pb.g.nfull)
            w = np.zeros(pb.g.nfull)
        x, hist, _ = coarse_newton(pb, x, w, kmax, tol)
        hists.append(hist)
        w = x.copy()
    return x, hists
