"""Block-triangular Schur-complement preconditioner with the scaled BFBt approximation: the comparator
of the monolithic preconditioners (Sec. 1, the block form M_B and Eq. 4).  Test infrastructure.

Over the unknowns ordered [faces | cells] the Jacobian is J = [[F, B1], [B2, C]]:
F the velocity block, B1 the pressure-gradient columns, B2 the divergence rows, C = 0 except on the
pinned cells, whose rows read r = p (B2 zero there, C = 1).  The preconditioner is

    M_B = [[F, B1], [0, X]],   M_B^{-1} [v_u; v_p] = [F^{-1} (v_u - B1 y); y],   y = X^{-1} v_p,

applied on the right.  On pinned cells X = 1 (y = v_p).  On the other cells X approximates the Schur
complement S = -B2 F^{-1} B1 through the scaled BFBt form of Eq. 4,

    X^{-1} = -(B2 D^{-1} B1)^{-1} (B2 D^{-1} F D^{-1} B1) (B2 D^{-1} B1)^{-1},   D = diag(F),

which is Eq. 4 as printed when B1 = G^T and B2 = G; in the MAC convention of this code B1 = -B2^T, and
the same expression holds.

Readings (the paper uses this preconditioner only as a reference point and leaves these open):
* Build matrix: the Newton Jacobian at the linearisation state (as aPLMM_NS), built once.
* Inner solves with F and with L = B2 D^{-1} B1: either exact (sparse LU), or GMRES restarted never,
  at most `inner_its` iterations or a relative residual of `inner_tol`, right-preconditioned with block
  Jacobi over the pores (a face belongs to the pore of the cell on its high side, a cell to its own
  pore; pinned cells are left out of L).
* schur="exact" replaces X^{-1} by the exact inverse of S (dense; tiny problems only): the form in
  which block-triangular preconditioning converges in two iterations.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .krylov import fgmres


class BlockSchur:
    def __init__(self, g, pins, J, labels, inner="exact", inner_its=20, inner_tol=1e-2, schur="bfbt"):
        self.g = g
        unk = g.unknown
        nfu = g.dim * g.ncell
        self.fu = unk[unk < nfu]
        pin_idx = np.sort(g.pidx(np.asarray(pins, np.int64)))
        cells = unk[unk >= nfu]
        self.pinned = pin_idx
        self.cn = np.setdiff1d(cells, pin_idx)
        J = sp.csr_matrix(J)
        self.F = J[self.fu][:, self.fu].tocsc()
        self.B1 = J[self.fu][:, self.cn].tocsc()
        self.B1p = J[self.fu][:, self.pinned].tocsc()
        self.B2 = J[self.cn][:, self.fu].tocsc()
        self.d = self.F.diagonal()
        Dinv = sp.diags(1.0 / self.d)
        self.L = (self.B2 @ Dinv @ self.B1).tocsc()
        self.Mm = (self.B2 @ Dinv @ self.F @ Dinv @ self.B1).tocsc()
        self.inner, self.inner_its, self.inner_tol = inner, inner_its, inner_tol
        self.schur = schur
        if schur == "exact":
            Fd = self.F.toarray()
            S = -self.B2.toarray() @ np.linalg.solve(Fd, self.B1.toarray())
            self.S_inv = np.linalg.inv(S)
        if inner == "exact":
            self.luF = spla.splu(self.F)
            self.luL = spla.splu(self.L)
        else:
            lab = np.asarray(labels).ravel()
            cell_of_face = self.fu % g.ncell
            self.jac_F = self._block_jacobi(self.F, lab[cell_of_face])
            self.jac_L = self._block_jacobi(self.L, lab[self.cn - nfu])

    @staticmethod
    def _block_jacobi(A, part):
        """Dense inverses of the diagonal blocks of A over the partition `part` (one id per row)."""
        blocks = []
        for p in np.unique(part):
            idx = np.flatnonzero(part == p)
            blocks.append((idx, np.linalg.inv(A[idx][:, idx].toarray())))

        def apply(r):
            z = np.zeros_like(r)
            for idx, inv in blocks:
                z[idx] = inv @ r[idx]
            return z
        return apply

    def _gmres(self, A, prec, r):
        nb = np.linalg.norm(r)
        if nb == 0.0:
            return np.zeros_like(r)
        x, _, _ = fgmres(lambda v: A @ v, prec, r, self.inner_tol * nb, restart=self.inner_its,
                         maxit=self.inner_its)
        return x

    def solve_F(self, r):
        return self.luF.solve(r) if self.inner == "exact" else self._gmres(self.F, self.jac_F, r)

    def solve_L(self, r):
        return self.luL.solve(r) if self.inner == "exact" else self._gmres(self.L, self.jac_L, r)

    def X_inv(self, vn):
        """y = X^{-1} v on the cells that are not pinned (Eq. 4, or the exact Schur inverse)."""
        if self.schur == "exact":
            return self.S_inv @ vn
        t = self.solve_L(vn)
        return -self.solve_L(self.Mm @ t)

    def apply(self, v):
        """z = M_B^{-1} v (full layout in and out)."""
        v = np.asarray(v, np.float64)
        yn = self.X_inv(v[self.cn])
        yp = v[self.pinned]
        u = self.solve_F(v[self.fu] - self.B1 @ yn - self.B1p @ yp)
        z = np.zeros(self.g.nfull)
        z[self.fu] = u
        z[self.cn] = yn
        z[self.pinned] = yp
        return z
