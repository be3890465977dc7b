"""Two-level PLMM preconditioners: build and apply (Sec. 3.2.2-3.2.3, Sec. 4).

M^{-1} = M_G^{-1} + M_dp^{-1} (I - A M_G^{-1})                       (Eq. 4a with n_st = 1, M_l = M_dp)
M_dp^{-1} = M_d^{-1} + M_p^{-1} (I - A M_d^{-1})                      (Eq. 24)
M_p^{-1} = sum_i E_i (R_i A_b E_i)^{-1} R_i,  M_d likewise on dual grids   (Eq. 25)
M_G^{-1} = P^ (R^ A_b P^)^{-1} R^                                     (Eq. 20 with Remark 1)

A_b is the build matrix: gPLMM -> Jacobian of the modified residual (Eq. 27, wind w, inertia removed
on tagged faces); aPLMM_NS -> Newton Jacobian at the initial iterate; aPLMM_S -> Stokes Jacobian.
The A in the two residual updates is A_b by default ("build": M is one fixed operator made from the
build matrix, Sec. 4), or the operator FGMRES solves ("current").

Two independent formulations are given:

* `Plmm` (recipe form): index maps, sparse LU per block (SuperLU, partial pivoting), shape vectors
  p^{p_i}_{c_j} = -(Abar^{p_i})^{-1} sum_{k in c_j} A_b[p_i, k]  (Eq. 15), correction vectors
  c^{p_i} = (Abar^{p_i})^{-1} b_B^{p_i}  (Eq. 17), closure blocks Abar^{p_i} = A_b[p_i, p_i] +
  diag(row sums of A_b[p_i, f and other primary grids])  (Eqs. 6, 9), restriction sums over each
  interface's cells and over every unknown of each primary grid (Eq. 18).
* `literal_preconditioner` (tiny images only): the permutation W, the blocks of Eq. 5, csum/diag of
  Eqs. 6 and 9, Q of Eq. 11, P of Eq. 14, R of Eq. 18 and E/R of Eq. 25 as explicit matrices,
  multiplied out densely.

Readings: f faces get zero in P^ (no Eq. 8 back-substitution); interfaces adjacent to no
primary grid get no coarse unknown (their cells get zero in P^ and no row of R^); a primary grid on which
b_B vanishes (no face unknown along the body force) gets no coarse unknown either: its correction vector
c^{p_i} = 0 would be a zero column of P^ and leave A^o singular; Pi(C^T) is the structural
pattern of C (every unknown of p_i); b_B = -r(u=0, p=0) with the previous time level zero, i.e. rho b
on face rows and 0 on cell rows; the coarse unknowns are ordered [x^o (coarse interfaces); y^o (primary)].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .maps import NOT_UNKNOWN


def source_rhs(g, prm):
    """b_B over the full index space: rho * b_d on every face unknown of axis d, 0 elsewhere."""
    bb = np.zeros(g.nfull)
    for d in range(g.dim):
        bb[g.fidx(d, np.arange(g.ncell))] = np.where(g.face_unknown[d], prm.rho * prm.b[d], 0.0)
    return bb


def closure_block(A_b, m, i):
    """Abar^{p_i}: A_b restricted to p_i plus, on the diagonal, the row sums of its couplings to
    interface (f) faces and to unknowns of other primary grids (Eqs. 6 and 9)."""
    Pi = m.prim_unknowns[i]
    rows = A_b[Pi].tocsr()
    blk = rows[:, Pi].tocsc()
    own = m.owner[rows.indices]
    take = (own == -3) | ((own >= 0) & (own != i))
    sel = rows.copy()
    sel.data = np.where(take, sel.data, 0.0)
    extra = np.asarray(sel.sum(axis=1)).ravel()
    return (blk + sp.diags(extra)).tocsc()


class Plmm:
    """Recipe form of the preconditioner, built once from the build matrix A_b."""

    def __init__(self, g, prm, m, A_b, use_coarse=True, rowsum="all"):
        self.g, self.m = g, m
        self.use_coarse = use_coarse
        self.n_ci = len(m.coarse_ifaces)
        bB = source_rhs(g, prm)
        # primary grids with a coarse unknown y^o_i: those whose correction vector is not zero
        self.coarse_prim = np.array([i for i in range(m.n_prim) if np.any(bB[m.prim_unknowns[i]] != 0.0)],
                                    np.int64)
        self.coarse_of_prim = np.full(m.n_prim, -1, np.int64)
        self.coarse_of_prim[self.coarse_prim] = self.n_ci + np.arange(len(self.coarse_prim))
        self.n_o = self.n_ci + len(self.coarse_prim)
        self.lu_p = [spla.splu(A_b[P][:, P].tocsc()) for P in m.prim_unknowns]
        self.lu_d = [spla.splu(A_b[D][:, D].tocsc()) for D in m.dual_unknowns]
        if not use_coarse:
            return
        # prolongation P^ (nfull x n_o): shape vectors, correction vectors, 1 on interface cells
        prow, pcol, pval = [], [], []
        self.shape = []
        self.corr = []
        for i in range(m.n_prim):
            Pi = m.prim_unknowns[i]
            lu_bar = spla.splu(closure_block(A_b, m, i))
            rows = A_b[Pi].tocsc()
            sh = {}
            for j in m.C[i]:
                cells = g.pidx(m.iface_cells[j])
                rhs = np.asarray(rows[:, cells].sum(axis=1)).ravel()
                s = -lu_bar.solve(rhs)
                sh[int(j)] = s
                prow.append(Pi)
                pcol.append(np.full(len(Pi), m.coarse_of_iface[j]))
                pval.append(s)
            c = lu_bar.solve(bB[Pi])
            self.shape.append(sh)
            self.corr.append(c)
            if self.coarse_of_prim[i] >= 0:
                prow.append(Pi)
                pcol.append(np.full(len(Pi), self.coarse_of_prim[i]))
                pval.append(c)
        for k, j in enumerate(m.coarse_ifaces):
            cells = g.pidx(m.iface_cells[j])
            prow.append(cells)
            pcol.append(np.full(len(cells), k))
            pval.append(np.ones(len(cells)))
        self.Phat = sp.csr_matrix((np.concatenate(pval), (np.concatenate(prow), np.concatenate(pcol))),
                                  shape=(g.nfull, self.n_o))
        # restriction R^ (n_o x nfull): interface rows sum their cells; primary rows all unknowns of p_i
        # (Eq. 18, the pattern of C^T), or with rowsum = "cells" only the cells (pressures) of p_i
        rrow, rcol = [], []
        for k, j in enumerate(m.coarse_ifaces):
            cells = g.pidx(m.iface_cells[j])
            rrow.append(np.full(len(cells), k))
            rcol.append(cells)
        for i in self.coarse_prim:
            Pi = m.prim_unknowns[i]
            if rowsum == "cells":
                Pi = Pi[Pi >= g.pidx(0)]
            rrow.append(np.full(len(Pi), self.coarse_of_prim[i]))
            rcol.append(Pi)
        rr = np.concatenate(rrow)
        self.Rhat = sp.csr_matrix((np.ones(len(rr)), (rr, np.concatenate(rcol))), shape=(self.n_o, g.nfull))
        self.Ao = (self.Rhat @ A_b @ self.Phat).toarray()
        self.Ao_lu = sla.lu_factor(self.Ao)

    # --- pieces of the apply
    def coarse(self, v):
        """z_G = M_G^{-1} v."""
        if not self.use_coarse:
            return np.zeros_like(v)
        y = sla.lu_solve(self.Ao_lu, self.Rhat @ v)
        return self.Phat @ y

    def dual(self, t):
        """z_d = M_d^{-1} t (overlapping dual grids add)."""
        z = np.zeros_like(t)
        for D, lu in zip(self.m.dual_unknowns, self.lu_d):
            z[D] += lu.solve(t[D])
        return z

    def primary(self, t):
        """z_p = M_p^{-1} t."""
        z = np.zeros_like(t)
        for P, lu in zip(self.m.prim_unknowns, self.lu_p):
            z[P] = lu.solve(t[P])
        return z

    def apply(self, v, A):
        """z = M^{-1} v with A the operator of the two residual updates (Eqs. 4a and 24)."""
        zG = self.coarse(v)
        t1 = v - A @ zG
        zd = self.dual(t1)
        t2 = t1 - A @ zd
        zp = self.primary(t2)
        return zG + zd + zp


# ----------------------------------------------------------------------------------------------
# literal matrix form (tiny images)
# ----------------------------------------------------------------------------------------------
def literal_preconditioner(g, prm, m, A_b, A_solve, use_coarse=True):
    """Dense M^{-1} assembled from the explicit matrices of Eqs. 5-25 (restricted to unknowns).
    Returns (Minv, MGinv, unknown index list) with matrices over the unknowns in global order."""
    unk = g.unknown
    N = len(unk)
    pos = -np.ones(g.nfull, np.int64)
    pos[unk] = np.arange(N)
    Ab = A_b[unk][:, unk].toarray()
    As = A_solve[unk][:, unk].toarray()
    # permuted order [p_1 .. p_n | c_1 .. c_m | f]
    p_lists = [pos[P] for P in m.prim_unknowns]
    c_lists = [pos[g.pidx(m.iface_cells[j])] for j in m.coarse_ifaces]
    orphan = [pos[g.pidx(m.iface_cells[j])] for j in range(m.n_iface) if m.coarse_of_iface[j] < 0]
    f_list = np.concatenate([pos[m.f_faces]] + orphan).astype(np.int64)
    order = np.concatenate(p_lists + c_lists + [f_list]).astype(np.int64)
    assert len(order) == N and len(np.unique(order)) == N
    W = np.zeros((N, N))
    W[order, np.arange(N)] = 1.0                          # x^ = W x
    A = W.T @ Ab @ W
    Np = sum(len(l) for l in p_lists)
    Nc = sum(len(l) for l in c_lists)
    p_s, c_s, f_s = slice(0, Np), slice(Np, Np + Nc), slice(Np + Nc, N)
    App, Apc, Apf = A[p_s, p_s], A[p_s, c_s], A[p_s, f_s]
    Acp, Acc, Acf = A[c_s, p_s], A[c_s, c_s], A[c_s, f_s]
    csum = lambda X: X @ np.ones(X.shape[1])
    At_pp = App + np.diag(csum(Apf))                      # Eq. 6
    At_cc = Acc + np.diag(csum(Acf))
    # Eq. 9: block-diagonalise At_pp
    bounds = np.cumsum([0] + [len(l) for l in p_lists])
    Abar_pp = np.zeros_like(At_pp)
    for i in range(m.n_prim):
        si = slice(bounds[i], bounds[i + 1])
        off = np.zeros(bounds[i + 1] - bounds[i])
        for j in range(m.n_prim):
            if j != i:
                off += csum(At_pp[si, bounds[j]:bounds[j + 1]])
        Abar_pp[si, si] = At_pp[si, si] + np.diag(off)
    Abar = np.block([[Abar_pp, Apc], [Acp, At_cc]])       # Eq. 10
    # Eq. 11: Q
    nci = len(c_lists)
    Qo = np.zeros((Nc, nci))
    cb = np.cumsum([0] + [len(l) for l in c_lists])
    for j in range(nci):
        Qo[cb[j]:cb[j + 1], j] = 1.0
    Q = np.block([[np.eye(Np), np.zeros((Np, nci))], [np.zeros((Nc, Np)), Qo]])
    AM = Q.T @ Abar @ Q                                   # Eq. 12
    Abar_pc = AM[:Np, Np:]
    Abar_pp_M = AM[:Np, :Np]
    # Eq. 15: B = -(Abar^p_p)^{-1} Abar^p_c (block-diagonal inverse -> per-grid shape vectors)
    B = -np.linalg.solve(Abar_pp_M, Abar_pc)
    # Eq. 17: C = blockdiag(c^{p_i}),  c^{p_i} = (Abar^{p_i})^{-1} b_B^{p_i}
    bB_full = source_rhs(g, prm)[unk]
    bB_p = (W.T @ bB_full)[:Np]
    # a primary grid whose b_B is zero has c^{p_i} = 0: its column of C and row of Pi(C^T) are left out
    kept = [i for i in range(m.n_prim) if np.any(bB_p[bounds[i]:bounds[i + 1]] != 0.0)]
    Cm = np.zeros((Np, len(kept)))
    for k, i in enumerate(kept):
        si = slice(bounds[i], bounds[i + 1])
        Cm[si, k] = np.linalg.solve(Abar_pp_M[si, si], bB_p[si])
    Pm = np.block([[B, Cm], [np.eye(nci), np.zeros((nci, len(kept)))]])   # Eq. 14
    # Eq. 18 with the structural pattern of C
    PiCT = np.zeros((len(kept), Np))
    for k, i in enumerate(kept):
        PiCT[k, bounds[i]:bounds[i + 1]] = 1.0
    Rm = np.block([[np.zeros((nci, Np)), np.eye(nci)], [PiCT, np.zeros((len(kept), nci))]])
    # Eq. 21: P^ = W Q P (f rows zero), R^ = R Q^T W^T (f columns dropped)
    QP = Q @ Pm
    QP_full = np.vstack([QP, np.zeros((N - Np - Nc, QP.shape[1]))])
    Phat = W @ QP_full
    Rhat = Rm @ Q.T @ (W.T)[:Np + Nc, :]
    MG = Phat @ np.linalg.solve(Rhat @ Ab @ Phat, Rhat) if use_coarse else np.zeros((N, N))   # Remark 1
    # Eq. 25: additive Schwarz on primary and dual grids with 0/1 restriction/extension matrices
    def schwarz(lists):
        Minv = np.zeros((N, N))
        for l in lists:
            E = np.zeros((N, len(l)))
            E[l, np.arange(len(l))] = 1.0
            Minv += E @ np.linalg.solve(E.T @ Ab @ E, E.T)
        return Minv
    Mp = schwarz([pos[P] for P in m.prim_unknowns])
    Md = schwarz([pos[D] for D in m.dual_unknowns])
    I = np.eye(N)
    Mdp = Md + Mp @ (I - As @ Md)                         # Eq. 24
    M = MG + Mdp @ (I - As @ MG)                          # Eq. 4a
    return M, MG, unk
