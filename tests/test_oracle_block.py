"""Pins of the block-triangular Schur comparator (oracle/block.py) against facts that do not depend on
its code: the two-iteration convergence of block-triangular preconditioning with the exact Schur
complement, the exactness of scaled BFBt when F is diagonal, and block Jacobi over a single pore being
the exact inverse."""
import numpy as np
import scipy.sparse as sp

from oracle import block, krylov, mac
from paper_2510_22077_gb300 import inputs


def _setup(kind="tiny2d", seed=0, mu=0.5, **kw):
    w = inputs.make_workload(kind, seed=seed, **kw)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)), w.periodic)
    x = krylov.stokes_solution(pb)
    return w, pb, x


def _rhs(pb, seed=0):
    b = np.zeros(pb.g.nfull)
    b[pb.g.unknown] = np.random.default_rng(seed).standard_normal(len(pb.g.unknown))
    return b


def test_exact_schur_converges_in_two_iterations():
    """With exact F^{-1} and X = S, J M_B^{-1} = I + N with N^2 = 0, so GMRES needs at most two
    iterations; a wrong sign or a transposed block breaks this."""
    for kind, kw in [("tiny2d", dict(n=16)), ("tiny3d", dict(n=8))]:
        w, pb, x = _setup(kind, **kw)
        J = pb.jacobian(x)
        M = block.BlockSchur(pb.g, pb.pins, J, w.labels, schur="exact")
        b = _rhs(pb)
        _, its, res = krylov.fgmres(lambda v: J @ v, M.apply, b, 1e-10 * np.linalg.norm(b))
        assert its <= 2 and res <= 1e-10 * np.linalg.norm(b), (kind, its, res)


def test_scaled_bfbt_is_the_exact_schur_inverse_when_F_is_diagonal():
    """If F = D = diag(F), Eq. 4 collapses to -(B2 D^{-1} B1)^{-1} = S^{-1} (S from a dense solve)."""
    w, pb, x = _setup("tiny2d", n=16)
    J = sp.csr_matrix(pb.jacobian(x))
    M0 = block.BlockSchur(pb.g, pb.pins, J, w.labels)
    fu = M0.fu
    E = sp.csr_matrix((np.ones(len(fu)), (fu, np.arange(len(fu)))), shape=(pb.g.nfull, len(fu)))
    off = M0.F - sp.diags(M0.F.diagonal())
    Jd = J - E @ off @ E.T
    bf = block.BlockSchur(pb.g, pb.pins, Jd, w.labels)
    ex = block.BlockSchur(pb.g, pb.pins, Jd, w.labels, schur="exact")
    v = np.random.default_rng(1).standard_normal(len(bf.cn))
    a, e = bf.X_inv(v), ex.X_inv(v)
    assert np.linalg.norm(a - e) / np.linalg.norm(e) < 1e-10
    # and with the real (non-diagonal) F the approximation is not exact
    a0, e0 = M0.X_inv(v), block.BlockSchur(pb.g, pb.pins, J, w.labels, schur="exact").X_inv(v)
    assert np.linalg.norm(a0 - e0) / np.linalg.norm(e0) > 1e-3


def test_block_jacobi_over_one_pore_is_exact():
    """One label over the whole void: block Jacobi is the exact inverse, the inner GMRES stops after one
    iteration and the apply equals the exact-inner apply."""
    w, pb, x = _setup("tiny2d", seed=2, n=14)
    lab = np.where(w.mask > 0, 1, 0).astype(np.int32)
    J = pb.jacobian(x)
    Mg = block.BlockSchur(pb.g, pb.pins, J, lab, inner="gmres", inner_its=20, inner_tol=1e-12)
    Me = block.BlockSchur(pb.g, pb.pins, J, lab, inner="exact")
    v = _rhs(pb, seed=3)
    zg, ze = Mg.apply(v), Me.apply(v)
    assert np.linalg.norm(zg - ze) / np.linalg.norm(ze) < 1e-9


def test_block_preconditioner_solves_the_c1_newton_system():
    """64 x 64 disk pack, first Newton system at the Stokes solution: FGMRES with the comparator
    (exact inner solves, and 20-iteration inner GMRES) reaches 1e-9."""
    w, pb, x = _setup("disks64", mu=3.87)
    J = pb.jacobian(x)
    r = -pb.residual(x)
    for inner in ("exact", "gmres"):
        M = block.BlockSchur(pb.g, pb.pins, J, w.labels, inner=inner)
        _, its, res = krylov.fgmres(lambda v: J @ v, M.apply, r, 1e-9 * np.linalg.norm(r), restart=100,
                                    maxit=600)
        assert res <= 1e-9 * np.linalg.norm(r), (inner, its, res)
        print(f"block comparator, inner {inner}: {its} FGMRES iterations")
