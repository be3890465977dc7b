"""Pins of the oracle's preconditioners (Sec. 3-4) and Krylov/Newton drivers (Sec. 8): two
independent formulations of M (literal matrices of Eqs. 5-25 vs the index recipe), the projection
property of M_G with Remark 1 (Proposition 1), exactness with a single subdomain, variant
equivalence in the Stokes limit (Sec. 8.1), scale invariance of the correction vectors, the gPLMM
coupling invariant (Sec. 4), FGMRES against a dense solve, and Newton-FGMRES against brute force."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov, mac, maps, plmm
from paper_2510_22077_gb300 import inputs

VARIANTS = ["gplmm", "aplmm_ns", "aplmm_s", "ml_only"]


def _tiny(kind, seed, rho=1.0, mu=0.3, b=(1.0, 0.0, 0.0), dt=0.0, n=None):
    kw = {} if n is None else {"n": n}
    w = inputs.make_workload(kind, seed=seed, **kw)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(rho, mu, b, dt))
    return pb


def _state(pb, seed=0):
    """A physical linearisation state: the Stokes solution plus a perturbation."""
    xs = krylov.stokes_solution(pb)
    rng = np.random.default_rng(seed)
    x = xs.copy()
    x[pb.g.unknown] += 0.1 * np.abs(xs).max() * rng.standard_normal(len(pb.g.unknown))
    return x


@pytest.mark.parametrize("kind,seed", [("tiny2d", 0), ("tiny2d", 4), ("tiny3d", 1)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_literal_equals_recipe(kind, seed, variant):
    pb = _tiny(kind, seed)
    g = pb.g
    if pb.maps.n_iface == 0:
        pytest.skip("fixture has no interface")
    x = _state(pb)
    M, A_b = pb.preconditioner(variant, x)
    Mlit, MGlit, unk = plmm.literal_preconditioner(g, pb.prm, pb.maps, A_b, A_b, use_coarse=(variant != "ml_only"))
    rng = np.random.default_rng(2)
    for _ in range(3):
        v = np.zeros(g.nfull)
        v[unk] = rng.standard_normal(len(unk))
        z = M.apply(v, A_b)
        zl = Mlit @ v[unk]
        # cond(A_b) reaches 1e5 on these perturbed states, so two factorisation orders agree to
        # ~1e-12; a wrong term in either formulation shows as an O(1) difference
        assert np.linalg.norm(z[unk] - zl) / np.linalg.norm(zl) < 1e-11
        assert np.all(z[~g.unknown_mask] == 0.0)
        if variant != "ml_only":
            # two LU orderings of the coarse system: agreement to cond(A^o) * eps
            tol = max(1e-11, 50 * np.linalg.cond(M.Ao) * np.finfo(float).eps)
            zg = M.coarse(v)
            assert np.linalg.norm(zg[unk] - MGlit @ v[unk]) / np.linalg.norm(MGlit @ v[unk]) < tol


@pytest.mark.parametrize("variant", ["gplmm", "aplmm_ns", "aplmm_s"])
def test_coarse_is_projection_and_consistent(variant):
    """Remark 1: with M_G^{-1} = P^(R^ A P^)^{-1} R^ and the same A, E_G = I - M_G^{-1} A is a
    projection (eigenvalues exactly 0 and 1), and the restricted residual vanishes."""
    pb = _tiny("tiny2d", 0, n=14)
    g = pb.g
    x = _state(pb)
    M, A_b = pb.preconditioner(variant, x)
    unk = g.unknown
    _, MG, _ = plmm.literal_preconditioner(g, pb.prm, pb.maps, A_b, A_b)
    T = MG @ A_b[unk][:, unk].toarray()
    assert np.linalg.norm(T @ T - T) <= 1e-10 * np.linalg.norm(T)
    ev = np.linalg.eigvals(np.eye(len(unk)) - T)
    d = np.minimum(np.abs(ev), np.abs(ev - 1))
    assert d.max() < 1e-8
    rng = np.random.default_rng(3)
    v = np.zeros(g.nfull)
    v[unk] = rng.standard_normal(len(unk))
    res = M.Rhat @ (v - A_b @ M.coarse(v))
    # exact in exact arithmetic; the coarse LU solve leaves cond(A^o) * eps
    tol = max(1e-12, 100 * np.finfo(float).eps * np.linalg.cond(M.Ao))
    assert np.abs(res).max() <= tol * np.abs(M.Rhat @ v).max()


def test_correction_vector_scale_invariance():
    """A column scaling of P^ cancels in P^(R^AP^)^{-1}R^: multiplying b (hence b_B and every c^{p_i})
    by 3 leaves M_G unchanged when the build matrix does not depend on b (aPLMM_S)."""
    pb1 = _tiny("tiny2d", 0, n=14, b=(1.0, 0.0))
    pb3 = _tiny("tiny2d", 0, n=14, b=(3.0, 0.0))
    x = np.zeros(pb1.g.nfull)
    M1, _ = pb1.preconditioner("aplmm_s", x)
    M3, _ = pb3.preconditioner("aplmm_s", x)
    assert np.linalg.norm(M3.corr[0] - 3 * M1.corr[0]) <= 1e-13 * np.linalg.norm(M3.corr[0])
    rng = np.random.default_rng(1)
    v = np.zeros(pb1.g.nfull)
    v[pb1.g.unknown] = rng.standard_normal(len(pb1.g.unknown))
    z1, z3 = M1.coarse(v), M3.coarse(v)
    assert np.linalg.norm(z1 - z3) / np.linalg.norm(z1) < 1e-12


def test_variants_coincide_in_stokes_limit():
    """At a zero linearisation state the Newton Jacobian, the Oseen Jacobian (w = 0) and the Stokes
    Jacobian are one matrix, so gPLMM = aPLMM_NS = aPLMM_S (Sec. 8.1: gPLMM_S = aPLMM_S)."""
    pb = _tiny("tiny3d", 1)
    x0 = np.zeros(pb.g.nfull)
    Ms = [pb.preconditioner(v, x0) for v in ["gplmm", "aplmm_ns", "aplmm_s"]]
    A0 = Ms[0][1]
    for _, A in Ms[1:]:
        # the same entries, summed in a different order (zero inertia terms included or not)
        assert abs(A - A0).max() <= 4 * np.finfo(float).eps * abs(A0).max()
    rng = np.random.default_rng(0)
    v = np.zeros(pb.g.nfull)
    v[pb.g.unknown] = rng.standard_normal(len(pb.g.unknown))
    zs = [M.apply(v, A) for M, A in Ms]
    for z in zs[1:]:
        assert np.linalg.norm(z - zs[0]) <= 1e-13 * np.linalg.norm(zs[0])


def test_single_subdomain_is_exact():
    """One label over the whole void: no interfaces, M_p is the exact inverse, so
    M^{-1} = M_G^{-1} + A^{-1}(I - A M_G^{-1}) = A^{-1} and FGMRES stops after one iteration."""
    w = inputs.make_workload("tiny2d", seed=2, n=14)
    lab = np.where(w.mask > 0, 1, 0).astype(np.int32)
    pb = krylov.Problem(w.mask, lab, mac.Params(1.0, 0.3, (1.0, 0.0)))
    assert pb.maps.n_iface == 0 and pb.maps.n_prim == 1
    x0 = krylov.stokes_solution(pb)
    # aPLMM_NS built at the current iterate: build matrix == solved operator
    M, A_b = pb.preconditioner("aplmm_ns", x0)
    r = pb.residual(x0)
    J = pb.jacobian(x0)
    dx, its, beta = krylov.fgmres(lambda v: J @ v, lambda v: M.apply(v, A_b), -r, 1e-12 * np.linalg.norm(r))
    assert its == 1
    ref = np.zeros(pb.g.nfull)
    ref[pb.g.unknown] = spla.spsolve(mac.restrict(pb.g, J).tocsc(), -r[pb.g.unknown])
    assert np.linalg.norm(dx - ref) / np.linalg.norm(ref) < 1e-10      # cond(J) ~ 1e5 times eps


def test_fgmres_against_dense_solve():
    rng = np.random.default_rng(7)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, its, beta = krylov.fgmres(lambda v: A @ v, lambda v: v, b, 1e-13, restart=17)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(b)
    Ainv = np.linalg.inv(A)
    x1, its1, _ = krylov.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-10)
    assert its1 == 1


def test_gplmm_coupling_invariant(c1_workload):
    """Sec. 4: with inertia removed on tagged faces, the rows of primary grid p_i of J~_w couple to
    unknowns outside p_i and its interface cells only through the viscous term (value -mu)."""
    w = c1_workload
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 0.37, (1.0, 0.0)))
    x = _state(pb)
    A = pb.build_matrix("gplmm", x).tocoo()
    own = pb.maps.owner
    rows_p = own[A.row] >= 0
    outside = rows_p & ((own[A.col] == -3) | ((own[A.col] >= 0) & (own[A.col] != own[A.row])))
    assert outside.any()
    assert np.allclose(A.data[outside], -0.37, rtol=0, atol=1e-15)


def test_dual_fraction_in_paper_range(c1_workload):
    w = c1_workload
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 1.0, (1.0, 0.0)))
    fd = maps.dual_fraction(pb.g, pb.maps)
    assert 0.05 < fd < 0.5, fd


@pytest.mark.parametrize("kind,seed,variant", [("tiny2d", 0, "gplmm"), ("tiny2d", 3, "aplmm_ns"),
                                               ("tiny3d", 1, "gplmm"), ("tiny3d", 2, "aplmm_s")])
def test_newton_fgmres_matches_brute_force(kind, seed, variant):
    pb = _tiny(kind, seed, rho=1.0, mu=0.5)
    x0 = krylov.stokes_solution(pb)
    x, st = krylov.newton(pb, x0, variant=variant, tol=1e-12, inner_tol=1e-13)
    assert st["converged"]
    xd = x0.copy()
    for _ in range(20):
        dx = pb.direct_step(xd)
        xd += dx
        if np.linalg.norm(dx) <= 1e-14 * np.linalg.norm(xd):
            break
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10


def test_newton_fgmres_on_c1(c1_workload):
    """The 64^2 disk pack at Re ~ 1 (mu from the Stokes calibration): gPLMM Newton-FGMRES reaches
    a 1e-8 Newton residual and agrees with a direct sparse Newton solve."""
    w = c1_workload
    mu = 3.8746364606724244
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0)))
    x0 = krylov.stokes_solution(pb)
    x, st = krylov.newton(pb, x0, variant="gplmm", tol=1e-11, inner_tol=1e-12)
    assert st["converged"]
    xd = x0.copy()
    for _ in range(10):
        xd += pb.direct_step(xd)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_orphan_interface_gets_no_coarse_unknown():
    """3 x 5, x-periodic.  Cell (1,2) (label 1) touches only interface cells of pair (2,3) and solid,
    so its interface (pair (1,2)) is adjacent to no primary grid.  It must get no coarse unknown: the
    coarse matrix stays nonsingular and the literal and recipe forms still agree."""
    lab = np.array([[3, 3, 0, 3, 3],
                    [2, 2, 1, 2, 2],
                    [3, 3, 0, 3, 3]])
    mask = (lab > 0).astype(np.uint8)[None]
    pb = krylov.Problem(mask, lab[None].astype(np.int32), mac.Params(1.0, 0.5, (1.0, 0.0)))
    m = pb.maps
    # hand-derived: interface 0 = pair (2,3) cells {5, 6, 8, 9}; interface 1 = pair (1,2) cell {7}
    assert [sorted(c.tolist()) for c in m.iface_cells] == [[5, 6, 8, 9], [7]]
    assert list(m.dropped_labels) == [1, 2]        # every cell of labels 1 and 2 is an interface cell
    assert [list(c) for c in m.C] == [[0]]
    assert list(m.coarse_ifaces) == [0] and list(m.coarse_of_iface) == [0, -1]
    x = krylov.stokes_solution(pb)
    for variant in ["gplmm", "aplmm_s"]:
        M, A_b = pb.preconditioner(variant, x)
        assert M.n_o == 2
        assert np.isfinite(np.linalg.cond(M.Ao)) and np.linalg.cond(M.Ao) < 1e12
        Mlit, _, unk = plmm.literal_preconditioner(pb.g, pb.prm, m, A_b, A_b)
        v = np.zeros(pb.g.nfull)
        v[unk] = np.random.default_rng(0).standard_normal(len(unk))
        zl = Mlit @ v[unk]
        assert np.linalg.norm(M.apply(v, A_b)[unk] - zl) / np.linalg.norm(zl) < 1e-11
        assert M.coarse(v)[pb.g.pidx(7)] == 0.0


def test_primary_grid_without_source_gets_no_coarse_unknown():
    """6 x 5, x-periodic, body force along x.  A channel of label 1 (rows 0-2) with a one-cell-wide
    dead-end branch of label 2 (column 2, rows 3-5).  The branch's primary grid holds three cells and
    three y faces and no x face, so b_B = rho b vanishes on it and its correction vector
    c = Abar^{-1} b_B is zero: a coarse unknown for it would be a zero column of P^ and make A^o
    singular.  It must get none; the literal and recipe forms still agree."""
    lab = np.zeros((6, 5), int)
    lab[0:3, :] = 1
    lab[3:6, 2] = 2
    mask = (lab > 0).astype(np.uint8)[None]
    pb = krylov.Problem(mask, lab[None].astype(np.int32), mac.Params(1.0, 0.5, (1.0, 0.0)))
    g, m = pb.g, pb.maps
    # hand-derived: interface = channel cell (row 2, col 2) = 12; the branch primary grid holds the
    # y faces of cells 17, 22, 27 (rows 3-5 of column 2) and their three cells
    assert [sorted(c.tolist()) for c in m.iface_cells] == [[12]]
    assert sorted(m.prim_unknowns[1].tolist()) == [g.fidx(1, 17), g.fidx(1, 22), g.fidx(1, 27),
                                                   g.pidx(17), g.pidx(22), g.pidx(27)]
    assert [list(c) for c in m.C] == [[0], [0]]
    x = krylov.stokes_solution(pb)
    for variant in ["gplmm", "aplmm_s"]:
        M, A_b = pb.preconditioner(variant, x)
        assert list(M.coarse_prim) == [0] and list(M.coarse_of_prim) == [1, -1] and M.n_o == 2
        assert not np.any(M.corr[1])
        assert np.linalg.cond(M.Ao) < 1e12
        Mlit, _, unk = plmm.literal_preconditioner(pb.g, pb.prm, m, A_b, A_b)
        v = np.zeros(pb.g.nfull)
        v[unk] = np.random.default_rng(0).standard_normal(len(unk))
        zl = Mlit @ v[unk]
        assert np.linalg.norm(M.apply(v, A_b)[unk] - zl) / np.linalg.norm(zl) < 1e-11



@pytest.mark.parametrize("kind,seed", [("tiny2d", 0), ("tiny3d", 1)])
def test_cells_only_restriction_leaves_the_coarse_matrix_singular(kind, seed):
    """Eq. 18 sums every unknown of p_i (the pattern of C^T).  Summing only its cells, the alternative
    some readings allow, makes every coarse row a sum of continuity equations, which are linearly
    dependent over a closed or periodic domain: A^o becomes singular, so that form is not offered by the
    library."""
    w = inputs.make_workload(kind, seed=seed)
    conds = {}
    for r in ("all", "cells"):
        pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 0.3, (1.0, 0.0, 0.0)), rowsum=r)
        if pb.maps.n_iface == 0:
            pytest.skip("fixture has no interface")
        M, A_b = pb.preconditioner("gplmm", krylov.stokes_solution(pb))
        sv = np.linalg.svd(M.Ao, compute_uv=False)
        conds[r] = sv[0] / sv[-1]
        if r == "cells":
            prim_rows = M.Rhat[M.n_ci:].tocoo()
            assert prim_rows.nnz > 0 and np.all(prim_rows.col >= pb.g.pidx(0))
    assert conds["all"] < 1e6
    assert conds["cells"] > 1e12
