"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Bars: integer maps bit-exact; FP64 residual / Jacobian / operators to 1e-13 (different summation
order only); preconditioner applies 1e-9 (FP64; cond of the local blocks ~1e5 times eps), 1e-5
(FP32) and 2e-2 (BF16); converged velocity and pressure to 1e-8 relative L2 (both sides solved to
1e-11 or tighter)."""
import numpy as np
import pytest

from gpu_util import oracle_converged, problem, random_state, random_vector, rel, solver, to_dev
from oracle import mac, plmm
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [("tiny2d", dict(n=16), 0), ("tiny2d", dict(n=20, n_disks=3), 5), ("tiny3d", dict(n=8), 1),
         ("tiny3d", dict(n=10, porosity=0.55), 2)]


def _wl(kind, kw, seed):
    return inputs.make_workload(kind, seed=seed, **kw)


@pytest.fixture(scope="module")
def c1():
    return inputs.make_workload("disks64", seed=0)


@pytest.mark.parametrize("kind,kw,seed", CASES + [("disks64", {}, 0)])
def test_maps_bit_exact(kind, kw, seed):
    w = _wl(kind, kw, seed)
    pb = problem(w)
    S = solver(w)
    got = S.pns_export_maps()
    m, g = pb.maps, pb.g
    assert np.array_equal(got["pins"], pb.pins)
    assert np.array_equal(got["cell_prim"], m.cell_prim)
    assert np.array_equal(got["cell_iface"], m.cell_iface)
    for d in range(g.dim):
        assert np.array_equal(got["face_class"][d], m.face_class[d])
        assert np.array_equal(got["tags"][d], m.tags[d])
    cnt = np.zeros(g.nfull, np.int32)
    for u in m.dual_unknowns:
        cnt[u] += 1
    assert np.array_equal(got["dual_count"], cnt)
    inf = S.info()
    assert inf["n_prim"] == m.n_prim and inf["n_iface"] == m.n_iface
    assert inf["n_unknowns"] == len(g.unknown)


@pytest.mark.parametrize("kind,kw,seed", CASES + [("disks64", {}, 0)])
@pytest.mark.parametrize("dt", [0.0, 0.37])
def test_residual_and_jacobian(kind, kw, seed, dt):
    w = _wl(kind, kw, seed)
    pb = problem(w, dt=dt)
    S = solver(w, dt=dt)
    x = random_state(pb, seed=3)
    xp = random_state(pb, seed=4) if dt > 0 else None
    r_o = pb.residual(x, xp)
    r_g = S.pns_residual(to_dev(x), to_dev(xp) if xp is not None else None).cpu().numpy()
    assert rel(r_g, r_o) < 1e-13
    assert np.all(r_g[~pb.g.unknown_mask] == 0)
    v = random_vector(pb, seed=5)
    y_o = pb.jacobian(x) @ v
    y_g = S.pns_jacobian_apply(to_dev(x), to_dev(v)).cpu().numpy()
    assert rel(y_g, y_o) < 1e-13
    for var in ["gplmm", "aplmm_ns", "aplmm_s"]:
        A = pb.build_matrix(var, x)
        assert rel(S.pns_operator_apply(var, to_dev(x), to_dev(v)).cpu().numpy(), A @ v) < 1e-13


@pytest.mark.parametrize("kind,kw,seed", CASES)
@pytest.mark.parametrize("variant", ["gplmm", "aplmm_ns", "aplmm_s", "ml_only"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5), ("bf16", 2e-2)])
def test_precond_apply(kind, kw, seed, variant, precision, tol):
    """Built at a physical linearisation state (the Stokes solution with 2% noise), as in a solve."""
    w = _wl(kind, kw, seed)
    pb = problem(w)
    S = solver(w, variant=variant, precision=precision)
    x = random_state(pb, seed=7, scale=0.1)
    M, A_b = pb.preconditioner(variant, x)
    S.pns_build_precond(to_dev(x))
    for k in range(2):
        v = random_vector(pb, seed=11 + k)
        z_o = M.apply(v, A_b)
        z_g = S.pns_precond_apply(to_dev(v)).cpu().numpy()
        err = rel(z_g, z_o)
        print(f"precond apply {kind}{kw} {variant} {precision}: rel err {err:.2e}")
        assert err < tol, (variant, precision, err)
        assert np.all(z_g[~pb.g.unknown_mask] == 0)


@pytest.mark.parametrize("kind,kw,seed", CASES)
@pytest.mark.parametrize("variant", ["gplmm", "aplmm_ns", "aplmm_s"])
def test_precond_apply_fp64_noisy_state(kind, kw, seed, variant):
    """FP64 stress case: linearisation state with 10% random noise (reaction terms far from a flow)."""
    w = _wl(kind, kw, seed)
    pb = problem(w)
    S = solver(w, variant=variant, precision="fp64")
    x = random_state(pb, seed=7, scale=0.5)
    M, A_b = pb.preconditioner(variant, x)
    S.pns_build_precond(to_dev(x))
    v = random_vector(pb, seed=11)
    err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v, A_b))
    print(f"precond apply noisy {kind}{kw} {variant} fp64: rel err {err:.2e}")
    assert err < 1e-6


def test_precond_apply_c1(c1):
    pb = problem(c1, mu=3.87)
    x = random_state(pb, seed=2, scale=0.1)
    for variant in ["gplmm", "aplmm_ns"]:
        M, A_b = pb.preconditioner(variant, x)
        v = random_vector(pb, seed=3)
        z_o = M.apply(v, A_b)
        for precision, tol in [("fp64", 1e-9), ("fp32", 1e-5), ("bf16", 2e-2)]:
            S = solver(c1, mu=3.87, variant=variant, precision=precision)
            S.pns_build_precond(to_dev(x))
            err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), z_o)
            print(f"precond apply C1 {variant} {precision}: rel err {err:.2e}")
            assert err < tol, (variant, precision, err)
            S.close()


def test_stokes_solve_matches_oracle(c1):
    from oracle import krylov
    pb = problem(c1, mu=3.87)
    S = solver(c1, mu=3.87, newton_tol=1e-12, inner_tol=1e-12)
    x, st = S.pns_stokes_solve()
    assert rel(x.cpu().numpy(), krylov.stokes_solution(pb)) < 1e-8


@pytest.mark.parametrize("variant", ["gplmm", "aplmm_ns", "aplmm_s"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_newton_c1_matches_oracle(c1, variant, precision):
    """64x64 disk pack at Re ~ 1: Newton-FGMRES on the GPU, converged solution vs the oracle's
    direct Newton solve (both to 1e-12)."""
    from oracle import krylov
    mu = 3.8746364606724244
    pb = problem(c1, mu=mu)
    x_ref = oracle_converged(pb, krylov.stokes_solution(pb))
    S = solver(c1, mu=mu, variant=variant, precision=precision, newton_tol=1e-12, inner_tol=1e-12)
    x, _ = S.pns_stokes_solve()
    st = S.pns_newton_solve(x)
    assert st["status"] == "PNS_OK"
    err = rel(x.cpu().numpy(), x_ref)
    assert err < 1e-8, (err, st)
    # Newton residual check with the oracle's residual function
    assert np.linalg.norm(pb.residual(x.cpu().numpy())) / pb.r0 < 1e-11


def test_single_subdomain_one_iteration():
    """One label over all void: M^{-1} = A^{-1} for aPLMM_NS built at the iterate -> 1 FGMRES iteration."""
    w = inputs.make_workload("tiny2d", seed=2, n=14)
    w.labels = np.where(w.mask > 0, 1, 0).astype(np.int32)
    S = solver(w, variant="aplmm_ns", newton_tol=1e-12, inner_tol=1e-10, max_newton=1)
    x, _ = S.pns_stokes_solve()
    S.pns_build_precond(x)
    st = S.pns_newton_solve(x, check=False)
    assert st["fgmres_its"][0] == 1


def test_transient_step_matches_oracle(c1):
    from oracle import krylov
    mu, dt = 3.87, 0.5
    pb = problem(c1, mu=mu, dt=dt)
    import scipy.sparse.linalg as spla
    x0 = krylov.stokes_solution(pb) * 0.5
    # oracle: one backward-Euler step from x0 solved to convergence by direct Newton
    x = x0.copy()
    for _ in range(20):
        r = pb.residual(x, x0)
        J = mac.restrict(pb.g, pb.jacobian(x))
        dx = np.zeros(pb.g.nfull)
        dx[pb.g.unknown] = spla.spsolve(J.tocsc(), -r[pb.g.unknown])
        x += dx
        if np.linalg.norm(dx) < 1e-14 * np.linalg.norm(x):
            break
    S = solver(c1, mu=mu, dt=dt, variant="aplmm_ns", newton_tol=1e-12, inner_tol=1e-12)
    xg = to_dev(x0)
    xprev = to_dev(x0)
    st = S.pns_newton_solve(xg, xprev)
    assert rel(xg.cpu().numpy(), x) < 1e-8, st


def test_bad_labels_rejected():
    from paper_2510_22077_gb300 import pns
    w = inputs.make_workload("tiny2d", seed=0)
    lab = w.labels.copy()
    lab[w.mask == 0] = 3
    with pytest.raises(pns.PnsError):
        pns.Solver(w.mask, lab, 1.0, 1.0, (1.0, 0.0))


def test_apply_before_build_is_state_error():
    from paper_2510_22077_gb300 import pns
    w = inputs.make_workload("tiny2d", seed=0)
    S = solver(w)
    with pytest.raises(pns.PnsError) as e:
        S.pns_precond_apply(S.zeros())
    assert e.value.code == -7


def test_orphan_interface_fixture():
    """Hand fixture with an interface adjacent to no primary grid (it gets no coarse unknown)."""
    from types import SimpleNamespace
    lab = np.array([[3, 3, 0, 3, 3], [2, 2, 1, 2, 2], [3, 3, 0, 3, 3]])[None].astype(np.int32)
    w = SimpleNamespace(mask=(lab > 0).astype(np.uint8), labels=lab, periodic=(True, False, False))
    pb = problem(w)
    S = solver(w, variant="gplmm")
    got = S.pns_export_maps()
    assert np.array_equal(got["cell_iface"], pb.maps.cell_iface)
    x = random_state(pb, seed=1, scale=0.1)
    M, A_b = pb.preconditioner("gplmm", x)
    S.pns_build_precond(to_dev(x))
    v = random_vector(pb, seed=2)
    assert rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v, A_b)) < 1e-9


@pytest.mark.parametrize("variant", ["gplmm", "aplmm_s"])
def test_primary_grid_without_source_fixture(variant):
    """Hand fixture: a dead-end branch whose primary grid has no x face, so b_B = rho b is zero on it
    and it has no coarse unknown; its coarse slot is an identity row and column, and the apply matches
    the oracle's."""
    from types import SimpleNamespace
    lab = np.zeros((6, 5), np.int32)
    lab[0:3, :] = 1
    lab[3:6, 2] = 2
    w = SimpleNamespace(mask=(lab > 0).astype(np.uint8)[None], labels=lab[None], periodic=(True, False, False))
    pb = problem(w)
    x = random_state(pb, seed=1, scale=0.1)
    M, A_b = pb.preconditioner(variant, x)
    assert list(M.coarse_prim) == [0]
    S = solver(w, variant=variant, precision="fp64")
    S.pns_build_precond(to_dev(x))
    ao_inv = S.pns_export_coarse()
    assert ao_inv.shape == (3, 3)
    assert np.array_equal(ao_inv[2], [0.0, 0.0, 1.0]) and np.array_equal(ao_inv[:, 2], [0.0, 0.0, 1.0])
    assert rel(ao_inv[:2, :2], np.linalg.inv(M.Ao)) < 1e-10
    for seed in (2, 3):
        v = random_vector(pb, seed=seed)
        assert rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v, A_b)) < 1e-9


@pytest.mark.parametrize("variant", ["gplmm", "aplmm_s"])
def test_coarse_inverse_matches_oracle_and_repeats(c1, variant):
    """The coarse inverse (A^o = R^ A_b P^, Remark 1) equals the oracle's, and two builds at the same
    state give the same inverse (the pivoting is race-free: FP64 throughout, only the order of the
    atomic segment sums differs)."""
    pb = problem(c1, mu=3.87)
    x = random_state(pb, seed=2, scale=0.1)
    M, A_b = pb.preconditioner(variant, x)
    ref = np.linalg.inv(M.Ao)
    S = solver(c1, mu=3.87, variant=variant, precision="fp64")
    got = []
    for _ in range(2):
        S.pns_build_precond(to_dev(x))
        got.append(S.pns_export_coarse())
    tol = max(1e-10, 100 * np.finfo(float).eps * np.linalg.cond(M.Ao))
    # the library keeps one coarse slot per primary grid; those without a coarse unknown in the oracle
    # (b_B = 0 on them) hold identity rows and columns
    kept = list(range(M.n_ci)) + [M.n_ci + int(i) for i in M.coarse_prim]
    assert rel(got[0][np.ix_(kept, kept)], ref) < tol, rel(got[0][np.ix_(kept, kept)], ref)
    assert rel(got[1], got[0]) < 1e-12


def test_aplmm_s_stokes_preconditioner_is_kept(c1):
    """With variant aPLMM_S the Stokes solve's preconditioner is the context's own: Newton reuses it
    (its apply equals a fresh aPLMM_S build's) and the converged solution matches the oracle."""
    from oracle import krylov
    mu = 3.8746364606724244
    pb = problem(c1, mu=mu)
    S = solver(c1, mu=mu, variant="aplmm_s", precision="fp32", newton_tol=1e-12, inner_tol=1e-12)
    x, _ = S.pns_stokes_solve()
    S.pns_build_precond(x)          # returns at once: the aPLMM_S build does not depend on x
    v = to_dev(random_vector(pb, seed=4))
    z_kept = S.pns_precond_apply(v).cpu().numpy()
    S2 = solver(c1, mu=mu, variant="aplmm_s", precision="fp32")
    S2.pns_build_precond(S2.zeros())
    assert rel(z_kept, S2.pns_precond_apply(v).cpu().numpy()) < 1e-6
    st = S.pns_newton_solve(x)
    assert st["status"] == "PNS_OK"
    x_ref = oracle_converged(pb, krylov.stokes_solution(pb))
    assert rel(x.cpu().numpy(), x_ref) < 1e-8


@pytest.mark.parametrize("refine_steps", [-1, 2])
def test_fp32_refinement_modes_meet_the_bar(c1, refine_steps):
    """FP32 local inverses refined either inside each local solve (default, -1) or by Newton-Schulz
    steps at build time (2): both applies match the FP64 oracle to 1e-5."""
    pb = problem(c1, mu=3.87)
    x = random_state(pb, seed=2, scale=0.1)
    M, A_b = pb.preconditioner("gplmm", x)
    v = random_vector(pb, seed=3)
    z_o = M.apply(v, A_b)
    S = solver(c1, mu=3.87, variant="gplmm", precision="fp32", refine_steps=refine_steps)
    S.pns_build_precond(to_dev(x))
    err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), z_o)
    print(f"fp32 apply, refine_steps {refine_steps}: rel err {err:.2e}")
    assert err < 1e-5, err
