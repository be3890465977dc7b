"""Parity of the block-triangular Schur comparator (variant block_schur) with the oracle
(oracle/block.py): the Newton Jacobian at a linearisation state, scaled BFBt Schur approximation
(Eq. 4), inner GMRES with block Jacobi over the pores."""
import numpy as np
import pytest

from gpu_util import oracle_converged, problem, random_state, random_vector, rel, solver, to_dev
from oracle import block
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [("tiny2d", dict(n=16), 0), ("tiny3d", dict(n=8), 1), ("disks64", {}, 0)]


@pytest.mark.parametrize("kind,kw,seed", CASES)
def test_block_apply_fixed_inner_iterations_fp64(kind, kw, seed):
    """Inner GMRES with a fixed count (tolerance 1e-300 never stops it early): both sides minimise
    over the same Krylov spaces, so the applies agree to rounding."""
    w = inputs.make_workload(kind, seed=seed, **kw)
    pb = problem(w)
    x = random_state(pb, seed=7, scale=0.1)
    its = 8
    M = block.BlockSchur(pb.g, pb.pins, pb.jacobian(x), w.labels, inner="gmres", inner_its=its, inner_tol=1e-300)
    S = solver(w, variant="block_schur", precision="fp64", block_inner_its=its, block_inner_tol=1e-300)
    S.pns_build_precond(to_dev(x))
    for k in range(2):
        v = random_vector(pb, seed=11 + k)
        err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v))
        print(f"block apply {kind} fp64: rel err {err:.2e}")
        assert err < 1e-9, err


@pytest.mark.parametrize("kind,kw,seed", CASES[:2])
def test_block_apply_converged_inner_matches_exact_blocks(kind, kw, seed):
    """Inner solves run to 1e-13: the apply equals the oracle's with exact (LU) inner solves."""
    w = inputs.make_workload(kind, seed=seed, **kw)
    pb = problem(w)
    x = random_state(pb, seed=7, scale=0.1)
    M = block.BlockSchur(pb.g, pb.pins, pb.jacobian(x), w.labels, inner="exact")
    S = solver(w, variant="block_schur", precision="fp64", block_inner_its=100, block_inner_tol=1e-13)
    S.pns_build_precond(to_dev(x))
    v = random_vector(pb, seed=3)
    err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v))
    assert err < 1e-8, err


def test_block_apply_fp32_blocks():
    w = inputs.make_workload("disks64", seed=0)
    pb = problem(w)
    x = random_state(pb, seed=7, scale=0.1)
    its = 8
    M = block.BlockSchur(pb.g, pb.pins, pb.jacobian(x), w.labels, inner="gmres", inner_its=its, inner_tol=1e-300)
    S = solver(w, variant="block_schur", precision="fp32", block_inner_its=its, block_inner_tol=1e-300)
    S.pns_build_precond(to_dev(x))
    v = random_vector(pb, seed=5)
    err = rel(S.pns_precond_apply(to_dev(v)).cpu().numpy(), M.apply(v))
    print(f"block apply disks64 fp32: rel err {err:.2e}")
    assert err < 1e-4, err


def test_newton_with_block_comparator_matches_oracle():
    """64 x 64 disk pack at Re ~ 1: Newton-FGMRES with the comparator (default inner settings)
    converges to the oracle's solution."""
    from oracle import krylov
    w = inputs.make_workload("disks64", seed=0)
    mu = 3.8746364606724244
    pb = problem(w, mu=mu)
    x_ref = oracle_converged(pb, krylov.stokes_solution(pb))
    S = solver(w, mu=mu, variant="block_schur", precision="fp32", newton_tol=1e-12, inner_tol=1e-12)
    x, _ = S.pns_stokes_solve()
    S.pns_build_precond(x)
    st = S.pns_newton_solve(x)
    assert st["status"] == "PNS_OK"
    print("block comparator Newton:", st["fgmres_its"])
    assert rel(x.cpu().numpy(), x_ref) < 1e-8


def test_static_apply_refuses_the_block_comparator():
    from paper_2510_22077_gb300 import pns
    w = inputs.make_workload("tiny2d", seed=0, n=16)
    S = solver(w, variant="block_schur")
    S.pns_build_precond(S.zeros())
    with pytest.raises(pns.PnsError) as e:
        S.pns_precond_apply_static(S.zeros())
    assert e.value.code == -1
