"""The closure solves the library makes with the Woodbury identity, checked against the oracle's direct
factorisation of the closure blocks (Eqs. 6 and 9), on CPU.

The closure block of a primary grid differs from its local block only on the diagonal of the rows K
coupled to f faces or to other primary grids: Abar = A_p + E_K D E_K^T, D = diag(delta).  Hence
  Abar^{-1} = X - X E_K (D^{-1} + E_K^T X E_K)^{-1} E_K^T X,   X = A_p^{-1},
with the k x k capacitance matrix D^{-1} + X_KK.  The library inverts the capacitance matrices by
Gauss-Jordan without pivoting, in FP32 in the FP32 build; these tests pin that this is safe on the
workloads' closure blocks (Gauss-Jordan without pivoting, emulated in FP32, reaches FP32 accuracy) and
that the identity with the oracle's blocks reproduces the oracle's closure solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov, mac, plmm
from paper_2510_22077_gb300 import inputs


def gauss_jordan_no_pivot(C, dtype):
    """In-place Gauss-Jordan inverse without pivoting in the given precision (rank-1 form per pivot)."""
    D = np.array(C, dtype=dtype)
    for t in range(len(D)):
        r = D[t, :].copy()
        r[t] = 1
        c = D[:, t].copy()
        c[t] = -1
        inv = dtype(1) / D[t, t]
        D[t, :] = 0
        D[:, t] = 0
        D -= np.outer(c, r * inv).astype(dtype)
    return D


def _blocks(kind, kw, variant):
    w = inputs.make_workload(kind, seed=0, **kw)
    mu = 3.87 if kind == "disks64" else inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)))
    _, A_b = pb.preconditioner(variant, krylov.stokes_solution(pb))
    A_b = A_b.tocsr()
    for i in range(pb.maps.n_prim):
        P = pb.maps.prim_unknowns[i]
        A_p = A_b[P][:, P].tocsc()
        Abar = plmm.closure_block(A_b, pb.maps, i)
        delta = (Abar - A_p).diagonal()
        K = np.nonzero(delta)[0]
        if 0 < len(K) <= 600:
            yield i, A_p, Abar, K, delta[K]


@pytest.mark.parametrize("kind,kw,variant", [("disks64", {}, "gplmm"), ("spheres", {"n": 24}, "aplmm_ns"),
                                             ("spheres", {"n": 32}, "gplmm")])
def test_capacitance_inverse_without_pivoting_and_woodbury_solve(kind, kw, variant):
    rng = np.random.default_rng(1)
    worst32, worst_wb, seen = 0.0, 0.0, 0
    for i, A_p, Abar, K, dK in _blocks(kind, kw, variant):
        n, k = A_p.shape[0], len(K)
        lu = spla.splu(A_p)
        E = np.zeros((n, k))
        E[K, np.arange(k)] = 1.0
        XE = lu.solve(E)                              # X E_K  (n x k)
        cap = np.diag(1.0 / dK) + XE[K]
        ci = np.linalg.inv(cap)
        c32 = gauss_jordan_no_pivot(cap.astype(np.float32), np.float32)
        worst32 = max(worst32, np.linalg.norm(c32 - ci) / np.linalg.norm(ci))
        # the same without pivoting in FP64 equals the pivoted inverse to rounding
        c64 = gauss_jordan_no_pivot(cap, np.float64)
        assert np.linalg.norm(c64 - ci) / np.linalg.norm(ci) < 1e-9, i
        # Woodbury with the oracle's X against the oracle's direct closure solve, two right-hand sides
        b = rng.standard_normal((n, 2))
        Xb = lu.solve(b)
        z = Xb - XE @ (ci @ Xb[K])
        z_direct = spla.splu(Abar.tocsc()).solve(b)
        worst_wb = max(worst_wb, np.linalg.norm(z - z_direct) / np.linalg.norm(z_direct))
        seen += 1
    assert seen >= 3
    print(f"{kind}{kw} {variant}: {seen} closure blocks; FP32 no-pivot capacitance inverse rel err {worst32:.2e}; "
          f"Woodbury vs direct closure solve {worst_wb:.2e}")
    # FP32 rounding amplified by the capacitance condition numbers of these blocks (measured: below 1e-5)
    assert worst32 < 1e-4
    assert worst_wb < 1e-9
