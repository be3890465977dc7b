"""The FP32 local inverses built with the Gauss-Jordan update on the 5th-generation tensor cores
(gj_tensor_cores = 2: tcgen05.mma kind::tf32 with a 3-term split, TMA-staged operands) against the FP64
oracle and against the same build on the FP32 FMA units.  The blocks of these workloads span one to
several dozen 128-wide panels with ragged last tiles, so every tile kind of the update is exercised.

Bars: the refined apply (the default local solve) meets the FP32 bar of 1e-5 against the oracle; the
raw inverses (refine_steps = 0) of the two update kernels agree to FP32 rounding amplified by the block
condition numbers (1e-3 relative on the apply), where a wrong layout or a dropped product would leave
an O(1) difference."""
import numpy as np
import pytest

from gpu_util import problem, random_state, random_vector, rel, solver, to_dev
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,kw,variant", [("disks64", {}, "gplmm"), ("spheres", {"n": 32}, "aplmm_s"),
                                             ("spheres", {"n": 48}, "aplmm_ns")])
def test_tensor_core_update_matches_oracle_and_fma(kind, kw, variant):
    w = inputs.make_workload(kind, seed=0, **kw)
    mu = 3.87 if kind == "disks64" else inputs.mu_kozeny_carman(w.mask, 1.0)
    pb = problem(w, mu=mu)
    x = random_state(pb, seed=2, scale=0.1)
    M, A_b = pb.preconditioner(variant, x)
    v = random_vector(pb, seed=3)
    z_o = M.apply(v, A_b)
    out = {}
    for gj in (0, 2):
        for refine in (-1, 0):
            S = solver(w, mu=mu, variant=variant, precision="fp32", refine_steps=refine, gj_tensor_cores=gj)
            S.pns_build_precond(to_dev(x))
            out[gj, refine] = S.pns_precond_apply(to_dev(v)).cpu().numpy()
            S.close()
    e_tc = rel(out[2, -1], z_o)
    e_fma = rel(out[0, -1], z_o)
    d_raw = rel(out[2, 0], out[0, 0])
    print(f"{kind}{kw} {variant}: refined apply vs oracle tcgen05 {e_tc:.2e} fma {e_fma:.2e}; "
          f"raw inverses tcgen05 vs fma {d_raw:.2e}; raw tcgen05 vs oracle {rel(out[2, 0], z_o):.2e}")
    assert e_tc < 1e-5
    assert d_raw < 1e-3
