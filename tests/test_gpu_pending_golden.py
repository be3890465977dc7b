"""Full-size parity of one preconditioner apply on sampled outputs: aPLMM_S with FP32 local inverses on
the 96^3 sphere pack of the benchmark, against FP64 oracle values stored by
tests/golden/make_spheres96_aplmm_s_apply.py (the oracle's build takes minutes, too slow for a test).
Marked gpu_pending: it joins the gpu set once it has run on a GPU."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu_pending

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spheres96_aplmm_s_apply.json")


def test_aplmm_s_apply_full_size_sampled():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from gpu_util import problem, solver, to_dev
    from paper_2510_22077_gb300 import inputs
    ref = json.load(open(GOLDEN))
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    assert abs(mu - ref["mu"]) <= 1e-15 * mu
    pb = problem(w, mu=mu)
    g = pb.g
    v = np.zeros(g.nfull)
    v[g.unknown] = np.random.default_rng(ref["v_seed"]).standard_normal(len(g.unknown))
    assert abs(np.linalg.norm(v) - ref["norm_v"]) <= 1e-12 * ref["norm_v"]
    S = solver(w, mu=mu, variant="aplmm_s", precision="fp32")
    S.pns_build_precond(S.zeros())
    z = S.pns_precond_apply(to_dev(v)).cpu().numpy()
    idx = np.asarray(ref["idx"])
    zo = np.asarray(ref["z"])
    err = np.linalg.norm(z[idx] - zo) / np.linalg.norm(zo)
    print(f"96^3 aPLMM_S fp32 apply, sampled: rel err {err:.2e}; norm {np.linalg.norm(z):.6e} vs {ref['norm_z']:.6e}")
    assert err < 1e-5
    assert abs(np.linalg.norm(z) - ref["norm_z"]) <= 1e-5 * ref["norm_z"]
    S.close()
