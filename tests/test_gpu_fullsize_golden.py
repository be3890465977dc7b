"""Parity of one preconditioner apply at the full size of the benchmark (the 96^3 sphere pack, 1.15 M
unknowns, blocks of up to 43,863 unknowns), on sampled outputs, against FP64 oracle values stored by
tests/golden/make_spheres96_applies.py (the oracle's build takes minutes, too slow for a test):
aPLMM_S with FP32 and BF16 local inverses, and gPLMM at a seeded synthetic wind with FP32 local
inverses.  The samples cover every decile of primary-grid size, the largest primary grid, the
interface unknowns and the dual-grid unknowns; the error of each group is printed."""
import json
import os

import numpy as np
import pytest

from gpu_util import problem, solver, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GROUPS = {**{d: f"size decile {d}" for d in range(10)}, 10: "largest grid", 11: "interface", 12: "dual"}


@pytest.fixture(scope="module")
def c2():
    from paper_2510_22077_gb300 import inputs
    w = inputs.make_workload("spheres", seed=0, n=96)
    mu = inputs.mu_kozeny_carman(w.mask, 1.0)
    return w, mu, problem(w, mu=mu)


@pytest.mark.parametrize("variant,precision,tol", [("aplmm_s", "fp32", 1e-5), ("aplmm_s", "bf16", 2e-2),
                                                   ("gplmm", "fp32", 1e-5)])
def test_precond_apply_full_size_sampled(c2, variant, precision, tol):
    from paper_2510_22077_gb300 import inputs
    w, mu, pb = c2
    ref = json.load(open(os.path.join(GOLDEN, f"spheres96_{variant}_apply.json")))
    assert abs(mu - ref["mu"]) <= 1e-15 * mu
    g = pb.g
    v = np.zeros(g.nfull)
    v[g.unknown] = np.random.default_rng(ref["v_seed"]).standard_normal(len(g.unknown))
    assert abs(np.linalg.norm(v) - ref["norm_v"]) <= 1e-12 * ref["norm_v"]
    x_lin = np.zeros(g.nfull)
    if variant == "gplmm":
        x_lin = inputs.synthetic_wind(w.mask.shape, seed=ref["wind_seed"])
        keep = np.zeros(g.nfull, bool)
        keep[g.unknown] = True
        x_lin[~keep] = 0.0
    S = solver(w, mu=mu, variant=variant, precision=precision)
    S.pns_build_precond(to_dev(x_lin))
    z = S.pns_precond_apply(to_dev(v)).cpu().numpy()
    S.close()
    idx = np.asarray(ref["idx"])
    grp = np.asarray(ref["group"])
    zo = np.asarray(ref["z"])
    zs = z[idx]
    err = np.linalg.norm(zs - zo) / np.linalg.norm(zo)
    lines = [f"96^3 {variant} {precision} apply, {len(idx)} sampled outputs: rel err {err:.2e} (bar {tol:g}); "
             f"norm {np.linalg.norm(z):.6e} vs oracle {ref['norm_z']:.6e}"]
    worst = 0.0
    for gq, name in GROUPS.items():
        m = grp == gq
        if not m.any():
            continue
        eg = np.linalg.norm(zs[m] - zo[m]) / max(np.linalg.norm(zo[m]), 1e-300)
        worst = max(worst, eg)
        lines.append(f"  {name:>14}: {m.sum():5d} outputs, rel err {eg:.2e}")
    print("\n".join(lines))
    assert err < tol
    assert abs(np.linalg.norm(z) - ref["norm_z"]) <= tol * ref["norm_z"]
    assert worst < 10 * tol
