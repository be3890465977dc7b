"""pns_precond_apply_static: the preconditioner apply for callers that cannot allocate device memory
when they apply it.  It must return what pns_precond_apply returns (same arithmetic, scratch taken
from a fixed device array instead of the context), call after call, and refuse problems whose
scratch does not fit.  Collected last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

from gpu_util import problem, random_state, random_vector, rel, solver, to_dev
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,kw,precision", [("disks64", {}, "fp64"), ("disks64", {}, "fp32"),
                                               ("tiny3d", {"n": 10}, "bf16")])
def test_static_apply_matches_allocating_apply(kind, kw, precision):
    w = inputs.make_workload(kind, seed=0, **kw)
    pb = problem(w)
    S = solver(w, variant="gplmm", precision=precision)
    S.pns_build_precond(to_dev(random_state(pb, seed=1, scale=0.1)))
    # the two entry points differ only in where their scratch lives; the dual-grid sums use atomics,
    # so the results agree to rounding (1e-12 relative), for two calls in a row
    for k in range(2):
        v = to_dev(random_vector(pb, seed=20 + k))
        z_ref = S.pns_precond_apply(v).cpu().numpy()
        z_st = S.pns_precond_apply_static(v).cpu().numpy()
        assert rel(z_st, z_ref) < 1e-12, (k, rel(z_st, z_ref))


def test_static_apply_rejects_problems_beyond_its_scratch():
    from paper_2510_22077_gb300 import pns
    # 512 x 512 void, labels on 8 x 8 squares (small local blocks, cheap to build); the full layout
    # has 3 * 262144 entries, whose five FP64 scratch vectors alone exceed the 24 MiB array
    n = 512
    mask = np.ones((1, n, n), np.uint8)
    jj, ii = np.mgrid[0:n, 0:n]
    labels = (1 + (jj // 8) * (n // 8) + ii // 8).astype(np.int32)[None]
    S = pns.Solver(mask, labels, 1.0, 1.0, (1.0, 0.0, 0.0), variant="ml_only", precision="fp32")
    S.pns_build_precond(S.zeros())
    with pytest.raises(pns.PnsError) as e:
        S.pns_precond_apply_static(S.zeros())
    assert e.value.code == -1 and "scratch" in str(e.value)
