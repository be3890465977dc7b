"""pns_precond_apply_static: the preconditioner apply for callers that cannot allocate device memory
when they apply it (another component owns the device allocator, or the footprint has to stay fixed
after start-up).  It must return what pns_precond_apply returns (the same apply body, scratch taken from a
fixed device array instead of the context), call after call, for every variant and local-solve mode,
refuse problems whose scratch does not fit, and leave the device's free memory unchanged.  Collected
last on purpose: a failure here leaves every other test already run."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import problem, random_state, random_vector, rel, solver, to_dev
from paper_2510_22077_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("variant", ["gplmm", "aplmm_ns", "aplmm_s", "ml_only"])
@pytest.mark.parametrize("precision,refine", [("fp64", -1), ("fp32", -1), ("fp32", 0), ("bf16", -1), ("bf16", 0)])
def test_static_apply_matches_allocating_apply(variant, precision, refine):
    w = inputs.make_workload("disks64", seed=0)
    pb = problem(w)
    S = solver(w, variant=variant, precision=precision, refine_steps=refine)
    S.pns_build_precond(to_dev(random_state(pb, seed=1, scale=0.1)))
    info = S.info()
    assert 0 < info["static_apply_bytes"] <= info["static_scratch_capacity"]
    # the two entry points differ only in where their scratch lives; the dual-grid sums use atomics,
    # so the results agree to rounding (1e-12 relative), for two calls in a row
    for k in range(2):
        v = to_dev(random_vector(pb, seed=20 + k))
        z_ref = S.pns_precond_apply(v).cpu().numpy()
        z_st = S.pns_precond_apply_static(v).cpu().numpy()
        assert rel(z_st, z_ref) < 1e-12, (k, rel(z_st, z_ref))
    S.close()


def test_static_apply_with_current_jacobian_in_the_updates():
    # combine = current: the residual updates inside M use the Newton Jacobian FGMRES solves, which only a
    # Newton solve sets; the static apply then runs inside no solve and uses the build matrix, as the
    # context's own apply does outside a solve
    w = inputs.make_workload("disks64", seed=0)
    pb = problem(w)
    S = solver(w, variant="gplmm", precision="fp32", combine="current")
    S.pns_build_precond(to_dev(random_state(pb, seed=1, scale=0.1)))
    v = to_dev(random_vector(pb, seed=5))
    assert rel(S.pns_precond_apply_static(v).cpu().numpy(), S.pns_precond_apply(v).cpu().numpy()) < 1e-12
    S.close()


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
    info = S.info()
    assert info["static_apply_bytes"] > info["static_scratch_capacity"]
    with pytest.raises(pns.PnsError) as e:
        S.pns_precond_apply_static(S.zeros())
    assert e.value.code == -1 and "scratch" in str(e.value)
    S.close()


FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import torch
from gpu_util import problem, random_state, random_vector, rel, solver, to_dev
from paper_2510_22077_gb300 import inputs
w = inputs.make_workload("disks64", seed=0)
pb = problem(w)
S = solver(w, variant="gplmm", precision="fp32")
S.pns_build_precond(to_dev(random_state(pb, seed=1, scale=0.1)))
v = to_dev(random_vector(pb, seed=3))
z = S.zeros()
z_ref = S.pns_precond_apply(v).cpu().numpy()   # loads the apply kernels' code (lazy module loading)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
S.pns_precond_apply_static(v, z)                # first static call of the process
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
S.pns_precond_apply_static(v, z)
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info()[0]
print(free0, free1, free2, rel(z.cpu().numpy(), z_ref))
"""


def test_first_static_call_in_a_fresh_process_allocates_nothing():
    # the address of the static array is taken during set-up, so the first static call of a process
    # finds the array resident: the device's free memory is the same before and after it
    r = subprocess.run([sys.executable, "-c", FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    free0, free1, free2, err = r.stdout.strip().splitlines()[-1].split()
    assert int(free1) == int(free0) and int(free2) == int(free0), (free0, free1, free2)
    assert float(err) < 1e-12
