"""The persistent, size-binned local-solve launch (pns_autotune / pns_set_tuning): every shape of the
tuning table gives the same preconditioner apply -- the shapes differ only in how a row's dot product is
split over lanes, so FP64 inverses agree to 1e-12 and FP32 / BF16 inverses (per-lane FP32 partial sums,
then one refinement step) to 1e-9, where a shape that skipped or repeated columns would be O(1) off --
and the autotuner returns a valid table with a time for every (bin, shape) that has blocks."""
import numpy as np
import pytest

from gpu_util import problem, random_state, random_vector, rel, solver, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,kw,precision", [("disks64", {}, "fp32"), ("spheres", {"n": 32}, "bf16"),
                                               ("spheres", {"n": 32}, "fp64")])
def test_every_shape_gives_the_same_apply(kind, kw, precision):
    from paper_2510_22077_gb300 import inputs, pns
    w = inputs.make_workload(kind, seed=0, **kw)
    pb = problem(w)
    S = solver(w, variant="gplmm", precision=precision)
    S.pns_build_precond(to_dev(random_state(pb, seed=1, scale=0.1)))
    v = to_dev(random_vector(pb, seed=4))
    z0 = S.pns_precond_apply(v).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-9
    for cfg in range(pns.TUNE_CONFIGS):
        S.pns_set_tuning([cfg] * pns.TUNE_BINS)
        d = rel(S.pns_precond_apply(v).cpu().numpy(), z0)
        print(f"{kind}{kw} {precision} shape {cfg}: rel diff {d:.2e}")
        assert d < tol, (cfg, d)
    table, ms = S.pns_autotune()
    sizes = [len(u) for u in pb.maps.prim_unknowns] + [len(u) for u in pb.maps.dual_unknowns]
    bins = np.searchsorted(pns.TUNE_BIN_EDGES, sizes)
    print(f"{kind}{kw} {precision}: table {table}; ms per bin and shape\n{np.array2string(ms, precision=3)}")
    for b in range(pns.TUNE_BINS):
        assert 0 <= table[b] < pns.TUNE_CONFIGS
        if (bins == b).any():
            assert (ms[b] > 0).all() and ms[b, table[b]] == ms[b].min()
        else:
            assert (ms[b] == 0).all()
    assert rel(S.pns_precond_apply(v).cpu().numpy(), z0) < tol
    S.close()
