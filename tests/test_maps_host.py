"""Integer maps (index maps of the domain decomposition) computed by the library on the host,
bit-exact against the oracle, up to the full-size workloads: the 64x64 disk pack, the 96^3 sphere
pack the bench solves, and the 128^3 pack at porosity 0.40.  Runs without a GPU (host code only)."""
import numpy as np
import pytest

from oracle import krylov, mac
from paper_2510_22077_gb300 import inputs, pns


def _compare(w):
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 1.0, (1.0, 0.0, 0.0)), w.periodic)
    m, g = pb.maps, pb.g
    got = pns.pns_maps_host(w.mask, w.labels, w.periodic)
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
    assert got["n_prim"] == m.n_prim and got["n_iface"] == m.n_iface
    return got


def test_maps_host_disk_pack_64():
    _compare(inputs.make_workload("disks64", seed=0))


def test_maps_host_sphere_pack_96_bench_workload():
    """The workload bench.py times: 209 primary grids, 542 contact interfaces."""
    got = _compare(inputs.make_workload("spheres", seed=0, n=96))
    assert got["n_prim"] == 209 and got["n_iface"] == 542


def test_maps_host_sphere_pack_128_porosity_040():
    _compare(inputs.make_workload("spheres", seed=0, n=128, porosity=0.40))


def test_maps_host_rejects_inconsistent_labels():
    mask = np.ones((1, 4, 4), np.uint8)
    labels = np.zeros((1, 4, 4), np.int32)
    with pytest.raises(pns.PnsError):
        pns.pns_maps_host(mask, labels)
