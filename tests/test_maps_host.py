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


def _fixture_labels():
    """The hand-drawn label images of the map and preconditioner fixtures (2D, x-periodic unless
    stated), whose oracle maps are checked against hand-derived values elsewhere in the suite."""
    f = {}
    f["two_pores_channel"] = (np.array([[1, 1, 1, 2, 2, 2]] * 3), (True, False, False))
    lab = np.zeros((6, 6), int)
    lab[:3, :3] = 1
    lab[:3, 3:] = 2
    lab[3:, :] = 3
    f["three_pores_meeting"] = (lab, (False, False, False))
    lab = np.zeros((5, 6), int)
    lab[:2] = 1
    lab[2:, [5, 0, 1]] = 2
    lab[2:, [2, 3, 4]] = 3
    f["pairs_across_the_seam"] = (lab, (True, False, False))
    f["orphan_interface"] = (np.array([[3, 3, 0, 3, 3], [2, 2, 1, 2, 2], [3, 3, 0, 3, 3]]), (True, False, False))
    lab = np.zeros((6, 5), int)
    lab[0:3, :] = 1
    lab[3:6, 2] = 2
    f["dead_end_branch"] = (lab, (True, False, False))
    return f


@pytest.mark.parametrize("name", sorted(_fixture_labels()))
@pytest.mark.parametrize("n_dilate,n_tag", [(1, 1), (2, 1), (1, 2)])
def test_maps_host_hand_fixtures(name, n_dilate, n_tag):
    lab, per = _fixture_labels()[name]
    lab = np.asarray(lab, np.int32)[None]
    mask = (lab > 0).astype(np.uint8)
    pb = krylov.Problem(mask, lab, mac.Params(1.0, 1.0, (1.0, 0.0, 0.0)), per, n_dilate, n_tag)
    m, g = pb.maps, pb.g
    got = pns.pns_maps_host(mask, lab, per, n_dilate, n_tag)
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
    assert got["n_dropped_labels"] == len(m.dropped_labels)


@pytest.mark.parametrize("kind,kw,seed", [("tiny3d", dict(n=8), 1), ("tiny3d", dict(n=10, porosity=0.55), 2),
                                          ("tiny2d", dict(n=20, n_disks=3), 5), ("spheres", dict(n=32), 0)])
@pytest.mark.parametrize("n_dilate,n_tag", [(1, 1), (2, 2), (0, 1)])
def test_maps_host_seeded_images_all_depths(kind, kw, seed, n_dilate, n_tag):
    w = inputs.make_workload(kind, seed=seed, **kw)
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, 1.0, (1.0, 0.0, 0.0)), w.periodic, n_dilate, n_tag)
    m, g = pb.maps, pb.g
    got = pns.pns_maps_host(w.mask, w.labels, w.periodic, n_dilate, n_tag)
    assert np.array_equal(got["cell_prim"], m.cell_prim) and np.array_equal(got["cell_iface"], m.cell_iface)
    for d in range(g.dim):
        assert np.array_equal(got["face_class"][d], m.face_class[d])
        assert np.array_equal(got["tags"][d], m.tags[d])
    cnt = np.zeros(g.nfull, np.int32)
    for u in m.dual_unknowns:
        cnt[u] += 1
    assert np.array_equal(got["dual_count"], cnt)
