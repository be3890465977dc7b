"""Hand-drawn fixtures for the domain-decomposition maps (Sec. 3.2.1-3.2.2, Sec. 4).  Every expected
value below was worked out by hand from the rules (not produced by running the oracle)."""
import numpy as np

from oracle import mac
from oracle.maps import F_FACE, NOT_UNKNOWN, build_maps


def _maps(labels, periodic, n_dilate=1, n_tag=1):
    lab = np.asarray(labels, dtype=np.int32)[None]
    mask = (lab > 0).astype(np.uint8)
    g = mac.Grid(mask, periodic)
    pins = mac.pressure_pins(g)
    return g, build_maps(g, lab, pins, n_dilate, n_tag), pins


def test_two_pores_periodic_channel():
    # 2D 3 x 6, x-periodic; label 1 in columns 0-2, label 2 in columns 3-5.
    lab = [[1, 1, 1, 2, 2, 2]] * 3
    g, m, pins = _maps(lab, (True, False, False), n_dilate=1)
    assert list(pins) == [0]
    # label-1 cells next to a label-2 cell: column 2 (right) and column 0 (wrap to column 5); both are
    # pair (1, 2), so they form one interface although they are not connected
    assert m.n_iface == 1
    ifc = m.cell_iface.reshape(3, 6)
    assert (ifc[:, [0, 2]] == 0).all() and (ifc[:, [1, 3, 4, 5]] == -1).all()
    assert m.n_prim == 2
    cp = m.cell_prim.reshape(3, 6)
    assert (cp[:, 1] == 0).all() and (cp[:, 3:] == 1).all() and (cp[:, [0, 2]] == -1).all()
    # x-faces (low face of each cell): columns 0..5 -> p1 p0 p0 p1 p1 p1 in every row
    fx = m.face_class[0].reshape(3, 6)
    assert (fx == np.array([1, 0, 0, 1, 1, 1])).all()
    # y-faces: row 0 is the wall; rows 1,2: f in interface columns 0 and 2
    fy = m.face_class[1].reshape(3, 6)
    assert (fy[0] == NOT_UNKNOWN).all()
    assert (fy[1:] == np.array([F_FACE, 0, F_FACE, 1, 1, 1])).all()
    assert [list(c) for c in m.C] == [[0], [0]]
    # tags: f faces; x-faces in columns 0,1,2,3 (an x-neighbour in the other grid);
    #       y-faces in columns 1 (f on both sides), 3 (f at column 2), 5 (f at column 0)
    tx = m.tags[0].reshape(3, 6)
    assert (tx == np.array([1, 1, 1, 1, 0, 0], bool)).all()
    ty = m.tags[1].reshape(3, 6)
    assert not ty[0].any()
    assert (ty[1:] == np.array([1, 1, 1, 1, 0, 1], bool)).all()
    # dual grid = columns {0, 2} dilated once with wrap: columns {5, 0, 1, 2, 3}
    assert set(np.asarray(m.dual_cells[0]) % 6) == {5, 0, 1, 2, 3}
    assert len(m.dual_cells[0]) == 15
    # unknowns: all 18 x-faces (each has a flanking cell in the set), y-faces of the 5 columns in
    # rows 1,2 (10), 15 cells
    assert len(m.dual_unknowns[0]) == 18 + 10 + 15


def test_component_reading_splits_the_pair():
    lab = [[1, 1, 1, 2, 2, 2]] * 3
    lab = np.asarray(lab, dtype=np.int32)[None]
    g = mac.Grid((lab > 0).astype(np.uint8), (True, False, False))
    m = build_maps(g, lab, mac.pressure_pins(g), 2, 1, iface_mode="component")
    assert m.n_iface == 2
    ifc = m.cell_iface.reshape(3, 6)
    assert (ifc[:, 0] == 0).all() and (ifc[:, 2] == 1).all()
    # dual grid 0 = column 0 dilated twice with wrap: columns {4,5,0,1,2}; dual 1: {0,1,2,3,4}
    assert set(np.asarray(m.dual_cells[0]) % 6) == {4, 5, 0, 1, 2}
    assert set(np.asarray(m.dual_cells[1]) % 6) == {0, 1, 2, 3, 4}


def test_three_pores_meeting():
    # 6 x 6, not periodic.  rows 0-2: label 1 (cols 0-2) | label 2 (cols 3-5); rows 3-5: label 3.
    lab = np.zeros((6, 6), int)
    lab[:3, :3] = 1
    lab[:3, 3:] = 2
    lab[3:, :] = 3
    g, m, _ = _maps(lab, (False, False, False))
    # interfaces by lowest cell index: A = pair (1,2) cells {2, 8, 14} (cell 14 = (2,2) touches 2 and
    # 3 -> smaller partner 2), B = pair (1,3) {12, 13}, C = pair (2,3) {15, 16, 17}
    assert m.n_iface == 3
    assert [sorted(c.tolist()) for c in m.iface_cells] == [[2, 8, 14], [12, 13], [15, 16, 17]]
    assert [tuple(p) for p in m.iface_pair] == [(1, 2), (1, 3), (2, 3)]
    cp = m.cell_prim.reshape(6, 6)
    assert (cp[:2, :2] == 0).all() and (cp[:2, 3:] == 1).all() and (cp[3:, :] == 2).all()
    assert [list(c) for c in m.C] == [[0, 1], [0, 2], [0, 1, 2]]
    fx = m.face_class[0].reshape(6, 6)
    fy = m.face_class[1].reshape(6, 6)
    assert fx[2, 1] == F_FACE and fx[2, 2] == F_FACE and fx[2, 3] == F_FACE   # along row 2
    assert fy[3, 2] == 2                       # between (2,2) in A and (3,2) in p2
    assert fx[0, 0] == NOT_UNKNOWN             # left wall, not periodic
    assert fx[0, 3] == 1                       # between (0,2) in A and (0,3) in p1


def test_interfaces_grouped_by_pair_across_the_seam():
    # 4 x 6, x-periodic. rows 0-1 label 1; rows 2-3: label 2 in columns {5, 0, 1}, label 3 in {2, 3, 4}
    lab = np.zeros((4, 6), int)
    lab[:2] = 1
    lab[2:, [5, 0, 1]] = 2
    lab[2:, [2, 3, 4]] = 3
    g, m, _ = _maps(lab, (True, False, False))
    # pair (1,2): cells 6, 7, 11 (11 reaches 6 through the seam); pair (1,3): 8, 9, 10;
    # pair (2,3): label-2 cells next to label 3: 13, 19 (column 1) and 17, 23 (column 5)
    assert [sorted(c.tolist()) for c in m.iface_cells] == [[6, 7, 11], [8, 9, 10], [13, 17, 19, 23]]
    assert m.n_prim == 3
    cp = m.cell_prim.reshape(4, 6)
    assert (cp[0] == 0).all() and cp[2, 0] == 1 and cp[3, 0] == 1 and (cp[2:, 2:5] == 2).all()
    assert (m.cell_prim[[13, 19, 17, 23]] == -1).all()


def test_dropped_pore_and_pins():
    # a label whose every cell is an interface cell is dropped; two void components -> two pins
    lab = np.zeros((3, 7), int)
    lab[0, :] = 2
    lab[0, 3] = 1                 # single label-1 cell between label-2 cells: all of label 1 is interface
    lab[2, 1:3] = 3               # separate component (row 1 is solid)
    g, m, pins = _maps(lab, (True, False, False))
    assert list(pins) == [0, 15]
    assert list(m.dropped_labels) == [1]
    assert sorted(np.flatnonzero(m.cell_iface >= 0).tolist()) == [3]
    assert m.n_iface == 1 and m.n_prim == 2          # labels 2 and 3 survive, numbered 0 and 1
    assert (m.cell_prim[[0, 1, 2, 4, 5, 6]] == 0).all()
    # component 2 has one label (3) and no interface: it is a primary grid containing its pin
    assert m.cell_prim[15] == 1 and m.cell_prim[16] == 1
    assert [list(c) for c in m.C] == [[0], []]
