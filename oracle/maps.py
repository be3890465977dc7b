"""Domain decomposition index maps (Sec. 3.2.1 and the permutation paragraph of Sec. 3.2.2; Sec. 4).

Readings fixed where the paper is silent:

* Contact interfaces (Sec. 3.2.2, "thinnest 4-/6-connected collection of pixels that separate two
  primary grids", one interface Gamma_ij per pair of adjacent primary grids): a void cell of label a
  is an interface cell when a face-neighbour (wrapping along periodic axes) is void with a label
  b > a; its pair is (a, smallest such b).  The interface of a pair is the set of all interface cells
  with that pair (connected or not), numbered by its lowest cell index.  iface_mode="component"
  splits each pair's set into face-connected components instead (an alternative reading kept for
  comparison: on 3D sphere packs it gives ~4x more, much smaller interfaces and a far weaker
  preconditioner).
* Primary grid of label a = its cells that are not interface cells; labels that keep at least one
  cell are numbered in ascending label order (others are dropped and counted).
* Faces (Sec. 3.2.2): a face unknown with at least one flanking cell in primary grid i belongs to i
  (two different primary grids never flank one face); a face flanked by two interface cells is an
  interface face ("f").
* C^{p_i} = interfaces owning a cell face-adjacent to a cell of p_i (sorted ascending).
* Coarse interfaces: an interface adjacent to no primary grid (possible at 3D junctions, where all its
  neighbours are interface cells of other pairs) has no shape vector, so its column of P^ would be
  the bare cell indicator and A^o singular; only interfaces in some C^{p_i} get a coarse unknown, in
  ascending order.  The cells of the others get zero from M_G (like interface faces).
* Dual grid j (Sec. 3.2.1): cells of interface j dilated `n_dilate` times (default 1: the dual grids
  then cover 20-25% of the unknowns, inside the 10-30% the paper states in Sec. 7) over
  face-neighbouring void cells; its unknowns are those cells and every face unknown with a flanking
  cell among them.
* gPLMM tags (Sec. 4, "faces within a few layers of each contact interface", 3-point stencil):
  every f face, plus every primary face whose same-component neighbour along some axis is an unknown
  outside its own primary grid; `n_tag` > 1 adds faces adjacent (same rule) to tagged faces.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mac import void_adjacency as mac_void_adjacency

F_FACE = -1        # face class of interface (f) faces
NOT_UNKNOWN = -2


class Maps:
    pass


def build_maps(g, labels, pins, n_dilate=1, n_tag=1, iface_mode="pair"):
    L = np.asarray(labels).ravel().astype(np.int64)
    if np.any(L[g.void] < 1) or np.any(L[~g.void] != 0):
        raise ValueError("labels must be >= 1 on void cells and 0 on solid cells")
    m = Maps()
    m.pins = np.asarray(pins)
    # --- interface cells and their pairs
    big = np.iinfo(np.int64).max
    partner = np.full(g.ncell, big)
    for a in range(g.dim):
        for t in (0, 1):
            n = g.nb[a][t]
            ok = g.void & (n >= 0)
            ns = np.where(ok, n, 0)
            ok &= g.void[ns]
            cand = np.where(ok & (L[ns] > L), L[ns], big)
            partner = np.minimum(partner, cand)
    is_if = g.void & (partner < big)
    # --- interfaces: components of same-pair interface cells
    from scipy.sparse.csgraph import connected_components
    adj = mac_void_adjacency(g).tocoo()
    if iface_mode == "component":
        same = is_if[adj.row] & is_if[adj.col] & (L[adj.row] == L[adj.col]) & (partner[adj.row] == partner[adj.col])
        sub = sp.coo_matrix((np.ones(int(same.sum())), (adj.row[same], adj.col[same])), shape=(g.ncell, g.ncell))
        _, comp = connected_components(sub.tocsr(), directed=False)
    else:
        # one interface per label pair (a, b): all interface cells with that pair, connected or not
        key = np.where(is_if, L * (int(L.max()) + 2) + np.where(is_if, partner, 0), -1)
        _, comp = np.unique(key, return_inverse=True)
    iface = np.full(g.ncell, -1, np.int64)
    cells_if = np.flatnonzero(is_if)                     # ascending
    uniq, first = np.unique(comp[cells_if], return_index=True)   # first = lowest cell of each component
    order = np.argsort(cells_if[first], kind="stable")   # number components by their lowest cell
    rank = np.empty(len(uniq), np.int64)
    rank[order] = np.arange(len(uniq))
    iface[cells_if] = rank[np.searchsorted(uniq, comp[cells_if])]
    n_if = len(uniq)
    m.n_iface = n_if
    m.cell_iface = iface
    m.iface_pair = np.zeros((n_if, 2), np.int64)
    srt = cells_if[np.argsort(iface[cells_if], kind="stable")]
    m.iface_cells = np.split(srt, np.cumsum(np.bincount(iface[cells_if], minlength=n_if))[:-1]) if n_if else []
    for j in range(n_if):
        c = m.iface_cells[j][0]
        m.iface_pair[j] = (L[c], partner[c])
    # --- primary grids
    prim_cells = g.void & ~is_if
    labs = np.unique(L[prim_cells])
    all_labs = np.unique(L[g.void])
    m.dropped_labels = np.setdiff1d(all_labs, labs)
    lab2p = {int(v): i for i, v in enumerate(labs)}
    cell_prim = np.full(g.ncell, -1, np.int64)
    for c in np.flatnonzero(prim_cells):
        cell_prim[c] = lab2p[int(L[c])]
    m.n_prim = len(labs)
    m.cell_prim = cell_prim
    # --- face classes
    m.face_class = []
    for d in range(g.dim):
        lo = g.nb[d][0]
        los = np.where(lo >= 0, lo, 0)
        pl = np.where(lo >= 0, cell_prim[los], -1)
        ph = cell_prim
        clash = g.face_unknown[d] & (pl >= 0) & (ph >= 0) & (pl != ph)
        if np.any(clash):
            raise RuntimeError("a face is flanked by two different primary grids")
        cls = np.where(ph >= 0, ph, np.where(pl >= 0, pl, F_FACE))
        m.face_class.append(np.where(g.face_unknown[d], cls, NOT_UNKNOWN))
    # --- C^{p_i}
    cp = [set() for _ in range(m.n_prim)]
    for c in np.flatnonzero(is_if):
        for a in range(g.dim):
            for t in (0, 1):
                n = g.nb[a][t][c]
                if n >= 0 and cell_prim[n] >= 0:
                    cp[cell_prim[n]].add(int(iface[c]))
    m.C = [np.array(sorted(s), np.int64) for s in cp]
    used = sorted(set(int(j) for C in m.C for j in C))
    m.coarse_ifaces = np.array(used, np.int64)
    m.coarse_of_iface = np.full(m.n_iface, -1, np.int64)
    m.coarse_of_iface[m.coarse_ifaces] = np.arange(len(used))
    # --- unknown lists (global indices, ascending: faces by axis, then cells)
    own_all = np.concatenate(m.face_class + [np.where(cell_prim >= 0, cell_prim, NOT_UNKNOWN)])
    glob = np.flatnonzero(own_all >= 0)                   # ascending global index
    srt = glob[np.argsort(own_all[glob], kind="stable")]  # grouped by primary grid, ascending inside
    m.prim_unknowns = np.split(srt, np.cumsum(np.bincount(own_all[glob], minlength=m.n_prim))[:-1])
    m.f_faces = np.concatenate([g.fidx(d, np.flatnonzero(m.face_class[d] == F_FACE)) for d in range(g.dim)])
    # --- dual grids
    adj_csr = mac_void_adjacency(g)
    m.dual_unknowns = []
    m.dual_cells = []
    for j in range(n_if):
        cells = m.iface_cells[j]
        for _ in range(n_dilate):
            nbrs = adj_csr[cells].indices
            cells = np.union1d(cells, nbrs)
        inset = np.zeros(g.ncell, bool)
        inset[cells] = True
        parts = []
        for d in range(g.dim):
            # faces stored at c (low face of c) and at c + e_d (high face of c) for every c in the set
            hi = g.nb[d][1][cells]
            cand = np.union1d(cells, hi[hi >= 0])
            parts.append(g.fidx(d, cand[g.face_unknown[d][cand]]))
        parts.append(g.pidx(cells))
        m.dual_unknowns.append(np.concatenate(parts))
        m.dual_cells.append(cells)
    # --- gPLMM tags
    tags = [np.zeros(g.ncell, bool) for _ in range(g.dim)]
    for d in range(g.dim):
        cls = m.face_class[d]
        tags[d] |= cls == F_FACE
        for a in range(g.dim):
            for t in (0, 1):
                ix, ok = g.face_at(d, g.nb[a][t])
                other = ok & (m.face_class[d][ix] != cls)
                tags[d] |= (cls >= 0) & other
    for _ in range(n_tag - 1):
        new = [t.copy() for t in tags]
        for d in range(g.dim):
            cls = m.face_class[d]
            for a in range(g.dim):
                for t in (0, 1):
                    ix, ok = g.face_at(d, g.nb[a][t])
                    new[d] |= (cls >= 0) & ok & tags[d][ix]
        tags = new
    m.tags = tags
    # --- owner of every global unknown: primary id, -1 interface cell, -3 f face, -2 not unknown
    owner = np.full(g.nfull, NOT_UNKNOWN, np.int64)
    for d in range(g.dim):
        cls = m.face_class[d]
        owner[g.fidx(d, np.arange(g.ncell))] = np.where(cls == F_FACE, -3, cls)
    cellown = np.where(cell_prim >= 0, cell_prim, np.where(iface >= 0, -1, NOT_UNKNOWN))
    owner[g.pidx(np.arange(g.ncell))] = cellown
    m.owner = owner
    return m


def dual_fraction(g, m):
    """Fraction f^d of unknowns covered by at least one dual grid (Sec. 7 cost model: 10-30%)."""
    cov = np.zeros(g.nfull, bool)
    for u in m.dual_unknowns:
        cov[u] = True
    return cov.sum() / len(g.unknown)
