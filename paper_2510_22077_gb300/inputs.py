"""Seeded synthetic porous images, pore labels and Reynolds-number helpers.

This module makes the inputs of the solver and nothing else: binary void masks shaped like the paper's
porous samples (disk packs as in PD4/GLD4, sphere packs as in Granular, a thresholded Gaussian random
field as a stand-in for a sandstone), a watershed labelling of the void into pores (the primary-grid
decomposition of Sec. 3.2.1 takes these labels as given), and the Reynolds-number definition of
Sec. 6 (Re = rho U l / mu with U = U_D / phi and l = V_s / A_w).  It holds none of the solver's
arithmetic: no discretisation, no preconditioner, no Krylov step.

Image convention: arrays of shape (nz, ny, nx), C order, x fastest; a 2D image has nz == 1.
mask == 1 marks void (fluid) cells.  Axis 0 of the solver is x, axis 1 is y, axis 2 is z.
`periodic` is a tuple of three booleans (x, y, z); the default workloads are periodic in x only.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np
from scipy import ndimage

X_PERIODIC = (True, False, False)


# ----------------------------------------------------------------------------------------------
# geometry generators
# ----------------------------------------------------------------------------------------------
def _wrap_delta(a, b, n):
    """Signed distance a - b on a ring of length n (minimum image)."""
    d = (a - b) % n
    return np.where(d > n / 2, d - n, d)


def disk_pack_2d(n: int = 64, n_disks: int = 12, rmin: float = 4.0, rmax: float = 8.0, seed: int = 0,
                 max_tries: int = 200000) -> np.ndarray:
    """Non-overlapping disks with radius U[rmin, rmax] and uniform centres, x-periodic, clipped at the
    y walls (rejection sampling).  Returns the void mask, shape (1, n, n), uint8."""
    rng = np.random.default_rng(seed)
    disks = []
    tries = 0
    while len(disks) < n_disks:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("disk packing did not finish; lower n_disks or radii")
        r = rng.uniform(rmin, rmax)
        cx, cy = rng.uniform(0, n), rng.uniform(0, n)
        ok = True
        for (qx, qy, qr) in disks:
            dx = _wrap_delta(cx, qx, n)
            if dx * dx + (cy - qy) ** 2 < (r + qr) ** 2:
                ok = False
                break
        if ok:
            disks.append((cx, cy, r))
    y, x = np.mgrid[0:n, 0:n] + 0.5
    solid = np.zeros((n, n), bool)
    for (cx, cy, r) in disks:
        dx = _wrap_delta(x, cx, n)
        solid |= dx * dx + (y - cy) ** 2 < r * r
    return (~solid).astype(np.uint8)[None]


def sphere_pack_3d(n: int = 96, rmin: float = 6.0, rmax: float = 10.0, porosity: float = 0.35,
                   seed: int = 0) -> np.ndarray:
    """Spheres with radius U[rmin, rmax] at uniform random centres (x-periodic, overlap allowed),
    added one at a time until the porosity first drops to `porosity` or below.  Returns (n, n, n)."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((n, n, n), bool)
    zc, yc, xc = (np.arange(n) + 0.5,) * 3
    target = porosity * n ** 3
    void = float(n ** 3)
    while void > target:
        r = rng.uniform(rmin, rmax)
        cx, cy, cz = rng.uniform(0, n, size=3)
        # bounding box in y and z (walls clip), x wraps
        zlo, zhi = max(0, int(np.floor(cz - r))), min(n, int(np.ceil(cz + r)) + 1)
        ylo, yhi = max(0, int(np.floor(cy - r))), min(n, int(np.ceil(cy + r)) + 1)
        dz = zc[zlo:zhi, None, None] - cz
        dy = yc[None, ylo:yhi, None] - cy
        dx = _wrap_delta(xc[None, None, :], cx, n)
        ball = dz * dz + dy * dy + dx * dx < r * r
        sub = solid[zlo:zhi, ylo:yhi, :]
        void -= np.count_nonzero(ball & ~sub)
        sub |= ball
    return (~solid).astype(np.uint8)


def gaussian_field_3d(n: int = 256, corr_len: float = 8.0, porosity: float = 0.20, seed: int = 0) -> np.ndarray:
    """Threshold of a Gaussian random field: white noise smoothed by FFT with a Gaussian kernel whose
    covariance is exp(-r^2 / (2 l^2)) (kernel std l / sqrt(2)); void = field below its `porosity`
    quantile.  Returns (n, n, n) uint8."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n) * 2 * np.pi
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    s = corr_len / np.sqrt(2.0)
    filt = np.exp(-0.5 * s * s * (kx * kx + ky * ky + kz * kz))
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    thr = np.quantile(field, porosity)
    return (field < thr).astype(np.uint8)


def channel(nx: int, ny: int, nz: int = 1, width: int | None = None) -> np.ndarray:
    """Straight channel along x: void rows 0..width-1 in y (whole z), walls above (solid) and the
    y box walls.  Returns (nz, ny, nx) uint8."""
    w = ny if width is None else width
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, :w, :] = 1
    return m


# ----------------------------------------------------------------------------------------------
# connectivity helpers (periodic seams)
# ----------------------------------------------------------------------------------------------
def _face_structure(ndim):
    return ndimage.generate_binary_structure(ndim, 1)


def _squeeze2d(mask):
    """View of the image as 2D (ny, nx) when nz == 1, else 3D; returns (array, axis map)."""
    if mask.shape[0] == 1:
        return mask[0], {0: 1, 1: 0}          # solver axis -> numpy axis of the 2D array
    return mask, {0: 2, 1: 1, 2: 0}


def void_components(mask: np.ndarray, periodic=X_PERIODIC):
    """Face-connected components of the void with wrap along periodic axes.
    Returns (labels image int32 (0 = solid), count)."""
    arr, amap = _squeeze2d(np.asarray(mask).astype(bool))
    lab, n = ndimage.label(arr, structure=_face_structure(arr.ndim))
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax_solver, ax_np in amap.items():
        if not periodic[ax_solver]:
            continue
        lo = np.take(lab, 0, axis=ax_np)
        hi = np.take(lab, arr.shape[ax_np] - 1, axis=ax_np)
        both = (lo > 0) & (hi > 0)
        for a, b in zip(lo[both].ravel(), hi[both].ravel()):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(n + 1)])
    uniq, comp = np.unique(roots, return_inverse=True)
    comp = comp.astype(np.int32)  # root 0 (solid) maps to 0 because roots[0] == 0 is the smallest
    out = comp[lab]
    return out.reshape(mask.shape), len(uniq) - 1


def percolating_void(mask: np.ndarray, periodic=X_PERIODIC):
    """Drop void components that do not wrap around the periodic x axis (they carry no net flow).
    A component percolates when its lift to the x-unrolled image is not simply x-bounded: some
    cycle through the x seam has non-zero winding.  Returns (new mask, fraction of void dropped)."""
    m = np.asarray(mask).astype(bool)
    arr, amap = _squeeze2d(m)
    lab, n = ndimage.label(arr, structure=_face_structure(arr.ndim))
    # graph over non-periodic components; x-seam edges carry winding +1, other periodic seams 0
    edges = []
    for ax_solver, ax_np in amap.items():
        if not periodic[ax_solver]:
            continue
        lo = np.take(lab, 0, axis=ax_np)
        hi = np.take(lab, arr.shape[ax_np] - 1, axis=ax_np)
        both = (lo > 0) & (hi > 0)
        pairs = set(zip(hi[both].ravel().tolist(), lo[both].ravel().tolist()))
        w = 1 if ax_solver == 0 else 0
        edges += [(a, b, w) for (a, b) in pairs]
    adj = {a: [] for a in range(1, n + 1)}
    for a, b, w in edges:
        adj[a].append((b, w))
        adj[b].append((a, -w))
    pot = {}
    perc_root = {}
    for s in range(1, n + 1):
        if s in pot:
            continue
        pot[s] = 0
        stack, members, wraps = [s], [s], False
        while stack:
            a = stack.pop()
            for b, w in adj[a]:
                if b not in pot:
                    pot[b] = pot[a] + w
                    stack.append(b)
                    members.append(b)
                elif pot[b] != pot[a] + w:
                    wraps = True
        for a in members:
            perc_root[a] = wraps
    keep = np.zeros(n + 1, bool)
    for a, v in perc_root.items():
        keep[a] = v
    newarr = keep[lab] & arr
    dropped = 1.0 - newarr.sum() / max(1, arr.sum())
    return newarr.astype(np.uint8).reshape(mask.shape), float(dropped)


# ----------------------------------------------------------------------------------------------
# pore labelling: periodic EDT -> plateau markers -> priority-flood watershed
# ----------------------------------------------------------------------------------------------
def _pad_periodic(arr, amap, periodic, width, solid_value):
    """Pad: wrap along periodic axes, constant `solid_value` (walls) along the others."""
    pads = [(0, 0)] * arr.ndim
    out = arr
    for ax_solver, ax_np in amap.items():
        pw = [(0, 0)] * arr.ndim
        pw[ax_np] = (width, width)
        if periodic[ax_solver]:
            out = np.pad(out, pw, mode="wrap")
        else:
            out = np.pad(out, pw, mode="constant", constant_values=solid_value)
        pads[ax_np] = (width, width)
    return out, pads


def _crop(arr, pads):
    sl = tuple(slice(a, arr.shape[i] - b) for i, (a, b) in enumerate(pads))
    return arr[sl]


def distance_to_solid(mask: np.ndarray, periodic=X_PERIODIC) -> np.ndarray:
    """Euclidean distance of each void cell to the nearest solid cell (box walls count as solid,
    periodic axes wrap).  Shape of `mask`, float64."""
    arr, amap = _squeeze2d(np.asarray(mask).astype(bool))
    width = max(arr.shape)
    padded, pads = _pad_periodic(arr, amap, periodic, width, False)
    d = ndimage.distance_transform_edt(padded)
    return _crop(d, pads).reshape(mask.shape)


@dataclass
class Labelling:
    labels: np.ndarray      # int32, same shape as mask; 0 on solid, >= 1 on void
    n_labels: int
    window: int             # marker window half-width that was chosen
    dist: np.ndarray        # distance map used as the flooding height


def _markers(dist, arr, amap, periodic, w):
    padded, pads = _pad_periodic(dist, amap, periodic, w, 0.0)
    mx = ndimage.maximum_filter(padded, size=2 * w + 1, mode="constant", cval=0.0)
    mx = _crop(mx, pads)
    peak = arr & (dist >= mx) & (dist >= 1.0)
    return peak


def _nms_markers(dist, arr, amap, periodic, dmin, rmin=1.0):
    """Local maxima of the distance (3^d neighbourhood), accepted in order of decreasing distance
    (ties: lowest linear index) when farther than dmin from every accepted marker (minimum image
    along periodic axes).  Returns the accepted linear indices."""
    padded, pads = _pad_periodic(dist, amap, periodic, 1, 0.0)
    mx = _crop(ndimage.maximum_filter(padded, size=3, mode="constant", cval=0.0), pads)
    cand = np.flatnonzero((dist >= mx) & arr & (dist >= rmin))
    cand = cand[np.argsort(-dist.ravel()[cand], kind="stable")]
    coords = np.array(np.unravel_index(cand, arr.shape)).T.astype(np.float64)
    ext = np.array(arr.shape, np.float64)
    wrap = np.array([periodic[[k for k, v in amap.items() if v == ax][0]] for ax in range(arr.ndim)])
    acc = np.zeros((0, arr.ndim))
    keep = []
    for k in range(len(cand)):
        if len(acc):
            dlt = np.abs(acc - coords[k])
            dlt = np.where(wrap, np.minimum(dlt, ext - dlt), dlt)
            if np.min((dlt * dlt).sum(axis=1)) < dmin * dmin:
                continue
        acc = np.vstack([acc, coords[k]])
        keep.append(cand[k])
    return np.array(keep, np.int64)


def _flood(arr, amap, periodic, flat_d, seeds_lab):
    """Priority flood of labels over the face-connected void (highest distance first; ties by
    insertion order).  seeds_lab: flat label array with markers > 0."""
    shape = arr.shape
    lab = seeds_lab.copy()
    flat_void = arr.ravel()
    strides = np.array([int(np.prod(shape[a + 1:])) for a in range(len(shape))])
    wraps = {ax_np: periodic[ax_s] for ax_s, ax_np in amap.items()}
    heap = []
    counter = 0
    for c in np.flatnonzero(lab > 0):
        heapq.heappush(heap, (-flat_d[c], counter, int(c)))
        counter += 1
    while heap:
        _, _, c = heapq.heappop(heap)
        lc = lab[c]
        idx = np.unravel_index(c, shape)
        for ax in range(len(shape)):
            for sgn in (-1, 1):
                v = idx[ax] + sgn
                if v < 0 or v >= shape[ax]:
                    if not wraps[ax]:
                        continue
                    v %= shape[ax]
                nb = c + (v - idx[ax]) * strides[ax]
                if flat_void[nb] and lab[nb] == 0:
                    lab[nb] = lc
                    heapq.heappush(heap, (-flat_d[nb], counter, int(nb)))
                    counter += 1
    return lab


def _touches_solid(cells, arr, amap, periodic):
    """True when one of the flat `cells` has a face-neighbour that is solid or a non-periodic box wall."""
    shape = arr.shape
    wraps = {ax_np: periodic[ax_s] for ax_s, ax_np in amap.items()}
    idx = np.array(np.unravel_index(cells, shape))
    flat_void = arr.ravel()
    strides = np.array([int(np.prod(shape[a + 1:])) for a in range(len(shape))])
    for ax in range(len(shape)):
        for sgn in (-1, 1):
            v = idx[ax] + sgn
            out = (v < 0) | (v >= shape[ax])
            if not wraps[ax] and np.any(out):
                return True
            v = v % shape[ax]
            nb = cells + (v - idx[ax]) * strides[ax]
            if np.any(~flat_void[nb]):
                return True
    return False


def _bisect(cells, arr, amap, periodic):
    """Two-way split of a region with a single distance basin: cut at the median of its longest extent
    (coordinates unwrapped around the region's first cell along periodic axes); each face-connected
    part becomes a piece.  Returns a flat piece-label array (0 outside the region)."""
    shape = arr.shape
    idx = np.array(np.unravel_index(cells, shape)).astype(np.int64)
    wraps = {ax_np: periodic[ax_s] for ax_s, ax_np in amap.items()}
    for ax in range(len(shape)):
        if wraps[ax]:
            ref = idx[ax, 0]
            d = (idx[ax] - ref + shape[ax] // 2) % shape[ax] - shape[ax] // 2
            idx[ax] = ref + d
    ext = idx.max(axis=1) - idx.min(axis=1)
    ax = int(np.argmax(ext))
    cut = np.median(idx[ax])
    side = (idx[ax] > cut).astype(np.int64) + 1
    if side.min() == side.max():
        side = (idx[ax] >= cut).astype(np.int64) + 1
    pieces = np.zeros(arr.size, np.int64)
    nxt = 1
    for sd in (1, 2):
        sel = np.zeros(arr.size, bool)
        sel[cells[side == sd]] = True
        comp, nc = ndimage.label(sel.reshape(shape), structure=_face_structure(len(shape)))
        comp = comp.ravel()
        for c in range(1, nc + 1):
            pieces[comp == c] = nxt
            nxt += 1
    return pieces


def _split_large(lab, arr, amap, periodic, dist, flat_d, w0, max_cells):
    """Split every region larger than `max_cells` by a watershed of the distance restricted to it, with
    marker windows w0 - 1, w0 - 2, ... 1 (the first that gives at least two markers), recursively.
    A piece that touches no solid joins the neighbouring piece it shares most faces with."""
    lab = lab.copy()
    nxt = int(lab.max()) + 1
    todo = [int(l) for l in np.unique(lab[lab > 0])]
    while todo:
        l = todo.pop()
        cells = np.flatnonzero(lab == l)
        if cells.size <= max_cells:
            continue
        inside = np.zeros(arr.size, bool)
        inside[cells] = True
        inside = inside.reshape(arr.shape)
        d_in = np.where(inside, dist, 0.0)
        pieces = None
        for w in range(max(w0 - 1, 1), 0, -1):
            peak = _markers(d_in, inside, amap, periodic, w)
            plab, npk = ndimage.label(peak, structure=np.ones((3,) * arr.ndim, bool))
            if npk >= 2:
                seeds = plab.ravel().astype(np.int64)
                pieces = _flood(inside, amap, periodic, flat_d, seeds)
                break
        if pieces is None:
            pieces = _bisect(cells, arr, amap, periodic)
        ids = [int(q) for q in np.unique(pieces[cells]) if q > 0]
        # pieces that touch no solid join their best-connected neighbouring piece
        good = {q for q in ids if _touches_solid(np.flatnonzero(pieces == q), arr, amap, periodic)}
        if not good:
            continue
        for q in ids:
            if q in good:
                continue
            sub = pieces.copy()
            sub[(sub > 0) & ~np.isin(sub, [q] + sorted(good))] = 0
            contacts = _region_contacts(sub.reshape(arr.shape), arr, amap, periodic)
            best, cnt = None, -1
            for (a, b), c in sorted(contacts.items()):
                other = b if a == q else (a if b == q else None)
                if other is not None and other in good and c > cnt:
                    best, cnt = other, c
            if best is not None:
                pieces[pieces == q] = best
        kept = sorted({int(q) for q in np.unique(pieces[cells]) if q > 0})
        if len(kept) < 2:
            continue
        for k, q in enumerate(kept):
            sel = cells[pieces[cells] == q]
            if k == 0:
                new = l
            else:
                new = nxt
                nxt += 1
            lab[sel] = new
            todo.append(new)
    return lab


def _region_contacts(lab, arr, amap, periodic):
    """Face contacts between distinct regions: dict (a, b) -> count with a < b."""
    L3 = lab.reshape(arr.shape)
    contacts = {}
    for ax_s, ax_np in amap.items():
        n = arr.shape[ax_np]
        a_ = np.take(L3, np.arange(n - 1), axis=ax_np)
        b_ = np.take(L3, np.arange(1, n), axis=ax_np)
        pairs = [(a_, b_)]
        if periodic[ax_s]:
            pairs.append((np.take(L3, [n - 1], axis=ax_np), np.take(L3, [0], axis=ax_np)))
        for x, y in pairs:
            sel = (x > 0) & (y > 0) & (x != y)
            lo = np.minimum(x[sel], y[sel])
            hi = np.maximum(x[sel], y[sel])
            key = lo.astype(np.int64) * (int(lab.max()) + 1) + hi
            uk, cnt = np.unique(key, return_counts=True)
            for k, c in zip(uk.tolist(), cnt.tolist()):
                pr = (k // (int(lab.max()) + 1), k % (int(lab.max()) + 1))
                contacts[pr] = contacts.get(pr, 0) + c
    return contacts


def _merge_regions(lab, arr, amap, periodic, min_cells, max_cells, target):
    """Greedy merging on the region adjacency graph.  Repeatedly take a region that touches no solid
    cell and no box wall (a pore is bounded by solid; such a region would make its closure block of
    Eqs. 6/9 singular: a constant velocity satisfies the closure on every side), else the smallest
    region below min_cells, or (while more than `target` regions remain) the smallest region, and
    merge it into the neighbour it shares the most faces with among those keeping the merged size
    <= max_cells (a region below min_cells may exceed max_cells if no neighbour fits).  Ties: lower
    label.  Regions are renumbered 1..K by their lowest linear index."""
    nl = int(lab.max())
    size = np.bincount(lab, minlength=nl + 1).astype(np.int64)
    size[0] = 0
    # regions touching a solid cell or a (non-periodic) box wall; the others are merged away
    wall = np.zeros(nl + 1, bool)
    L3 = lab.reshape(arr.shape)
    for ax_s, ax_np in amap.items():
        for sgn in (-1, 1):
            sh = np.roll(arr, sgn, axis=ax_np)
            solid_nb = ~sh
            if not periodic[ax_s]:
                edge = [slice(None)] * arr.ndim
                edge[ax_np] = 0 if sgn == 1 else arr.shape[ax_np] - 1
                solid_nb[tuple(edge)] = True
            wall[np.unique(L3[arr & solid_nb])] = True
    nbrs = {r: {} for r in range(1, nl + 1)}
    for (a_, b_), c in _region_contacts(lab, arr, amap, periodic).items():
        nbrs[a_][b_] = nbrs[a_].get(b_, 0) + c
        nbrs[b_][a_] = nbrs[b_].get(a_, 0) + c
    parent = np.arange(nl + 1)
    alive = set(r for r in range(1, nl + 1) if size[r] > 0)
    blocked = set()
    while True:
        cand = [r for r in alive if r not in blocked]
        if not cand:
            break
        inner = [q for q in cand if not wall[q]]
        r = min(inner, key=lambda q: (size[q], q)) if inner else min(cand, key=lambda q: (size[q], q))
        must = size[r] < min_cells or not wall[r]
        if not must and len(alive) <= target:
            break
        opts = [(c, q) for q, c in nbrs[r].items() if size[q] + size[r] <= max_cells]
        if not opts and must:
            opts = [(c, q) for q, c in nbrs[r].items()]
        if not opts:
            blocked.add(r)
            continue
        best = sorted(opts, key=lambda t: (-t[0], t[1]))[0][1]
        # merge r into best
        parent[r] = best
        wall[best] |= wall[r]
        size[best] += size[r]
        size[r] = 0
        alive.discard(r)
        for q, c in nbrs[r].items():
            if q == best:
                continue
            nbrs[best][q] = nbrs[best].get(q, 0) + c
            nbrs[q][best] = nbrs[q].get(best, 0) + c
            nbrs[q].pop(r, None)
        nbrs[best].pop(r, None)
        nbrs.pop(r)
        blocked.discard(best)
    # resolve parents
    root = np.arange(nl + 1)
    for r in range(1, nl + 1):
        q = r
        while parent[q] != q:
            q = parent[q]
        root[r] = q
    lab = root[lab]
    uniq = np.unique(lab[lab > 0])
    first = np.full(nl + 1, np.iinfo(np.int64).max)
    idx = np.flatnonzero(lab > 0)
    np.minimum.at(first, lab[idx], idx)
    order = sorted(uniq.tolist(), key=lambda v: first[v])
    remap = np.zeros(nl + 1, np.int64)
    remap[order] = np.arange(1, len(order) + 1)
    return remap[lab]


def label_pores(mask: np.ndarray, target: int, periodic=X_PERIODIC, windows=range(1, 25), method="window",
                min_cells: int = 0, max_cells: int = 0, oversegment: float = 4.0, split_cells: int = 0) -> Labelling:
    """Watershed decomposition of the void into about `target` pores (heights: the distance to the
    solid; priority flood, highest distance first, ties by insertion order, over the face-connected
    void wrapping along periodic axes).

    method="window" (default): markers are plateau components of cells that are maxima of the distance
    within a (2w+1)-wide window, w chosen from `windows` to bring the count closest to `target`; every
    region is a basin of the distance map, so it reaches the solid all around.
    method="nms" (alternative, not used by the workloads): markers are distance maxima accepted greedily in order of decreasing distance when
    farther than a spacing d from every accepted marker, d bisected to bring the count closest to
    `oversegment * target`; the flooded regions are then merged on their adjacency graph (smallest
    first, into the neighbour sharing most faces, keeping merged sizes <= max_cells) until about
    `target` remain and none is below min_cells (0 disables a bound).  Merged regions can carry
    appendages that touch no solid; under the closure of Eqs. 6/9 a constant velocity there is a null
    vector of the closure block (seen on a 96^3 sphere pack), so the workloads use "window".
    Void components without a marker get one at their deepest cell (lowest linear index among ties).

    split_cells > 0 (window method only): every region larger than split_cells is re-segmented, by a
    watershed of the distance restricted to it with smaller marker windows, or, when it has a single
    distance maximum, by a median bisection along its longest extent; a piece that touches no solid
    joins the neighbouring piece it shares most faces with."""
    m = np.asarray(mask).astype(bool)
    arr, amap = _squeeze2d(m)
    dist2 = _squeeze2d(distance_to_solid(m, periodic))[0]
    flat_d = dist2.ravel()
    lab = np.zeros(arr.size, np.int64)
    chosen = 0
    if method == "nms":
        lo, hi = 1.0, float(max(arr.shape))
        best = None
        for _ in range(18):
            mid = 0.5 * (lo + hi)
            mk = _nms_markers(dist2, arr, amap, periodic, mid)
            want = int(round(oversegment * target)) if (min_cells or max_cells) else target
            score = abs(len(mk) - want)
            if best is None or score < best[0]:
                best = (score, mid, mk)
            if len(mk) > want:
                lo = mid
            else:
                hi = mid
        _, chosen, mk = best
        lab[np.sort(mk)] = np.arange(1, len(mk) + 1)
        npk = len(mk)
    else:
        best = None
        for w in windows:
            peak = _markers(dist2, arr, amap, periodic, w)
            plab, npk = ndimage.label(peak, structure=np.ones((3,) * arr.ndim, bool))
            score = abs(npk - target)
            if best is None or score < best[0]:
                best = (score, w, plab, npk)
            if npk < target:
                break
        _, chosen, plab, npk = best
        lab = plab.ravel().astype(np.int64).copy()
        if npk > 0:
            first = ndimage.minimum(np.arange(lab.size), labels=plab.ravel(), index=np.arange(1, npk + 1))
            order = np.argsort(first, kind="stable")
            remap = np.zeros(npk + 1, np.int64)
            remap[order + 1] = np.arange(1, npk + 1)
            lab = remap[lab]
    comp, ncomp = void_components(m, periodic)
    comp = _squeeze2d(comp)[0].ravel()
    has = np.zeros(ncomp + 1, bool)
    has[comp[lab > 0]] = True
    nl = int(lab.max()) if lab.size else 0
    for cidx in range(1, ncomp + 1):
        if not has[cidx]:
            cells = np.flatnonzero(comp == cidx)
            c = cells[np.argmax(flat_d[cells])]
            nl += 1
            lab[c] = nl
    lab = _flood(arr, amap, periodic, flat_d, lab)
    if method == "window" and split_cells > 0:
        lab = _split_large(lab, arr, amap, periodic, dist2, flat_d, int(chosen), split_cells)
    if method == "nms":
        lab = _merge_regions(lab, arr, amap, periodic, min_cells, max_cells or arr.size,
                             target if (min_cells or max_cells) else arr.size)
    labels = lab.reshape(arr.shape).astype(np.int32).reshape(mask.shape)
    return Labelling(labels=labels, n_labels=int(lab.max()), window=chosen, dist=dist2.reshape(mask.shape))


# ----------------------------------------------------------------------------------------------
# Reynolds number (Sec. 6)
# ----------------------------------------------------------------------------------------------
def characteristic_length(mask: np.ndarray, periodic=X_PERIODIC) -> float:
    """l = V_s / A_w: solid voxel count over the count of void-solid voxel faces inside the image
    (wrapping along periodic axes; the box walls are not counted)."""
    m = np.asarray(mask).astype(bool)
    arr, amap = _squeeze2d(m)
    vs = float((~arr).sum())
    aw = 0
    for ax_solver, ax_np in amap.items():
        a = arr
        b = np.roll(arr, -1, axis=ax_np)
        diff = a != b
        if not periodic[ax_solver]:
            diff = np.take(diff, np.arange(arr.shape[ax_np] - 1), axis=ax_np)
        aw += int(diff.sum())
    return vs / max(1, aw)


def darcy_velocity(ux_faces: np.ndarray) -> float:
    """U_D: mean of the x-face velocity array over the whole box (solid faces count zero)."""
    return float(np.mean(ux_faces))


def reynolds(mask, ux_faces, rho, mu, periodic=X_PERIODIC) -> float:
    phi = float(np.mean(mask))
    return rho * (darcy_velocity(ux_faces) / phi) * characteristic_length(mask, periodic) / mu


def mu_for_reynolds(mask, ux_faces_at_mu1, re_target, rho=1.0, periodic=X_PERIODIC) -> float:
    """Viscosity that gives `re_target` given the Stokes x-velocity computed at mu = 1 (the Stokes
    velocity scales as 1/mu, so Re(mu) = Re(1)/mu^2)."""
    re1 = reynolds(mask, ux_faces_at_mu1, rho, 1.0, periodic)
    return float(np.sqrt(re1 / re_target))


def mu_kozeny_carman(mask, re_target, rho=1.0, b=1.0, periodic=X_PERIODIC) -> float:
    """Viscosity for a target Re from geometry alone: Kozeny-Carman permeability for a bed of grains
    of diameter 6 l (l = V_s / A_w), k = phi^3 l^2 / (5 (1 - phi)^2); Darcy U_D = k rho b / mu,
    U = U_D / phi, Re = rho U l / mu  =>  mu = sqrt(rho^2 b k l / (phi Re)).  The Re actually reached
    is measured from the solution (`reynolds`)."""
    phi = float(np.mean(mask))
    l = characteristic_length(mask, periodic)
    k = phi ** 3 * l * l / (5.0 * (1.0 - phi) ** 2)
    return float(np.sqrt(rho * rho * b * k * l / (phi * re_target)))


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mask: np.ndarray
    labels: np.ndarray
    periodic: tuple
    dropped: float
    n_labels: int


def make_workload(kind: str, seed: int = 0, **kw) -> Workload:
    """Seeded image + percolation filter + labels.

    kind: 'disks64'  2D 64x64, 12 non-overlapping disks r~U[4,8], ~15 pores
          'spheres'  3D n^3 (n=96 default) sphere pack r~U[6,10] to porosity 0.35, ~200 pores
          'grf'      3D n^3 (n=256 default) Gaussian field l=8 at porosity 0.20, ~3000 pores
          'tiny2d' / 'tiny3d'  small disk/sphere packs for brute-force checks (n given by kw)"""
    per = X_PERIODIC
    min_cells = max_cells = 0
    split = 0
    if kind == "disks64":
        n = kw.get("n", 64)
        mask = disk_pack_2d(n, kw.get("n_disks", 12), 4.0, 8.0, seed)
        target = kw.get("target", 15)
    elif kind == "spheres":
        n = kw.get("n", 96)
        mask = sphere_pack_3d(n, kw.get("rmin", 6.0), kw.get("rmax", 10.0), kw.get("porosity", 0.35), seed)
        target = kw.get("target", 200)
        min_cells, max_cells = 135, 5400   # ~500 and ~20k unknowns (3.7 unknowns per void cell)
        split = kw.get("split_cells", 0)
    elif kind == "grf":
        n = kw.get("n", 256)
        mask = gaussian_field_3d(n, kw.get("corr_len", 8.0), kw.get("porosity", 0.20), seed)
        target = kw.get("target", 3000)
        min_cells, max_cells = 135, 5400
        # split_cells > 0 re-segments regions above that many cells (watershed inside the region, else a
        # median bisection) so that dense local inverses of the largest pores (up to ~27,000 cells at
        # 256^3) fit the device; off by default (see the labeller's split_cells)
        split = kw.get("split_cells", 0)
    elif kind == "tiny2d":
        n = kw.get("n", 16)
        mask = disk_pack_2d(n, kw.get("n_disks", 2), kw.get("rmin", 1.5), kw.get("rmax", 3.0), seed)
        target = kw.get("target", 3)
    elif kind == "tiny3d":
        n = kw.get("n", 8)
        mask = sphere_pack_3d(n, kw.get("rmin", 1.5), kw.get("rmax", 2.5), kw.get("porosity", 0.6), seed)
        target = kw.get("target", 3)
    else:
        raise ValueError(kind)
    mask, dropped = percolating_void(mask, per)
    lab = label_pores(mask, target, per, method=kw.get("method", "window"), min_cells=kw.get("min_cells", min_cells),
                      max_cells=kw.get("max_cells", max_cells), split_cells=split)
    return Workload(kind, mask, lab.labels, per, dropped, lab.n_labels)


# ----------------------------------------------------------------------------------------------
# seeded synthetic velocity fields
# ----------------------------------------------------------------------------------------------
def synthetic_wind(shape, seed: int = 0, mean_x: float = 0.3, amplitude: float = 0.3,
                   smooth: float = 2.0) -> np.ndarray:
    """A seeded smooth random velocity in the full layout [u_x | u_y | (u_z) | p] of an image of
    `shape` (nz, ny, nx): each velocity component is white noise smoothed by a Gaussian of width
    `smooth` voxels (wrapping), scaled to unit standard deviation, times `amplitude`, plus `mean_x` on
    u_x; the pressure block is zero.  It is a stand-in linearisation state ("wind") for tests of the
    preconditioner builds; it holds no solver arithmetic, and entries that are not unknowns are left
    to the caller to ignore or zero."""
    nz, ny, nx = shape
    dim = 2 if nz == 1 else 3
    rng = np.random.default_rng(seed)
    nc = nx * ny * nz
    out = np.zeros((dim + 1) * nc)
    for d in range(dim):
        f = rng.standard_normal(shape)
        f = ndimage.gaussian_filter(f, smooth, mode="wrap")
        f = f / max(float(f.std()), 1e-300)
        out[d * nc:(d + 1) * nc] = amplitude * f.ravel() + (mean_x if d == 0 else 0.0)
    return out
