"""MAC discretisation of steady / backward-Euler incompressible Navier-Stokes on a voxel image.

Follows Eq. 1 (governing equations), Eq. 3 (Newton system J dx = -r with J = [[F, G^T], [G, O]])
and Sec. 2 (MAC: velocity on cell faces, pressure at cell centres, grid = image voxels).
The details the paper leaves open are fixed as follows:

* h = 1.  Periodic along axes flagged in `periodic` (default x only); other box faces are no-slip
  walls; void-solid faces are no-slip.
* Face array of axis d at cell c holds the face on the LOW side of c along d.  It is an unknown iff
  both flanking cells (c - e_d, c) exist and are void.
* Neighbour of a face q along axis a that is not an unknown: value 0 when a == d (the face sits on a
  wall), ghost value -q when a != d (no-slip wall half a cell away).
* Viscous term: mu * sum_a (2q - q_{+a} - q_{-a}).  Pressure gradient at face: p_c - p_{c-e_d}.
  Divergence at cell: sum_a (u_a(high face) - u_a(low face)).
* Inertia (u . grad) u in advective form, first-order upwind with a 3-point stencil per axis
  (the "three-point upwind" of Sec. 4):  sum_a [max(U_a,0)(q - q_{-a}) + min(U_a,0)(q_{+a} - q)],
  U_d = q on the face's own axis, U_a (a != d) = mean of the four axis-a faces of the two flanking
  cells (non-unknowns count 0).  U_a >= 0 takes the backward branch.
* Backward Euler adds rho (q - q_prev) / dt.  Body force rho b enters as -rho b_d.
* Pressure gauge: in each face-connected void component (wrapping along periodic axes) the void
  cell with the lowest linear index is pinned: its continuity row is replaced by r = p.

Vectors are "full": length (dim + 1) * ncell, blocks [u_x, u_y, (u_z), p], each image-shaped; entries
that are not unknowns are zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Grid:
    """Image geometry: sizes, neighbour tables and the unknown masks."""

    def __init__(self, mask, periodic=(True, False, False)):
        mask = np.asarray(mask)
        assert mask.ndim == 3
        self.shape = mask.shape                      # (nz, ny, nx)
        nz, ny, nx = self.shape
        self.dim = 2 if nz == 1 else 3
        self.size = (nx, ny, nz)                     # extent along solver axis a
        self.periodic = tuple(bool(p) for p in periodic)
        self.ncell = nx * ny * nz
        self.void = mask.ravel().astype(bool)
        c = np.arange(self.ncell)
        self.coord = (c % nx, (c // nx) % ny, c // (nx * ny))
        self.stride = (1, nx, nx * ny)
        # nb[a][0] = neighbour at -1 along a, nb[a][1] = at +1 (-1 marks off-grid)
        self.nb = []
        for a in range(self.dim):
            pair = []
            for s in (-1, 1):
                v = self.coord[a] + s
                n = self.size[a]
                off = (v < 0) | (v >= n)
                if self.periodic[a]:
                    v = v % n
                    off = np.zeros_like(off)
                idx = c + (np.where(off, self.coord[a], v) - self.coord[a]) * self.stride[a]
                pair.append(np.where(off, -1, idx))
            self.nb.append(pair)
        self.face_unknown = []
        for d in range(self.dim):
            lo = self.nb[d][0]
            ok = self.void & (lo >= 0)
            ok &= self.void[np.where(lo >= 0, lo, 0)]
            self.face_unknown.append(ok)
        self.nfull = (self.dim + 1) * self.ncell
        mask_full = np.concatenate(self.face_unknown + [self.void])
        self.unknown = np.flatnonzero(mask_full)     # global indices of all unknowns
        self.unknown_mask = mask_full
        self.n_faces = int(sum(f.sum() for f in self.face_unknown))
        self.n_cells = int(self.void.sum())

    # global indices
    def fidx(self, d, c):
        return d * self.ncell + c

    def pidx(self, c):
        return self.dim * self.ncell + c

    def split(self, x):
        n = self.ncell
        return [x[d * n:(d + 1) * n] for d in range(self.dim)], x[self.dim * n:(self.dim + 1) * n]

    def face_at(self, d, cells):
        """For an array of cell indices (-1 = off grid): (safe index, is-unknown) of the axis-d face
        stored at that cell."""
        valid = cells >= 0
        safe = np.where(valid, cells, 0)
        return safe, valid & self.face_unknown[d][safe]


def void_adjacency(g: Grid):
    """Symmetric 0/1 matrix (ncell x ncell, CSR) linking face-neighbouring void cells (wrapping along
    periodic axes)."""
    rows, cols = [], []
    c = np.arange(g.ncell)
    for a in range(g.dim):
        n = g.nb[a][1]
        ok = g.void & (n >= 0)
        ok &= g.void[np.where(n >= 0, n, 0)]
        rows.append(c[ok])
        cols.append(n[ok])
    r = np.concatenate(rows)
    k = np.concatenate(cols)
    A = sp.coo_matrix((np.ones(2 * len(r)), (np.concatenate([r, k]), np.concatenate([k, r]))),
                      shape=(g.ncell, g.ncell)).tocsr()
    A.data[:] = 1.0
    return A


def pressure_pins(g: Grid):
    """Lowest-linear-index cell of every face-connected void component (periodic wrap)."""
    from scipy.sparse.csgraph import connected_components
    n, lab = connected_components(void_adjacency(g), directed=False)
    lab = np.where(g.void, lab, -1)
    pins = []
    for comp in np.unique(lab[g.void]):
        pins.append(int(np.flatnonzero(lab == comp)[0]))
    return np.array(sorted(pins), dtype=np.int64)


class Params:
    """Physical parameters: density, viscosity, body force per unit mass, time step (<= 0: steady)."""

    def __init__(self, rho, mu, b, dt=0.0):
        self.rho = float(rho)
        self.mu = float(mu)
        self.b = tuple(float(v) for v in b) + (0.0,) * (3 - len(b))
        self.dt = float(dt)

    @property
    def transient(self):
        return self.dt > 0


def _neighbour_values(g, q, d, a):
    """Values of face array q (axis d) at the +a and -a neighbours with the wall conventions."""
    ip, up = g.face_at(d, g.nb[a][1])
    im, um = g.face_at(d, g.nb[a][0])
    if a == d:
        qp = np.where(up, q[ip], 0.0)
        qm = np.where(um, q[im], 0.0)
    else:
        qp = np.where(up, q[ip], -q)
        qm = np.where(um, q[im], -q)
    return qp, qm, (ip, up), (im, um)


def _advecting(g, u, d, a):
    """Advecting velocity along axis a at the axis-d faces: U_d = u_d, else the mean of the four
    axis-a faces of the two flanking cells.  Also returns the four (index, valid) pairs."""
    if a == d:
        return u[d].copy(), []
    lo = g.nb[d][0]
    lo_safe = np.where(lo >= 0, lo, 0)
    lo_hi = np.where(lo >= 0, g.nb[a][1][lo_safe], -1)
    cells = [lo, lo_hi, np.arange(g.ncell), g.nb[a][1]]
    parts = [g.face_at(a, cc) for cc in cells]
    U = np.zeros(g.ncell)
    for (ix, ok) in parts:
        U += np.where(ok, u[a][ix], 0.0)
    return 0.25 * U, parts


def residual(g: Grid, prm: Params, x, pins, x_prev=None):
    """Full residual r(x) (Eq. 3 left side; steady or backward Euler)."""
    u, p = g.split(np.asarray(x, dtype=np.float64))
    u = [np.where(g.face_unknown[d], u[d], 0.0) for d in range(g.dim)]
    r = np.zeros(g.nfull)
    ru, rp = g.split(r)
    if x_prev is not None:
        up_, _ = g.split(np.asarray(x_prev, dtype=np.float64))
    for d in range(g.dim):
        q = u[d]
        acc = np.zeros(g.ncell)
        for a in range(g.dim):
            qp, qm, _, _ = _neighbour_values(g, q, d, a)
            acc += prm.mu * (2 * q - qp - qm)
            U, _ = _advecting(g, u, d, a)
            acc += prm.rho * np.where(U >= 0, U * (q - qm), U * (qp - q))
        lo = g.nb[d][0]
        acc += p - p[np.where(lo >= 0, lo, 0)]
        acc -= prm.rho * prm.b[d]
        if prm.transient:
            qn = np.where(g.face_unknown[d], up_[d], 0.0) if x_prev is not None else 0.0
            acc += prm.rho * (q - qn) / prm.dt
        ru[d][:] = np.where(g.face_unknown[d], acc, 0.0)
    div = np.zeros(g.ncell)
    for a in range(g.dim):
        ih, uh = g.face_at(a, g.nb[a][1])
        div += np.where(uh, u[a][ih], 0.0) - u[a]
    rp[:] = np.where(g.void, div, 0.0)
    rp[pins] = p[pins]
    return r


def reference_norm(g: Grid, prm: Params, pins):
    """||r(u=0, p=0)|| with the previous time level set to zero (Sec. 8 normalisation)."""
    return float(np.linalg.norm(residual(g, prm, np.zeros(g.nfull), pins, None)))


def assemble(g: Grid, prm: Params, pins, kind="newton", state=None, wind=None, tags=None):
    """Sparse matrix (CSR, nfull x nfull, empty rows/cols at non-unknowns) of:

    kind == 'newton': the Newton Jacobian J(x) at x = `state`, upwind branches frozen at x (Eq. 3);
    kind == 'oseen' : Jacobian of the modified residual of Eq. 27, inertia w . grad u with the wind
                      `wind` (a full vector; only its velocity is used), no inertia on `tags` rows;
    kind == 'stokes': rho = 0 in the inertia (the rho/dt term is kept).
    """
    rows, cols, vals = [], [], []

    def emit(r, c, v, sel=None):
        if sel is not None:
            r, c, v = r[sel], c[sel], (v[sel] if np.ndim(v) else np.full(int(sel.sum()), v))
        else:
            v = v if np.ndim(v) else np.full(len(r), v)
        rows.append(np.asarray(r))
        cols.append(np.asarray(c))
        vals.append(np.asarray(v, dtype=np.float64))

    cells = np.arange(g.ncell)
    if kind == "newton":
        u, _ = g.split(np.asarray(state, dtype=np.float64))
        u = [np.where(g.face_unknown[d], u[d], 0.0) for d in range(g.dim)]
    elif kind == "oseen":
        w, _ = g.split(np.asarray(wind, dtype=np.float64))
        w = [np.where(g.face_unknown[d], w[d], 0.0) for d in range(g.dim)]
    rho, mu = prm.rho, prm.mu
    for d in range(g.dim):
        F = g.face_unknown[d]
        R = g.fidx(d, cells)
        # transient
        if prm.transient:
            emit(R, R, rho / prm.dt, F)
        # viscous
        for a in range(g.dim):
            emit(R, R, 2 * mu, F)
            for t in (0, 1):
                ix, ok = g.face_at(d, g.nb[a][t])
                emit(R, g.fidx(d, ix), -mu, F & ok)
                if a != d:
                    emit(R, R, mu, F & ~ok)     # ghost -q
        # pressure gradient
        lo = g.nb[d][0]
        emit(R, g.pidx(cells), 1.0, F)
        emit(R, g.pidx(np.where(lo >= 0, lo, 0)), -1.0, F)
        # inertia
        if kind == "stokes":
            continue
        rowsel = F.copy()
        if kind == "oseen" and tags is not None:
            rowsel &= ~tags[d]
        for a in range(g.dim):
            ip, up = g.face_at(d, g.nb[a][1])
            im, um = g.face_at(d, g.nb[a][0])
            if kind == "newton":
                q = u[d]
                qp, qm, _, _ = _neighbour_values(g, q, d, a)
                U, parts = _advecting(g, u, d, a)
            else:
                U, _ = _advecting(g, w, d, a)
                parts = []
            back = U >= 0
            fwd = ~back
            # U * dD terms (both kinds)
            if a == d:
                emit(R, R, rho * U, rowsel & back)
                emit(R, g.fidx(d, im), -rho * U, rowsel & back & um)
                emit(R, R, -rho * U, rowsel & fwd)
                emit(R, g.fidx(d, ip), rho * U, rowsel & fwd & up)
            else:
                emit(R, R, rho * U * np.where(um, 1.0, 2.0), rowsel & back)
                emit(R, g.fidx(d, im), -rho * U, rowsel & back & um)
                emit(R, R, -rho * U * np.where(up, 1.0, 2.0), rowsel & fwd)
                emit(R, g.fidx(d, ip), rho * U, rowsel & fwd & up)
            if kind != "newton":
                continue
            # dU * D terms (Newton only)
            D = np.where(back, q - qm, qp - q)
            if a == d:
                emit(R, R, rho * D, rowsel)
            else:
                for (ix, ok) in parts:
                    emit(R, g.fidx(a, ix), 0.25 * rho * D, rowsel & ok)
    # continuity rows
    P = g.pidx(cells)
    pin_mask = np.zeros(g.ncell, bool)
    pin_mask[pins] = True
    cont = g.void & ~pin_mask
    for a in range(g.dim):
        ih, uh = g.face_at(a, g.nb[a][1])
        emit(P, g.fidx(a, ih), 1.0, cont & uh)
        emit(P, g.fidx(a, cells), -1.0, cont & g.face_unknown[a])
    emit(P, P, 1.0, pin_mask)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(g.nfull, g.nfull)).tocsr()
    A.sum_duplicates()
    return A


def restrict(g: Grid, A):
    """Square sub-matrix on the unknowns only (for direct solves)."""
    return A[g.unknown][:, g.unknown]


def modified_residual(g: Grid, prm: Params, x, pins, wind, tags=None, x_prev=None):
    """Modified residual of Eq. 27: inertia linearised about the wind w (w . grad u, upwind branch from
    w) and removed on tagged faces; everything else as in `residual`.  Linear in x."""
    u, p = g.split(np.asarray(x, dtype=np.float64))
    u = [np.where(g.face_unknown[d], u[d], 0.0) for d in range(g.dim)]
    w, _ = g.split(np.asarray(wind, dtype=np.float64))
    w = [np.where(g.face_unknown[d], w[d], 0.0) for d in range(g.dim)]
    r = residual(g, Params(0.0, prm.mu, (0.0, 0.0, 0.0), 0.0), x, pins)   # viscous, gradient, continuity
    ru, _ = g.split(r)
    if x_prev is not None:
        up_, _ = g.split(np.asarray(x_prev, dtype=np.float64))
    for d in range(g.dim):
        q = u[d]
        acc = np.zeros(g.ncell)
        for a in range(g.dim):
            qp, qm, _, _ = _neighbour_values(g, q, d, a)
            U, _ = _advecting(g, w, d, a)
            acc += prm.rho * np.where(U >= 0, U * (q - qm), U * (qp - q))
        if tags is not None:
            acc = np.where(tags[d], 0.0, acc)
        acc -= prm.rho * prm.b[d]
        if prm.transient:
            qn = np.where(g.face_unknown[d], up_[d], 0.0) if x_prev is not None else 0.0
            acc += prm.rho * (q - qn) / prm.dt
        ru[d][:] += np.where(g.face_unknown[d], acc, 0.0)
    return r
