// MAC stencil of the steady / backward-Euler Navier-Stokes residual and of its linearisations
// (Eq. 1, Eq. 3, Sec. 2; modified residual of Eq. 27 for gPLMM).  Device code shared by the
// residual, matrix-free operator and dense block-assembly kernels.
//
// Index space ("full layout"): face unknown (d, c) -> d * ncell + c; cell c -> dim * ncell + c.
// Cell flags (one byte per cell):
//   bit 0        void
//   bit 1 + d    the low face of the cell along axis d is an unknown
//   bit 4        the cell is a pressure pin (continuity row replaced by r = p)
//   bit 5 + d    gPLMM tag of the low face along d (inertia dropped in the modified residual)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pns {

enum : uint8_t { FL_VOID = 1, FL_PIN = 16 };
__host__ __device__ inline uint8_t fl_face(int d) { return (uint8_t)(2u << d); }
__host__ __device__ inline uint8_t fl_tag(int d) { return (uint8_t)(32u << d); }

// Operators whose rows the stencil enumerates.
enum Op : int {
  OP_NEWTON = 0,   // Newton Jacobian at a state x (upwind branches frozen at x)
  OP_OSEEN = 1,    // Jacobian of the modified residual (Eq. 27): wind w, no inertia on tagged faces
  OP_STOKES = 2,   // no inertia (rho/dt kept)
};

struct Geo {
  int nx, ny, nz, dim;
  int ncell;
  int per[3];
};

struct Phy {
  double rho, mu, inv_dt;   // inv_dt = 0 for the steady equations
  double b[3];
};

struct CellPos {
  int c;
  int x[3];
};

__host__ __device__ inline CellPos cell_pos(const Geo& G, int c) {
  CellPos p;
  p.c = c;
  p.x[0] = c % G.nx;
  int t = c / G.nx;
  p.x[1] = t % G.ny;
  p.x[2] = t / G.ny;
  return p;
}

__host__ __device__ inline int extent(const Geo& G, int a) { return a == 0 ? G.nx : (a == 1 ? G.ny : G.nz); }
__host__ __device__ inline int stride(const Geo& G, int a) { return a == 0 ? 1 : (a == 1 ? G.nx : G.nx * G.ny); }

// Neighbour of cell p along axis a, direction s (+1 / -1); -1 when off the grid (non-periodic).
__host__ __device__ inline int nbr(const Geo& G, const CellPos& p, int a, int s) {
  int n = extent(G, a);
  int v = p.x[a] + s;
  if (v < 0 || v >= n) {
    if (!G.per[a]) return -1;
    v = (v + n) % n;
  }
  return p.c + (v - p.x[a]) * stride(G, a);
}

__host__ __device__ inline int nbr_c(const Geo& G, int c, int a, int s) { return nbr(G, cell_pos(G, c), a, s); }

__host__ __device__ inline bool face_unknown(const uint8_t* fl, int d, int c) { return c >= 0 && (fl[c] & fl_face(d)); }

// ----------------------------------------------------------------------------------------------
// Row enumeration.  emit(col, val) is called once per (column, coefficient) contribution; the same
// column may appear several times (the caller sums).  T is the arithmetic type of the coefficients.
// `st` is the state of the linearisation (Newton: x; Oseen: the wind w), full layout, FP64.
// ----------------------------------------------------------------------------------------------
template <typename T, typename Emit>
__device__ __forceinline__ void face_row(const Geo& G, const Phy& P, const uint8_t* __restrict__ fl, int op,
                                         const double* __restrict__ st, int d, const CellPos& p, Emit& emit) {
  const int nc = G.ncell;
  const int c = p.c;
  const int R = d * nc + c;
  const T rho = (T)P.rho, mu = (T)P.mu;
  if (P.inv_dt > 0) emit(R, (T)(P.rho * P.inv_dt));
  int nm[3], np[3];
  bool um[3], up[3];
  for (int a = 0; a < G.dim; ++a) {
    np[a] = nbr(G, p, a, +1);
    nm[a] = nbr(G, p, a, -1);
    up[a] = face_unknown(fl, d, np[a]);
    um[a] = face_unknown(fl, d, nm[a]);
    // viscous: mu (2q - q+ - q-); a missing neighbour is 0 along d, ghost -q across d
    emit(R, (T)2 * mu);
    if (up[a]) emit(d * nc + np[a], -mu);
    else if (a != d) emit(R, mu);
    if (um[a]) emit(d * nc + nm[a], -mu);
    else if (a != d) emit(R, mu);
  }
  // pressure gradient p_c - p_{c - e_d}
  const int lo = nm[d];
  emit(G.dim * nc + c, (T)1);
  emit(G.dim * nc + lo, (T)-1);
  if (op == OP_STOKES) return;
  if (op == OP_OSEEN && (fl[c] & fl_tag(d))) return;
  const T q = (T)st[R];
  CellPos plo = cell_pos(G, lo);
  for (int a = 0; a < G.dim; ++a) {
    T U;
    int fa[4] = {-1, -1, -1, -1};
    if (a == d) {
      U = q;
    } else {
      // four axis-a faces of the flanking cells lo and c: low/high face of each
      fa[0] = lo;
      fa[1] = nbr(G, plo, a, +1);
      fa[2] = c;
      fa[3] = np[a];
      U = (T)0;
      for (int k = 0; k < 4; ++k) {
        if (face_unknown(fl, a, fa[k])) U += (T)st[a * nc + fa[k]];
        else fa[k] = -1;
      }
      U *= (T)0.25;
    }
    const bool back = U >= (T)0;
    if (a == d) {
      if (back) {
        emit(R, rho * U);
        if (um[a]) emit(d * nc + nm[a], -rho * U);
      } else {
        emit(R, -rho * U);
        if (up[a]) emit(d * nc + np[a], rho * U);
      }
    } else {
      if (back) {
        emit(R, rho * U * (um[a] ? (T)1 : (T)2));
        if (um[a]) emit(d * nc + nm[a], -rho * U);
      } else {
        emit(R, -rho * U * (up[a] ? (T)1 : (T)2));
        if (up[a]) emit(d * nc + np[a], rho * U);
      }
    }
    if (op != OP_NEWTON) continue;
    // reaction term dU * D (Newton only)
    T qm = um[a] ? (T)st[d * nc + nm[a]] : (a == d ? (T)0 : -q);
    T qp = up[a] ? (T)st[d * nc + np[a]] : (a == d ? (T)0 : -q);
    T D = back ? (q - qm) : (qp - q);
    if (a == d) {
      emit(R, rho * D);
    } else {
      for (int k = 0; k < 4; ++k)
        if (fa[k] >= 0) emit(a * nc + fa[k], (T)0.25 * rho * D);
    }
  }
}

template <typename T, typename Emit>
__device__ __forceinline__ void cell_row(const Geo& G, const uint8_t* __restrict__ fl, const CellPos& p, Emit& emit) {
  const int nc = G.ncell;
  const int c = p.c;
  if (fl[c] & FL_PIN) {
    emit(G.dim * nc + c, (T)1);
    return;
  }
  for (int a = 0; a < G.dim; ++a) {
    int hi = nbr(G, p, a, +1);
    if (face_unknown(fl, a, hi)) emit(a * nc + hi, (T)1);
    if (fl[c] & fl_face(a)) emit(a * nc + c, (T)-1);
  }
}

// Decode a full-layout index into (kind, axis, cell): kind 0 = face, 1 = cell.
__host__ __device__ inline void decode(const Geo& G, int g, int& is_cell, int& d, int& c) {
  int comp = g / G.ncell;
  c = g - comp * G.ncell;
  is_cell = comp == G.dim;
  d = comp;
}

template <typename T, typename Emit>
__device__ __forceinline__ void any_row(const Geo& G, const Phy& P, const uint8_t* __restrict__ fl, int op,
                                        const double* __restrict__ st, int g, Emit& emit) {
  int is_cell, d, c;
  decode(G, g, is_cell, d, c);
  CellPos p = cell_pos(G, c);
  if (is_cell) cell_row<T>(G, fl, p, emit);
  else face_row<T>(G, P, fl, op, st, d, p, emit);
}

}  // namespace pns
