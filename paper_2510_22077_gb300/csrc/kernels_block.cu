// Kernels of the block-triangular Schur-complement preconditioner (the comparator of Sec. 1: the block
// form M_B with the scaled BFBt approximation of Eq. 4).  Over [faces | cells] the Jacobian is
// J = [[F, B1], [B2, C]]: B1 is the pressure gradient (face (d, c): p_c - p_{c - e_d}), B2 the
// divergence (cell c: sum_a u_a(high face) - u_a(low face)), pinned cells read r = p.
//  * D = diag(F) on the face unknowns,
//  * gradients and divergences with the 1/D scaling of Eq. 4,
//  * dense pore blocks of L = B2 D^{-1} B1 on the cells that are not pinned (block Jacobi).
// All vectors are FP64 in the full layout; entries outside the space a kernel writes are zeroed.
#include "internal.h"

namespace pns {

namespace {

struct DiagEmit {
  int row;
  double v;
  __device__ __forceinline__ void operator()(int col, double val) {
    if (col == row) v += val;
  }
};

__global__ void k_diag_F(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                         double* __restrict__ D) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  CellPos p = cell_pos(G, c);
  const uint8_t f = fl[c];
  for (int d = 0; d < G.dim; ++d) {
    const int R = d * G.ncell + c;
    double v = 0.0;
    if (f & fl_face(d)) {
      DiagEmit e{R, 0.0};
      face_row<double>(G, P, fl, op, st, d, p, e);
      v = e.v;
    }
    D[R] = v;
  }
  D[G.dim * G.ncell + c] = 0.0;
}

__device__ __forceinline__ double cell_val(const Geo& G, const uint8_t* __restrict__ fl, const double* __restrict__ y,
                                           int c, int skip_pins) {
  if (skip_pins && (fl[c] & FL_PIN)) return 0.0;
  return y[G.dim * G.ncell + c];
}

// mode 0: t_f = (y_c - y_lo) / D_f with pinned cells read as 0       (D^{-1} B1 y on the unpinned cells)
// mode 1: t_f = v_f - (y_c - y_lo)                                     (v_u - B1 y, pins included)
// the cell block of t is zeroed
__global__ void k_grad(Geo G, const uint8_t* __restrict__ fl, const double* __restrict__ y,
                       const double* __restrict__ D, const double* __restrict__ v, int mode, double* __restrict__ t) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  const int nc = G.ncell;
  CellPos p = cell_pos(G, c);
  const uint8_t f = fl[c];
  for (int d = 0; d < G.dim; ++d) {
    const int R = d * nc + c;
    double out = 0.0;
    if (f & fl_face(d)) {
      const int lo = nbr(G, p, d, -1);
      if (mode == 0) out = (cell_val(G, fl, y, c, 1) - cell_val(G, fl, y, lo, 1)) / D[R];
      else out = v[R] - (cell_val(G, fl, y, c, 0) - cell_val(G, fl, y, lo, 0));
    }
    t[R] = out;
  }
  t[G.dim * nc + c] = 0.0;
}

// y_c = sum_a t[a, high face] - t[a, low face] on void cells that are not pinned, times `sign`;
// with `scale`, t_f is divided by D_f first.  The face block of y is zeroed.
__global__ void k_div(Geo G, const uint8_t* __restrict__ fl, const double* __restrict__ t,
                      const double* __restrict__ D, double sign, double* __restrict__ y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  const int nc = G.ncell;
  CellPos p = cell_pos(G, c);
  const uint8_t f = fl[c];
  double out = 0.0;
  if ((f & FL_VOID) && !(f & FL_PIN)) {
    for (int a = 0; a < G.dim; ++a) {
      int hi = nbr(G, p, a, +1);
      if (face_unknown(fl, a, hi)) out += D ? t[a * nc + hi] / D[a * nc + hi] : t[a * nc + hi];
      if (f & fl_face(a)) out -= D ? t[a * nc + c] / D[a * nc + c] : t[a * nc + c];
    }
  }
  for (int d = 0; d < G.dim; ++d) y[d * nc + c] = 0.0;
  y[G.dim * nc + c] = sign * out;
}

// pressure assembly: mode 0: out = v on unpinned void cells (faces and pins 0);
// mode 1: out cells = pinned ? v : -w, faces 0;  mode 2: out faces = u, cells = y (the final z)
__global__ void k_compose(Geo G, const uint8_t* __restrict__ fl, const double* __restrict__ a,
                          const double* __restrict__ b, int mode, double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  const int nc = G.ncell;
  const uint8_t f = fl[c];
  const int P = G.dim * nc + c;
  for (int d = 0; d < G.dim; ++d) out[d * nc + c] = (mode == 2) ? a[d * nc + c] : 0.0;
  double pv = 0.0;
  if (f & FL_VOID) {
    if (mode == 0) pv = (f & FL_PIN) ? 0.0 : a[P];
    else if (mode == 1) pv = (f & FL_PIN) ? a[P] : -b[P];
    else pv = b[P];
  }
  out[P] = pv;
}

__global__ void k_zero_cells(Geo G, double* __restrict__ y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < G.ncell) y[G.dim * G.ncell + c] = 0.0;
}

// Dense pore blocks of L = B2 D^{-1} B1 (row-major, ld; zero-initialised): one thread per block row.
// Row of cell c: -sum 1/D_f over its face unknowns on the diagonal, +1/D_f at the cell across f when
// that cell is not pinned and lies in the same block.
template <typename ST>
__global__ void k_assemble_L(Geo G, const uint8_t* __restrict__ fl, const double* __restrict__ D, int nblk,
                             const long long* __restrict__ ioff, const int* __restrict__ bn,
                             const int* __restrict__ bld, const long long* __restrict__ moff,
                             const int* __restrict__ idx, long long n_total, ST* __restrict__ mat) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ioff[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const int b = lo;
  const int r = (int)(t - ioff[b]);
  const int n = bn[b];
  if (r >= n) return;
  const int* bidx = idx + ioff[b];
  const int nc = G.ncell;
  const int c = bidx[r] - G.dim * nc;
  CellPos p = cell_pos(G, c);
  ST* row = mat + moff[b] + (long long)r * bld[b];
  auto put = [&](int cell, double w) {
    if (fl[cell] & FL_PIN) return;
    const int key = G.dim * nc + cell;
    int a = 0, e = n;
    while (a < e) {
      int m = (a + e) >> 1;
      if (bidx[m] < key) a = m + 1;
      else e = m;
    }
    if (a < n && bidx[a] == key) row[a] = (ST)((double)row[a] + w);
  };
  double diag = 0.0;
  const uint8_t f = fl[c];
  for (int a = 0; a < G.dim; ++a) {
    if (f & fl_face(a)) {
      double w = 1.0 / D[a * nc + c];
      diag -= w;
      put(nbr(G, p, a, -1), w);
    }
    int h = nbr(G, p, a, +1);
    if (face_unknown(fl, a, h)) {
      double w = 1.0 / D[a * nc + h];
      diag -= w;
      put(h, w);
    }
  }
  row[r] = (ST)((double)row[r] + diag);
}

inline unsigned cells_grid(const Geo& G) { return (unsigned)((G.ncell + 255) / 256); }

}  // namespace

cudaError_t launch_diag_F(const Ctx& C, int op, const double* state, double* D) {
  pns::count_launch();
  k_diag_F<<<cells_grid(C.G), 256, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state, D);
  return cudaGetLastError();
}

cudaError_t launch_grad(const Ctx& C, const double* y, const double* D, const double* v, int mode, double* t) {
  pns::count_launch();
  k_grad<<<cells_grid(C.G), 256, 0, C.stream>>>(C.G, C.flags.as<uint8_t>(), y, D, v, mode, t);
  return cudaGetLastError();
}

cudaError_t launch_div(const Ctx& C, const double* t, const double* D, double sign, double* y) {
  pns::count_launch();
  k_div<<<cells_grid(C.G), 256, 0, C.stream>>>(C.G, C.flags.as<uint8_t>(), t, D, sign, y);
  return cudaGetLastError();
}

cudaError_t launch_compose(const Ctx& C, const double* a, const double* b, int mode, double* out) {
  pns::count_launch();
  k_compose<<<cells_grid(C.G), 256, 0, C.stream>>>(C.G, C.flags.as<uint8_t>(), a, b, mode, out);
  return cudaGetLastError();
}

cudaError_t launch_zero_cells(const Ctx& C, double* y) {
  pns::count_launch();
  k_zero_cells<<<cells_grid(C.G), 256, 0, C.stream>>>(C.G, y);
  return cudaGetLastError();
}

template <typename ST>
cudaError_t launch_assemble_L(const Ctx& C, const BlockSet& B, const double* D, ST* mat) {
  if (B.nblk == 0) return cudaSuccess;
  pns::count_launch();
  k_assemble_L<ST><<<(unsigned)((B.n_total + 127) / 128), 128, 0, C.stream>>>(
      C.G, C.flags.as<uint8_t>(), D, B.nblk, B.d_ioff.as<long long>(), B.d_n.as<int>(), B.d_ld.as<int>(),
      B.d_moff.as<long long>(), B.idx.as<int>(), B.n_total, mat);
  return cudaGetLastError();
}
template cudaError_t launch_assemble_L<double>(const Ctx&, const BlockSet&, const double*, double*);
template cudaError_t launch_assemble_L<float>(const Ctx&, const BlockSet&, const double*, float*);

}  // namespace pns
