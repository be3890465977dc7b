// Matrix-free MAC stencil kernels: the FP64 Navier-Stokes residual (Eq. 3) and y = b - A v for the
// Newton / Oseen (Eq. 27) / Stokes operators.  One thread per cell handles the dim face rows stored
// at the cell and its continuity row; neighbours come through L1/L2 (x-fastest layout keeps the
// +-x accesses of a warp contiguous).
#include "internal.h"

namespace pns {

namespace {

__device__ __forceinline__ double face_residual(const Geo& G, const Phy& P, const uint8_t* __restrict__ fl,
                                                int stokes, const double* __restrict__ x,
                                                const double* __restrict__ xprev, int d, const CellPos& p) {
  const int nc = G.ncell, c = p.c;
  const int R = d * nc + c;
  const double q = x[R];
  double acc = 0.0;
  if (P.inv_dt > 0) acc += P.rho * P.inv_dt * (q - (xprev ? xprev[R] : 0.0));
  const int lo = nbr(G, p, d, -1);
  const CellPos plo = cell_pos(G, lo);
  for (int a = 0; a < G.dim; ++a) {
    int np = nbr(G, p, a, +1), nm = nbr(G, p, a, -1);
    bool up = face_unknown(fl, d, np), um = face_unknown(fl, d, nm);
    double qp = up ? x[d * nc + np] : (a == d ? 0.0 : -q);
    double qm = um ? x[d * nc + nm] : (a == d ? 0.0 : -q);
    acc += P.mu * (2.0 * q - qp - qm);
    if (stokes) continue;
    double U;
    if (a == d) {
      U = q;
    } else {
      int f[4] = {lo, nbr(G, plo, a, +1), c, np};
      U = 0.0;
      for (int k = 0; k < 4; ++k)
        if (face_unknown(fl, a, f[k])) U += x[a * nc + f[k]];
      U *= 0.25;
    }
    acc += P.rho * (U >= 0.0 ? U * (q - qm) : U * (qp - q));
  }
  acc += x[G.dim * nc + c] - x[G.dim * nc + lo];
  acc -= P.rho * P.b[d];
  return acc;
}

__global__ void k_residual(Geo G, Phy P, const uint8_t* __restrict__ fl, int stokes, const double* __restrict__ x,
                           const double* __restrict__ xprev, double* __restrict__ r) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  const int nc = G.ncell;
  CellPos p = cell_pos(G, c);
  const uint8_t f = fl[c];
  for (int d = 0; d < G.dim; ++d)
    r[d * nc + c] = (f & fl_face(d)) ? face_residual(G, P, fl, stokes, x, xprev, d, p) : 0.0;
  double rp = 0.0;
  if (f & FL_PIN) {
    rp = x[G.dim * nc + c];
  } else if (f & FL_VOID) {
    for (int a = 0; a < G.dim; ++a) {
      int hi = nbr(G, p, a, +1);
      if (face_unknown(fl, a, hi)) rp += x[a * nc + hi];
      if (f & fl_face(a)) rp -= x[a * nc + c];
    }
  }
  r[G.dim * nc + c] = rp;
}

template <typename T, typename VT>
struct AccEmit {
  const VT* __restrict__ v;
  T acc;
  __device__ __forceinline__ void operator()(int col, T val) { acc += val * (T)v[col]; }
};

template <typename T, typename VT>
__global__ void k_apply(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                        const VT* __restrict__ v, const VT* __restrict__ b, VT* __restrict__ y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncell) return;
  const int nc = G.ncell;
  CellPos p = cell_pos(G, c);
  const uint8_t f = fl[c];
  for (int d = 0; d < G.dim; ++d) {
    const int R = d * nc + c;
    if (f & fl_face(d)) {
      AccEmit<T, VT> e{v, (T)0};
      face_row<T>(G, P, fl, op, st, d, p, e);
      y[R] = b ? (VT)((T)b[R] - e.acc) : (VT)e.acc;
    } else {
      y[R] = (VT)0;
    }
  }
  const int R = G.dim * nc + c;
  if (f & FL_VOID) {
    AccEmit<T, VT> e{v, (T)0};
    cell_row<T>(G, fl, p, e);
    y[R] = b ? (VT)((T)b[R] - e.acc) : (VT)e.acc;
  } else {
    y[R] = (VT)0;
  }
}

__global__ void k_cast_d2f(const double* __restrict__ in, float* __restrict__ out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long s = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += s) out[i] = (float)in[i];
}
__global__ void k_cast_f2d(const float* __restrict__ in, double* __restrict__ out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long s = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += s) out[i] = (double)in[i];
}

}  // namespace

cudaError_t launch_residual(const Ctx& C, int stokes, const double* x, const double* xprev, double* r) {
  int thr = 256, blk = (C.G.ncell + thr - 1) / thr;
  { pns::count_launch(); k_residual<<<blk, thr, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), stokes, x, xprev, r); }
  return cudaGetLastError();
}

template <typename VT>
cudaError_t launch_apply(const Ctx& C, int op, const double* state, const VT* v, const VT* b, VT* y, bool fp64_math) {
  int thr = 256, blk = (C.G.ncell + thr - 1) / thr;
  if (fp64_math)
    { pns::count_launch(); k_apply<double, VT><<<blk, thr, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state, v, b, y); }
  else
    { pns::count_launch(); k_apply<float, VT><<<blk, thr, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state, v, b, y); }
  return cudaGetLastError();
}
template cudaError_t launch_apply<double>(const Ctx&, int, const double*, const double*, const double*, double*, bool);
template cudaError_t launch_apply<float>(const Ctx&, int, const double*, const float*, const float*, float*, bool);

cudaError_t launch_cast_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  { pns::count_launch(); k_cast_d2f<<<1216, 256, 0, s>>>(in, out, n); }
  return cudaGetLastError();
}
cudaError_t launch_cast_f2d(const float* in, double* out, long long n, cudaStream_t s) {
  { pns::count_launch(); k_cast_f2d<<<1216, 256, 0, s>>>(in, out, n); }
  return cudaGetLastError();
}

}  // namespace pns
