// FP64 kernels of flexible GMRES (Saad 1993) with classical Gram-Schmidt applied twice (CGS2):
// fused multi-dot products V^T w, fused updates w -= V h, norms, the Hessenberg/Givens update and
// the final x += Z y, all on the device.  Reductions: per-thread FP64 sums, warp shuffles, one
// partial per CTA, then a fixed-order second pass (results do not depend on scheduling).
#include "internal.h"

namespace pns {

namespace {

constexpr int RED_BLOCKS = 1024;
constexpr int MAXV = 128;   // vectors per multidot pass (restart length + 1 at most)

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[i * nblk + blockIdx.x] = sum over this CTA's elements of V_i . w
__global__ void __launch_bounds__(256) k_multidot(const double* __restrict__ V, long long ld, int nvec,
                                                  const double* __restrict__ w, long long n,
                                                  double* __restrict__ partial) {
  __shared__ double sh[8][MAXV + 1];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < nvec; i0 += 8) {
    int cnt = min(8, nvec - i0);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
      double wv = w[e];
      for (int q = 0; q < cnt; ++q) acc[q] += V[(long long)(i0 + q) * ld + e] * wv;
    }
    for (int q = 0; q < cnt; ++q) {
      double s = warp_sum(acc[q]);
      if (lane == 0) sh[warp][i0 + q] = s;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double s = 0;
    for (int wv = 0; wv < 8; ++wv) s += sh[wv][i];
    partial[(long long)i * gridDim.x + blockIdx.x] = s;
  }
}

// out[i] = sum_b partial[i * nblk + b]   (one CTA per vector, fixed order)
__global__ void k_reduce_rows(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long long)blockIdx.x * nblk + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}

// w += sign * sum_i h[i] V_i
__global__ void k_multi_axpy(double* __restrict__ w, const double* __restrict__ V, long long ld, int nvec,
                             const double* __restrict__ h, double sign, long long n) {
  __shared__ double hs[MAXV];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = sign * h[i];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < nvec; ++i) acc += hs[i] * V[(long long)i * ld + e];
    w[e] = acc;
  }
}

__global__ void k_scale(double* __restrict__ x, long long n, const double* __restrict__ num,
                        const double* __restrict__ den, int invert) {
  double f = invert ? 1.0 / sqrt(*den) : *num;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    x[e] *= f;
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += a * x[e];
}

// column j of H: H[i][j] = h1[i] + h2[i] (i <= j), H[j+1][j] = sqrt(nrm2)
__global__ void k_hcol(double* __restrict__ H, int ldh, int j, const double* __restrict__ h1,
                       const double* __restrict__ h2, const double* __restrict__ nrm2) {
  int i = threadIdx.x;
  for (; i <= j; i += blockDim.x) H[(long long)i * ldh + j] = h1[i] + (h2 ? h2[i] : 0.0);
  if (threadIdx.x == 0) H[(long long)(j + 1) * ldh + j] = sqrt(*nrm2);
}

// apply the previous rotations to column j, form rotation j, update g; out[0] = |g[j+1]|
__global__ void k_givens(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, int j, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < j; ++i) {
    double a = H[(long long)i * ldh + j], b = H[(long long)(i + 1) * ldh + j];
    H[(long long)i * ldh + j] = cs[i] * a + sn[i] * b;
    H[(long long)(i + 1) * ldh + j] = -sn[i] * a + cs[i] * b;
  }
  double a = H[(long long)j * ldh + j], b = H[(long long)(j + 1) * ldh + j];
  double den = hypot(a, b);
  double c = den > 0 ? a / den : 1.0, s = den > 0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  H[(long long)j * ldh + j] = den;
  H[(long long)(j + 1) * ldh + j] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  out[0] = fabs(g[j + 1]);
  out[1] = H[(long long)(j + 1) * ldh + j];
}

// y = R^{-1} g (k x k upper triangle of H), single thread
__global__ void k_trisolve(const double* __restrict__ H, int ldh, const double* __restrict__ g, int k,
                           double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(long long)i * ldh + q] * y[q];
    y[i] = s / H[(long long)i * ldh + i];
  }
}

}  // namespace

cudaError_t launch_multidot(const double* V, long long ld, int nvec, const double* w, long long n, double* partial,
                            int nblocks, double* out, cudaStream_t s) {
  if (nblocks <= 0 || nblocks > RED_BLOCKS) nblocks = RED_BLOCKS;
  for (int i0 = 0; i0 < nvec; i0 += MAXV) {
    int cnt = nvec - i0 < MAXV ? nvec - i0 : MAXV;
    { pns::count_launch(); k_multidot<<<nblocks, 256, 0, s>>>(V + (long long)i0 * ld, ld, cnt, w, n, partial); }
    { pns::count_launch(); k_reduce_rows<<<cnt, 256, 0, s>>>(partial, nblocks, out + i0); }
  }
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(double* w, const double* V, long long ld, int nvec, const double* h, double sign,
                              long long n, cudaStream_t s) {
  for (int i0 = 0; i0 < nvec; i0 += MAXV) {
    int cnt = nvec - i0 < MAXV ? nvec - i0 : MAXV;
    { pns::count_launch(); k_multi_axpy<<<1216, 256, 0, s>>>(w, V + (long long)i0 * ld, ld, cnt, h + i0, sign, n); }
  }
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* a, const double* b, long long n, double* partial, double* out, cudaStream_t s) {
  { pns::count_launch(); k_multidot<<<RED_BLOCKS, 256, 0, s>>>(a, 0, 1, b, n, partial); }
  { pns::count_launch(); k_reduce_rows<<<1, 256, 0, s>>>(partial, RED_BLOCKS, out); }
  return cudaGetLastError();
}

// invert == 1: x *= 1 / sqrt(*den)
cudaError_t launch_scale(double* x, long long n, const double* num, const double* den, int invert, cudaStream_t s) {
  { pns::count_launch(); k_scale<<<1216, 256, 0, s>>>(x, n, num, den, invert); }
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t s) {
  { pns::count_launch(); k_axpy<<<1216, 256, 0, s>>>(y, x, a, n); }
  return cudaGetLastError();
}

cudaError_t launch_hcol(double* H, int ldh, int j, const double* h1, const double* h2, const double* hnorm,
                        cudaStream_t s) {
  { pns::count_launch(); k_hcol<<<1, 128, 0, s>>>(H, ldh, j, h1, h2, hnorm); }
  return cudaGetLastError();
}

cudaError_t launch_givens(double* H, int ldh, double* cs, double* sn, double* g, int j, double* resid_out,
                          cudaStream_t s) {
  { pns::count_launch(); k_givens<<<1, 32, 0, s>>>(H, ldh, cs, sn, g, j, resid_out); }
  return cudaGetLastError();
}

// y = R^{-1} g, then x += Z y
cudaError_t launch_trisolve_update(const double* H, int ldh, const double* g, int k, double* y, const double* Z,
                                   long long ld, double* x, long long n, cudaStream_t s) {
  { pns::count_launch(); k_trisolve<<<1, 32, 0, s>>>(H, ldh, g, k, y); }
  return launch_multi_axpy(x, Z, ld, k, y, 1.0, n, s);
}

}  // namespace pns
