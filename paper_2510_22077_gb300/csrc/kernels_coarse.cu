// Coarse level of M_G (Eqs. 14, 18, 20 with Remark 1):
//  * R^ v: one sum per contact interface over its cells and one per primary grid over all its
//    unknowns (segment sums, FP64 accumulation),
//  * P^ x^o: shape and correction vectors of each primary grid weighted by the coarse unknowns,
//    the interface value on interface cells, zero on interface faces,
//  * the inverse of the coarse matrix A^o by Gauss-Jordan with partial pivoting (FP64), and
//  * the coarse GEMV x^o = (A^o)^{-1} R^ v (FP64).
#include <cuda_bf16.h>

#include "internal.h"

namespace pns {

namespace {

__device__ __forceinline__ int find_seg(const long long* __restrict__ off, int n, long long t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;   // valid in thread 0
}

constexpr int SEG_CHUNK = 2048;

template <typename VT>
__global__ void k_seg_sum(const int2* __restrict__ items, const int* __restrict__ idx, const long long* __restrict__ off,
                          const VT* __restrict__ v, double* __restrict__ out) {
  int2 it = items[blockIdx.x];
  long long a = off[it.x] + (long long)it.y * SEG_CHUNK;
  long long e = min(off[it.x + 1], a + SEG_CHUNK);
  double s = 0.0;
  for (long long k = a + threadIdx.x; k < e; k += blockDim.x) s += (double)v[idx[k]];
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out + it.x, s);
}

__device__ __forceinline__ double ld_st(const double* p) { return *p; }
__device__ __forceinline__ double ld_st(const float* p) { return (double)*p; }

// z on primary unknowns: sum_k basis[r][k] * xo[colid[k]]
template <typename ST, typename VT>
__global__ void k_prolong_prim(int nblk, const long long* __restrict__ ioff, const int* __restrict__ bn,
                               const int* __restrict__ idx, long long n_total, const ST* __restrict__ basis,
                               const long long* __restrict__ boff, const int* __restrict__ kcv,
                               const int* __restrict__ colid, const int* __restrict__ coloff,
                               const double* __restrict__ xo, VT* __restrict__ z) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int b = find_seg(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  if (r >= bn[b]) return;
  int kc = kcv[b];
  const ST* row = basis + boff[b] + (long long)r * kc;
  const int* cid = colid + coloff[b];
  double s = 0.0;
  for (int k = 0; k < kc; ++k) s += ld_st(row + k) * xo[cid[k]];
  z[idx[t]] = (VT)s;
}

// z on interface cells = x^o of the interface
template <typename VT>
__global__ void k_prolong_iface(const int* __restrict__ seg_idx, const long long* __restrict__ seg_off, int n_iface,
                                const double* __restrict__ xo, VT* __restrict__ z) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = seg_off[n_iface];
  if (t >= tot) return;
  int j = find_seg(seg_off, n_iface, t);
  z[seg_idx[t]] = (VT)xo[j];
}

// Gauss-Jordan with partial pivoting, step t: pick pivot row, swap, normalise row t, save column t.
__global__ void k_cpiv(double* __restrict__ A, int n, int t, double* __restrict__ col, int* __restrict__ perm,
                       int* __restrict__ bad) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int arg = t;
  for (int i = t + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(A[(long long)i * n + t]);
    if (v > best) { best = v; arg = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      if (bv[threadIdx.x + s] > bv[threadIdx.x] ||
          (bv[threadIdx.x + s] == bv[threadIdx.x] && bi[threadIdx.x + s] < bi[threadIdx.x])) {
        bv[threadIdx.x] = bv[threadIdx.x + s];
        bi[threadIdx.x] = bi[threadIdx.x + s];
      }
    }
    __syncthreads();
  }
  int p = bi[0];
  double pv = A[(long long)p * n + t];
  if (!(bv[0] > 0.0) || !(bv[0] < 1e300)) {
    if (threadIdx.x == 0) atomicOr(bad, 1);
    pv = 1.0;
  }
  if (threadIdx.x == 0) perm[t] = p;
  __syncthreads();   // every thread has read the pivot value before any thread swaps rows t and p
  if (p != t)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double a = A[(long long)t * n + j];
      A[(long long)t * n + j] = A[(long long)p * n + j];
      A[(long long)p * n + j] = a;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = A[(long long)i * n + t];
  __syncthreads();
  double inv = 1.0 / pv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) A[(long long)t * n + j] = (j == t) ? inv : A[(long long)t * n + j] * inv;
}

__global__ void k_celim(double* __restrict__ A, int n, int t, const double* __restrict__ col) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  if (i == t) return;
  double f = col[i];
  if (j == t) A[e] = -f * A[(long long)t * n + t];
  else A[e] -= f * A[(long long)t * n + j];
}

// undo the row interchanges on the inverse: column swaps in reverse order
__global__ void k_cunperm(double* __restrict__ A, int n, const int* __restrict__ perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = A + (long long)i * n;
  for (int t = n - 1; t >= 0; --t) {
    int p = perm[t];
    if (p != t) {
      double a = row[t];
      row[t] = row[p];
      row[p] = a;
    }
  }
}

template <typename ST>
__global__ void k_cgemv(const ST* __restrict__ A, int n, const double* __restrict__ x, double* __restrict__ y) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  const ST* a = A + (long long)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += ld_st(a + j) * x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

}  // namespace

cudaError_t launch_seg_sum(const Precond& pc, const void* v, int vt_is_double, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double) * pc.n_o, s);
  if (pc.nseg_items == 0) return cudaGetLastError();
  if (vt_is_double)
    { pns::count_launch(); k_seg_sum<double><<<pc.nseg_items, 256, 0, s>>>(pc.seg_items.as<int2>(), pc.seg_idx.as<int>(),
                                                    pc.seg_off.as<long long>(), (const double*)v, out); }
  else
    { pns::count_launch(); k_seg_sum<float><<<pc.nseg_items, 256, 0, s>>>(pc.seg_items.as<int2>(), pc.seg_idx.as<int>(),
                                                   pc.seg_off.as<long long>(), (const float*)v, out); }
  return cudaGetLastError();
}

template <typename ST, typename VT>
cudaError_t launch_prolong(const Ctx& C, const Precond& pc, const double* xo, VT* z) {
  cudaMemsetAsync(z, 0, sizeof(VT) * C.nfull, C.stream);
  const BlockSet& B = pc.prim;
  if (B.nblk > 0) {
    long long blk = (B.n_total + 255) / 256;
    { pns::count_launch(); k_prolong_prim<ST, VT><<<(unsigned)blk, 256, 0, C.stream>>>(
        B.nblk, B.d_ioff.as<long long>(), B.d_n.as<int>(), B.idx.as<int>(), B.n_total, pc.basis.as<ST>(),
        pc.d_boff.as<long long>(), pc.d_kcols.as<int>(), pc.d_colid.as<int>(), pc.d_coloff.as<int>(), xo, z); }
  }
  int nif = pc.n_cif;
  if (nif > 0) {
    long long tot = 0;
    for (int j : C.M.coarse_ifaces) tot += (long long)C.M.iface_cells[j].size();
    long long blk = (tot + 255) / 256;
    { pns::count_launch(); k_prolong_iface<VT><<<(unsigned)blk, 256, 0, C.stream>>>(pc.seg_idx.as<int>(), pc.seg_off.as<long long>(), nif, xo, z); }
  }
  return cudaGetLastError();
}
template cudaError_t launch_prolong<double, double>(const Ctx&, const Precond&, const double*, double*);
template cudaError_t launch_prolong<float, float>(const Ctx&, const Precond&, const double*, float*);
template cudaError_t launch_prolong<float, double>(const Ctx&, const Precond&, const double*, double*);

cudaError_t launch_coarse_invert(double* A, int n, double* work, int* perm, int* d_bad, cudaStream_t s) {
  long long nn = (long long)n * n;
  unsigned blk = (unsigned)((nn + 255) / 256);
  for (int t = 0; t < n; ++t) {
    { pns::count_launch(); k_cpiv<<<1, 1024, 0, s>>>(A, n, t, work, perm, d_bad); }
    { pns::count_launch(); k_celim<<<blk, 256, 0, s>>>(A, n, t, work); }
  }
  { pns::count_launch(); k_cunperm<<<(n + 127) / 128, 128, 0, s>>>(A, n, perm); }
  return cudaGetLastError();
}

template <typename ST>
cudaError_t launch_coarse_gemv(const ST* Ainv, int n, const double* rhs, double* x, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  long long thr = (long long)n * 32;
  { pns::count_launch(); k_cgemv<ST><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(Ainv, n, rhs, x); }
  return cudaGetLastError();
}
template cudaError_t launch_coarse_gemv<double>(const double*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse_gemv<float>(const float*, int, const double*, double*, cudaStream_t);

}  // namespace pns
