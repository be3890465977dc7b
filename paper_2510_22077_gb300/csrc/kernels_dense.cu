// Dense local blocks of the PLMM preconditioner (Eq. 25 smoother blocks, Eqs. 6/9 closure blocks):
//  * assembly of A_b restricted to each block from the matrix-free stencil rows,
//  * batched, variable-size, blocked Gauss-Jordan inversion without pivoting (unknowns ordered
//    faces first, cells last, so the elimination is the velocity block followed by the pressure
//    Schur complement; a non-finite or zero pivot raises a flag),
//  * skinny products X * RHS (shape and correction vectors, Eqs. 15 and 17),
//  * the batched local solve z[idx] (+)= X * t[idx] used by every preconditioner application.
// Blocks are stored row-major with a leading dimension padded to 8 elements; padding is zero.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace pns {

namespace {

constexpr int TB = 64;   // Gauss-Jordan panel width == tile edge


__device__ __forceinline__ int find_block(const long long* __restrict__ off, int nb, long long t) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int lower_idx(const int* __restrict__ a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// small per-thread list of (column, value) with duplicates merged.  A stencil row has at most 17
// distinct columns in 3D (the face itself, 6 viscous neighbours, 2 pressures, 8 advecting faces of the
// Newton reaction term); 32 slots leave room.
struct RowList {
  int col[32];
  double val[32];
  int n;
  __device__ void operator()(int c, double v) {
    for (int k = 0; k < n; ++k)
      if (col[k] == c) { val[k] += v; return; }
    if (n < 32) { col[n] = c; val[n] = v; ++n; }
  }
};

// ------------------------------------------------------------------------------ assembly
template <typename ST>
__global__ void k_assemble(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                           const int* __restrict__ owner, int nblk, const long long* __restrict__ ioff,
                           const int* __restrict__ bn, const int* __restrict__ bld, const long long* __restrict__ moff,
                           const int* __restrict__ idx, long long n_total, ST* __restrict__ mat, int closure) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int b = find_block(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  int n = bn[b];
  if (r >= n) return;                              // padding slot of the packed layout
  const int* bidx = idx + ioff[b];
  int g = bidx[r];
  RowList L;
  L.n = 0;
  any_row<double>(G, P, fl, op, st, g, L);
  ST* row = mat + moff[b] + (long long)r * bld[b];
  int me = closure ? owner[g] : -100;
  double extra = 0.0;
  for (int k = 0; k < L.n; ++k) {
    int lc = lower_idx(bidx, n, L.col[k]);
    if (lc < n && bidx[lc] == L.col[k]) {
      row[lc] = (ST)((double)row[lc] + L.val[k]);
    } else if (closure) {
      int o = owner[L.col[k]];
      if (o == -3 || (o >= 0 && o != me)) extra += L.val[k];
    }
  }
  if (closure) row[r] = (ST)((double)row[r] + extra);
}

// ------------------------------------------------------------------------------ Gauss-Jordan
// Blocked Gauss-Jordan with panel width TBK (64 for FP64, 128 for FP32).  Step k: panel rows/cols
// [k*TBK, k*TBK + nb).  Active blocks are the first `cnt` of `order`.  256 threads per CTA; the panel
// kernels give each thread an R x R patch (R = TBK / 16).
// In-place inverse of the nb x nb diagonal block of step k, one CTA per active block.  Thread
// (ty, tx) of a 16 x 16 grid keeps the R x R patch (rows ty*R.., cols tx*R..) in registers.  Pivot t with
// p = D[t][t], written as one rank-1 update of every entry:
//   D[i][j] <- keep(i, j) D[i][j] - c[i] * r[j] / p,   keep = (i != t && j != t),
//   c[i] = D[i][t] (i != t), c[t] = -1;   r[j] = D[t][j] (j != t), r[t] = 1,
// which gives D[t][j] / p on the pivot row, -D[i][t] / p on the pivot column and 1 / p at the pivot (the
// Gauss-Jordan step, same roundings as the row-by-row form).  The owners of row and column t + 1 publish
// c, r and p into the other of two shared buffers right after their own update of step t, so one barrier
// per pivot suffices; the pivot's position inside a patch is a compile-time index (the steps are unrolled
// R at a time).  Rows and columns past nb are zero and stay zero.
template <typename ST, int TBK>
__global__ void __launch_bounds__(256) k_gj_diag(int k, const int* __restrict__ order, const int* __restrict__ bn,
                                                 const int* __restrict__ bld, const long long* __restrict__ moff,
                                                 ST* __restrict__ mat, int* __restrict__ bad) {
  constexpr int R = TBK / 16;
  __shared__ ST rbuf[2][TBK];
  __shared__ ST cbuf[2][TBK];
  __shared__ ST pbuf[2];
  const int b = order[blockIdx.x];
  const int n = bn[b], ld = bld[b];
  const int p0 = k * TBK;
  const int nb = min(TBK, n - p0);
  ST* A = mat + moff[b] + (long long)p0 * ld + p0;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int i0 = ty * R, j0 = tx * R;
  ST P[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int i = i0 + r, j = j0 + c;
      P[r][c] = (i < nb && j < nb) ? A[(long long)i * ld + j] : (ST)0;
    }
  // publish pivot t = o * R + rt into buffer q: its row (with 1 at the pivot), its column (with -1 at the
  // pivot) and its value, then clear the row and the column in the patches (the update refills them).
  // Called only with rt a compile-time constant (after unrolling), so P is indexed statically.
  auto publish = [&](int o, int rt, int q) {
    const ST pv = P[rt][rt];   // meaningful in the diagonal patch only
    if (ty == o) {
#pragma unroll
      for (int c = 0; c < R; ++c) {
        rbuf[q][j0 + c] = (tx == o && c == rt) ? (ST)1 : P[rt][c];
        P[rt][c] = (ST)0;
      }
    }
    if (tx == o) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cbuf[q][i0 + r] = (ty == o && r == rt) ? (ST)-1 : P[r][rt];
        P[r][rt] = (ST)0;
      }
    }
    if (ty == o && tx == o) pbuf[q] = pv;
  };
  int q = 0;
  if (nb > 0) publish(0, 0, 0);
  __syncthreads();
  for (int t0 = 0; t0 < nb; t0 += R) {
    const int o = t0 / R;
#pragma unroll
    for (int rt = 0; rt < R; ++rt) {
      if (t0 + rt < nb) {
        ST piv = pbuf[q];
        const bool okp = (piv == piv) && piv != (ST)0 && (double)fabs((double)piv) < 1e300;
        if (!okp) {
          if (threadIdx.x == 0) atomicOr(bad, 1);
          piv = (ST)1;
        }
        const ST inv = (ST)1 / piv;
        ST cr[R], rw[R];
#pragma unroll
        for (int r = 0; r < R; ++r) cr[r] = cbuf[q][i0 + r];
#pragma unroll
        for (int c = 0; c < R; ++c) rw[c] = rbuf[q][j0 + c] * inv;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < R; ++c) P[r][c] -= cr[r] * rw[c];
        if (t0 + rt + 1 < nb) publish(rt + 1 < R ? o : o + 1, (rt + 1) % R, q ^ 1);
        __syncthreads();
        q ^= 1;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int i = i0 + r, j = j0 + c;
      if (i < nb && j < nb) A[(long long)i * ld + j] = P[r][c];
    }
}

__device__ __forceinline__ int tile_skip(int t, int k) { return t + (t >= k); }

// A[P, J] <- Dinv * A[P, J] for every column tile J != k
template <typename ST, int TBK>
__global__ void k_gj_rowpanel(int k, int cnt, const int* __restrict__ order, const long long* __restrict__ pre1,
                              const int* __restrict__ bn, const int* __restrict__ bld,
                              const long long* __restrict__ moff, ST* __restrict__ mat) {
  constexpr int R = TBK / 16;
  extern __shared__ unsigned char smraw[];
  ST(*Dv)[TBK + 1] = (ST(*)[TBK + 1])smraw;
  ST(*Tl)[TBK + 1] = (ST(*)[TBK + 1])(smraw + sizeof(ST) * TBK * (TBK + 1));
  long long w = blockIdx.x;
  int s = find_block(pre1, cnt, w);
  int b = order[s];
  int jt = tile_skip((int)(w - pre1[s]), k);
  int n = bn[b], ld = bld[b];
  int p0 = k * TBK, j0 = jt * TBK;
  int nb = min(TBK, n - p0), nj = min(TBK, n - j0);
  ST* A = mat + moff[b];
  for (int e = threadIdx.x; e < TBK * TBK; e += blockDim.x) {
    int i = e / TBK, j = e % TBK;
    Dv[i][j] = (i < nb && j < nb) ? A[(long long)(p0 + i) * ld + p0 + j] : (ST)0;
    Tl[i][j] = (i < nb && j < nj) ? A[(long long)(p0 + i) * ld + j0 + j] : (ST)0;
  }
  __syncthreads();
  int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  ST acc[R][R] = {};
  for (int kk = 0; kk < nb; ++kk) {
    ST a[R], bb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = Dv[ty * R + i][kk];
#pragma unroll
    for (int j = 0; j < R; ++j) bb[j] = Tl[kk][tx * R + j];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] += a[i] * bb[j];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int r = ty * R + i, cc = tx * R + j;
      if (r < nb && cc < nj) A[(long long)(p0 + r) * ld + j0 + cc] = acc[i][j];
    }
}

// A[I, J] -= A[I, P] * A[P, J] for tiles I != k, J != k (FP64 path; the FP32 path uses k_gj_update_tcp or,
// with gj_tensor_cores 0 / 1, k_mm128_gj_update / k_mm128_gj_update_tc)
template <typename ST, int TBK>
__global__ void k_gj_update(int k, int cnt, const int* __restrict__ order, const long long* __restrict__ pre2,
                            const int* __restrict__ bn, const int* __restrict__ bld, const long long* __restrict__ moff,
                            ST* __restrict__ mat) {
  constexpr int R = TBK / 16;
  extern __shared__ unsigned char smraw[];
  ST(*As)[TBK + 1] = (ST(*)[TBK + 1])smraw;
  ST(*Bs)[TBK + 1] = (ST(*)[TBK + 1])(smraw + sizeof(ST) * TBK * (TBK + 1));
  long long w = blockIdx.x;
  int s = find_block(pre2, cnt, w);
  int b = order[s];
  int n = bn[b], ld = bld[b];
  int T = (n + TBK - 1) / TBK;
  long long loc = w - pre2[s];
  int it = tile_skip((int)(loc / (T - 1)), k), jt = tile_skip((int)(loc % (T - 1)), k);
  int p0 = k * TBK, i0 = it * TBK, j0 = jt * TBK;
  int nb = min(TBK, n - p0), ni = min(TBK, n - i0), nj = min(TBK, n - j0);
  ST* A = mat + moff[b];
  for (int e = threadIdx.x; e < TBK * TBK; e += blockDim.x) {
    int i = e / TBK, j = e % TBK;
    As[i][j] = (i < ni && j < nb) ? A[(long long)(i0 + i) * ld + p0 + j] : (ST)0;
    Bs[i][j] = (i < nb && j < nj) ? A[(long long)(p0 + i) * ld + j0 + j] : (ST)0;
  }
  __syncthreads();
  int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  ST acc[R][R] = {};
  for (int kk = 0; kk < nb; ++kk) {
    ST a[R], bb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = As[ty * R + i][kk];
#pragma unroll
    for (int j = 0; j < R; ++j) bb[j] = Bs[kk][tx * R + j];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] += a[i] * bb[j];
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int r = ty * R + i, cc = tx * R + j;
      if (r < ni && cc < nj) {
        ST* q = A + (long long)(i0 + r) * ld + j0 + cc;
        *q = *q - acc[i][j];
      }
    }
}

// A[I, P] <- -A[I, P] * Dinv for row tiles I != k
template <typename ST, int TBK>
__global__ void k_gj_colpanel(int k, int cnt, const int* __restrict__ order, const long long* __restrict__ pre1,
                              const int* __restrict__ bn, const int* __restrict__ bld,
                              const long long* __restrict__ moff, ST* __restrict__ mat) {
  constexpr int R = TBK / 16;
  extern __shared__ unsigned char smraw[];
  ST(*Dv)[TBK + 1] = (ST(*)[TBK + 1])smraw;
  ST(*Tl)[TBK + 1] = (ST(*)[TBK + 1])(smraw + sizeof(ST) * TBK * (TBK + 1));
  long long w = blockIdx.x;
  int s = find_block(pre1, cnt, w);
  int b = order[s];
  int it = tile_skip((int)(w - pre1[s]), k);
  int n = bn[b], ld = bld[b];
  int p0 = k * TBK, i0 = it * TBK;
  int nb = min(TBK, n - p0), ni = min(TBK, n - i0);
  ST* A = mat + moff[b];
  for (int e = threadIdx.x; e < TBK * TBK; e += blockDim.x) {
    int i = e / TBK, j = e % TBK;
    Dv[i][j] = (i < nb && j < nb) ? A[(long long)(p0 + i) * ld + p0 + j] : (ST)0;
    Tl[i][j] = (i < ni && j < nb) ? A[(long long)(i0 + i) * ld + p0 + j] : (ST)0;
  }
  __syncthreads();
  int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  ST acc[R][R] = {};
  for (int kk = 0; kk < nb; ++kk) {
    ST a[R], bb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = Tl[ty * R + i][kk];
#pragma unroll
    for (int j = 0; j < R; ++j) bb[j] = Dv[kk][tx * R + j];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] += a[i] * bb[j];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int r = ty * R + i, cc = tx * R + j;
      if (r < ni && cc < nb) A[(long long)(i0 + r) * ld + p0 + cc] = -acc[i][j];
    }
}

// ------------------------------------------------------------------------------ FP32 tile GEMM
// acc (128 x 128 per CTA, 8 x 8 per thread) = A[rows, 0:K) * B[0:K, cols], both row-major FP32.
// K is staged through shared memory in chunks of 32, double-buffered: the next chunk is fetched
// into registers while the current one is multiplied.  A is stored k-major in shared memory so that
// every thread reads its 8 rows as two float4; B is stored as is.  Thread (ty, tx) owns rows
// {4ty..4ty+3, 64+4ty..64+4ty+3} and the same pattern of columns in tx.
constexpr int MT = 128;
constexpr int KC = 32;
constexpr int SROW = MT + 4;   // 16-byte aligned rows; k-major stores of A hit distinct banks

struct MmSmem {
  float a[2][KC][SROW];
  float b[2][KC][SROW];
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// rows_ok: rows of A that may be read (row < rows_ok); a_cols_ok: columns of A that may be read;
// cols_ok: columns of B that may be read; K: length of the contraction (A columns and B rows past K
// count as zero).  lda, ldb, a_cols_ok, cols_ok multiples of 4; A, B 16-byte aligned.
// B goes to shared memory by cp.async (zero-filled outside the valid range); A passes through
// registers because it is transposed on the way.
__device__ __forceinline__ void mm128_mainloop(const float* __restrict__ A, long long lda, int rows_ok,
                                               const float* __restrict__ B, long long ldb, int cols_ok, int K,
                                               int a_cols_ok, float acc[8][8], MmSmem& sm) {
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  float4 ra[4];
  auto fetch = [&](int c0, int st) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      int q = tid + rep * 256;
      // A: row i, four consecutive k starting at kq
      int i = q % MT, kq = (q / MT) * 4;
      int kg = c0 + kq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < rows_ok && kg < a_cols_ok) {
        v = *reinterpret_cast<const float4*>(A + (long long)i * lda + kg);
        if (kg + 0 >= K) v.x = 0.f;
        if (kg + 1 >= K) v.y = 0.f;
        if (kg + 2 >= K) v.z = 0.f;
        if (kg + 3 >= K) v.w = 0.f;
      }
      ra[rep] = v;
      // B: row kk, four consecutive columns, straight to shared memory
      int kk = q / 32, c = (q % 32) * 4;
      bool ok = (c0 + kk < K) && (c < cols_ok);
      const float* src = ok ? B + (long long)(c0 + kk) * ldb + c : B;
      cp_async16(&sm.b[st][kk][c], src, ok ? 16 : 0);
    }
    cp_async_commit();
  };
  auto stash = [&](int st) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      int q = tid + rep * 256;
      int i = q % MT, kq = (q / MT) * 4;
      sm.a[st][kq + 0][i] = ra[rep].x;
      sm.a[st][kq + 1][i] = ra[rep].y;
      sm.a[st][kq + 2][i] = ra[rep].z;
      sm.a[st][kq + 3][i] = ra[rep].w;
    }
  };
  const int nchunk = (K + KC - 1) / KC;
  fetch(0, 0);
  stash(0);
  cp_async_wait_all();
  __syncthreads();
  for (int ch = 0; ch < nchunk; ++ch) {
    const int st = ch & 1;
    if (ch + 1 < nchunk) fetch((ch + 1) * KC, st ^ 1);
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&sm.a[st][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sm.a[st][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sm.b[st][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sm.b[st][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    if (ch + 1 < nchunk) {
      stash(st ^ 1);
      cp_async_wait_all();
    }
    __syncthreads();
  }
}

// Same staging as mm128_mainloop, product on the tensor cores: mma.sync m16n8k8 TF32 with FP32
// accumulation, each operand split as x = hi + lo (hi = x rounded to TF32, lo = the remainder rounded
// to TF32) and acc += hi*hi + hi*lo + lo*hi, which keeps the product close to FP32 accuracy.  Warp w
// owns the 64 x 32 sub-tile at rows 64*(w/4), columns 32*(w%4): 4 x 4 MMA tiles of 16 x 8.
// Fragment layout of m16n8k8 (g = lane/4, t = lane%4): A rows g, g+8 and k t, t+4; B k t, t+4 and
// column g; C rows g, g+8 and columns 2t, 2t+1.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mm128_mainloop_tc(const float* __restrict__ A, long long lda, int rows_ok,
                                                  const float* __restrict__ B, long long ldb, int cols_ok, int K,
                                                  int a_cols_ok, float acc[4][4][4], MmSmem& sm) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  float4 ra[4];
  auto fetch = [&](int c0, int st) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      int q = tid + rep * 256;
      int i = q % MT, kq = (q / MT) * 4;
      int kg = c0 + kq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < rows_ok && kg < a_cols_ok) {
        v = *reinterpret_cast<const float4*>(A + (long long)i * lda + kg);
        if (kg + 0 >= K) v.x = 0.f;
        if (kg + 1 >= K) v.y = 0.f;
        if (kg + 2 >= K) v.z = 0.f;
        if (kg + 3 >= K) v.w = 0.f;
      }
      ra[rep] = v;
      int kk = q / 32, c = (q % 32) * 4;
      bool ok = (c0 + kk < K) && (c < cols_ok);
      const float* src = ok ? B + (long long)(c0 + kk) * ldb + c : B;
      cp_async16(&sm.b[st][kk][c], src, ok ? 16 : 0);
    }
    cp_async_commit();
  };
  auto stash = [&](int st) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      int q = tid + rep * 256;
      int i = q % MT, kq = (q / MT) * 4;
      sm.a[st][kq + 0][i] = ra[rep].x;
      sm.a[st][kq + 1][i] = ra[rep].y;
      sm.a[st][kq + 2][i] = ra[rep].z;
      sm.a[st][kq + 3][i] = ra[rep].w;
    }
  };
  const int nchunk = (K + KC - 1) / KC;
  fetch(0, 0);
  stash(0);
  cp_async_wait_all();
  __syncthreads();
  for (int ch = 0; ch < nchunk; ++ch) {
    const int st = ch & 1;
    if (ch + 1 < nchunk) fetch((ch + 1) * KC, st ^ 1);
#pragma unroll
    for (int k8 = 0; k8 < KC; k8 += 8) {
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int col = wn + ni * 8 + g;
        split_tf32(sm.b[st][k8 + t4][col], bh[ni][0], bl[ni][0]);
        split_tf32(sm.b[st][k8 + t4 + 4][col], bh[ni][1], bl[ni][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int row = wm + mi * 16 + g;
        uint32_t ah[4], al[4];
        split_tf32(sm.a[st][k8 + t4][row], ah[0], al[0]);
        split_tf32(sm.a[st][k8 + t4][row + 8], ah[1], al[1]);
        split_tf32(sm.a[st][k8 + t4 + 4][row], ah[2], al[2]);
        split_tf32(sm.a[st][k8 + t4 + 4][row + 8], ah[3], al[3]);
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          mma_tf32(acc[mi][ni], al, bh[ni]);
          mma_tf32(acc[mi][ni], ah, bl[ni]);
          mma_tf32(acc[mi][ni], ah, bh[ni]);
        }
      }
    }
    if (ch + 1 < nchunk) {
      stash(st ^ 1);
      cp_async_wait_all();
    }
    __syncthreads();
  }
}

// Gauss-Jordan trailing update on the tensor cores (3-term TF32 split); same tiles as
// k_mm128_gj_update.
__global__ void __launch_bounds__(256, 2) k_mm128_gj_update_tc(int k, int cnt, const int* __restrict__ order,
                                                               const long long* __restrict__ pre2,
                                                               const int* __restrict__ bn, const int* __restrict__ bld,
                                                               const long long* __restrict__ moff,
                                                               float* __restrict__ mat) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MmSmem& sm = *reinterpret_cast<MmSmem*>(smraw);
  long long w = blockIdx.x;
  int s = find_block(pre2, cnt, w);
  int b = order[s];
  int n = bn[b], ld = bld[b];
  int T = (n + MT - 1) / MT;
  long long loc = w - pre2[s];
  int it = tile_skip((int)(loc / (T - 1)), k), jt = tile_skip((int)(loc % (T - 1)), k);
  int p0 = k * MT, i0 = it * MT, j0 = jt * MT;
  int nb = min(MT, n - p0);
  int rows_ok = min(MT, ld - i0), cols_ok = min(MT, ld - j0);
  float* Ab = mat + moff[b];
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][c][e] = 0.f;
  mm128_mainloop_tc(Ab + (long long)i0 * ld + p0, ld, rows_ok, Ab + (long long)p0 * ld + j0, ld, cols_ok, nb,
                    ld - p0, acc, sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = wm + mi * 16 + g + h * 8;
      if (r >= rows_ok) continue;
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn + ni * 8 + 2 * t4;
        if (c >= cols_ok) continue;
        float2* q = reinterpret_cast<float2*>(Ab + (long long)(i0 + r) * ld + j0 + c);
        float2 v = *q;
        v.x -= acc[mi][ni][2 * h + 0];
        v.y -= acc[mi][ni][2 * h + 1];
        *q = v;
      }
    }
}

__device__ __forceinline__ int mm_row(int ty, int i) { return (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4); }

// Gauss-Jordan trailing update, FP32, panel width 128: A[I, J] -= A[I, P] * A[P, J] for I, J != k.
// Rows and columns are processed up to the padded leading dimension (padding is zero and stays so).
__global__ void __launch_bounds__(256, 2) k_mm128_gj_update(int k, int cnt, const int* __restrict__ order,
                                                            const long long* __restrict__ pre2,
                                                            const int* __restrict__ bn, const int* __restrict__ bld,
                                                            const long long* __restrict__ moff, float* __restrict__ mat) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MmSmem& sm = *reinterpret_cast<MmSmem*>(smraw);
  long long w = blockIdx.x;
  int s = find_block(pre2, cnt, w);
  int b = order[s];
  int n = bn[b], ld = bld[b];
  int T = (n + MT - 1) / MT;
  long long loc = w - pre2[s];
  int it = tile_skip((int)(loc / (T - 1)), k), jt = tile_skip((int)(loc % (T - 1)), k);
  int p0 = k * MT, i0 = it * MT, j0 = jt * MT;
  int nb = min(MT, n - p0);
  int rows_ok = min(MT, ld - i0), cols_ok = min(MT, ld - j0);
  float* Ab = mat + moff[b];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  mm128_mainloop(Ab + (long long)i0 * ld + p0, ld, rows_ok, Ab + (long long)p0 * ld + j0, ld, cols_ok, nb,
                 ld - p0, acc, sm);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r = mm_row(ty, i);
    if (r >= rows_ok) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int c = h * 64 + tx * 4;
      if (c >= cols_ok) continue;
      float4* q = reinterpret_cast<float4*>(Ab + (long long)(i0 + r) * ld + j0 + c);
      float4 v = *q;
      v.x -= acc[i][h * 4 + 0];
      v.y -= acc[i][h * 4 + 1];
      v.z -= acc[i][h * 4 + 2];
      v.w -= acc[i][h * 4 + 3];
      *q = v;
    }
  }
}

// Newton-Schulz product T = X * R per entry (n x n, FP32, 128 x 128 tiles over the padded ld).
__global__ void __launch_bounds__(256, 2) k_mm128_ns(const int* __restrict__ lst, const long long* __restrict__ tilepre,
                                                     int nent, const int* __restrict__ bn, const int* __restrict__ bld,
                                                     const long long* __restrict__ moff, const float* __restrict__ mat,
                                                     const long long* __restrict__ soff, const float* __restrict__ R,
                                                     float* __restrict__ Tout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MmSmem& sm = *reinterpret_cast<MmSmem*>(smraw);
  long long w = blockIdx.x;
  int e = find_block(tilepre, nent, w);
  int b = lst[e];
  int n = bn[b], ld = bld[b];
  int T = (n + MT - 1) / MT;
  long long loc = w - tilepre[e];
  int it = (int)(loc / T), jt = (int)(loc % T);
  int i0 = it * MT, j0 = jt * MT;
  int rows_ok = min(MT, ld - i0), cols_ok = min(MT, ld - j0);
  const float* X = mat + moff[b];
  const float* Rm = R + soff[e];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  mm128_mainloop(X + (long long)i0 * ld, ld, rows_ok, Rm + j0, ld, cols_ok, n, ld, acc, sm);
  float* To = Tout + soff[e];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r = mm_row(ty, i);
    if (r >= rows_ok) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int c = h * 64 + tx * 4;
      if (c >= cols_ok) continue;
      *reinterpret_cast<float4*>(To + (long long)(i0 + r) * ld + j0 + c) =
          make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
    }
  }
}

// ------------------------------------------------------------------------------ closure RHS
// rhs (n_i x kc_i, row-major, FP64) of primary grid i: column k < kc-1 = -sum_{cells of interface
// C_i[k]} A_b[row, cell] (so that X * rhs is the shape vector), last column = b_B (rho b_d on face
// rows, 0 on cell rows).
__global__ void k_closure_rhs(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                              const int* __restrict__ cell_iface, int nblk, const long long* __restrict__ ioff,
                              const int* __restrict__ bn, const int* __restrict__ idx, long long n_total,
                              const int* __restrict__ colbase, const int* __restrict__ cols,
                              const long long* __restrict__ roff, const int* __restrict__ kcv,
                              double* __restrict__ rhs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int b = find_block(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  if (r >= bn[b]) return;
  int g = idx[t];
  int kc = kcv[b];
  double* out = rhs + roff[b] + (long long)r * kc;
  const int* myc = cols + colbase[b];
  RowList L;
  L.n = 0;
  any_row<double>(G, P, fl, op, st, g, L);
  for (int k = 0; k < L.n; ++k) {
    int is_cell, d, c;
    decode(G, L.col[k], is_cell, d, c);
    if (!is_cell) continue;
    int j = cell_iface[c];
    if (j < 0) continue;
    int pos = lower_idx(myc, kc - 1, j);
    if (pos < kc - 1 && myc[pos] == j) out[pos] -= L.val[k];
  }
  int is_cell, d, c;
  decode(G, g, is_cell, d, c);
  out[kc - 1] = is_cell ? 0.0 : P.rho * P.b[d];
}

// ------------------------------------------------------------------------------ X * RHS
// Y_b = X_b R_b for every block of a set (X_b: n x n FP32 / FP64 rows at leading dimension ld; R_b, Y_b:
// n x kc FP64 rows at offset roff[b]): the products of the closure solves.  kc = |C_i| + 1 is small (2 to
// ~30), so this is a skinny product whose cost is the one stream of X.  A CTA takes 8 RW rows of one block
// and KQ columns of R (item = (block, first row, first column of R)): warp w keeps rows RW w.. of Y in
// registers, and per 128-column chunk of X each lane loads 4 consecutive columns of each of its rows
// (16 bytes) and multiplies them with the matching 4 rows of the chunk of R, which the CTA stages in
// shared memory transposed (Rs[q][c], one 16-byte read per lane and column q).  Lane partials are summed
// by butterfly shuffles at the end.  Accumulation in the storage precision of X.
template <typename ST, int KQ, int RW>
__global__ void __launch_bounds__(256) k_block_mm_s(const int4* __restrict__ items, const int* __restrict__ bn,
                                                    const int* __restrict__ bld, const long long* __restrict__ moff,
                                                    const ST* __restrict__ mat, const double* __restrict__ rhs,
                                                    const long long* __restrict__ roff, const int* __restrict__ kcv,
                                                    double* __restrict__ out) {
  constexpr int CK = 128, CKP = CK + 4;
  __shared__ __align__(16) ST Rs[KQ][CKP];
  const int4 it = items[blockIdx.x];
  const int b = it.x, r0 = it.y, q0 = it.z;
  const int n = bn[b], ld = bld[b], kc = kcv[b];
  const int qn = min(KQ, kc - q0);
  const ST* X = mat + moff[b];
  const double* R = rhs + roff[b];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw0 = r0 + warp * RW;
  ST acc[RW][KQ];
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int q = 0; q < KQ; ++q) acc[i][q] = (ST)0;
  for (int c0 = 0; c0 < n; c0 += CK) {
    __syncthreads();
    // stage R[c0 .. c0 + 127][q0 .. q0 + KQ) transposed; consecutive threads walk q first (coalesced reads)
    for (int e = threadIdx.x; e < KQ * CK; e += blockDim.x) {
      const int q = e % KQ, c = e / KQ;
      Rs[q][c] = (q < qn && c0 + c < n) ? (ST)R[(long long)(c0 + c) * kc + q0 + q] : (ST)0;
    }
    __syncthreads();
    const int c = c0 + 4 * lane;
    ST xv[RW][4];
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      const int row = rw0 + i;
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[i][u] = (ST)0;
      if (row < n && c < n) {
        // c is a multiple of 4 below n <= ld (a multiple of 8): the 4 columns lie inside the row
        const ST* xr = X + (long long)row * ld + c;
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[i][u] = (c + u < n) ? xr[u] : (ST)0;
      }
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const ST* rq = &Rs[q][4 * lane];
      const ST r_0 = rq[0], r_1 = rq[1], r_2 = rq[2], r_3 = rq[3];
#pragma unroll
      for (int i = 0; i < RW; ++i) acc[i][q] += xv[i][0] * r_0 + xv[i][1] * r_1 + xv[i][2] * r_2 + xv[i][3] * r_3;
    }
  }
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int row = rw0 + i;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      ST v = acc[i][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && row < n && q < qn) out[roff[b] + (long long)row * kc + q0 + q] = (double)v;
    }
  }
}

// ------------------------------------------------------------------------------ local solve
template <typename PT>
__global__ void k_gather(const int* __restrict__ idx, long long n_total, const double* __restrict__ t,
                         PT* __restrict__ pk) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_total) return;
  int g = idx[i];
  pk[i] = g >= 0 ? (PT)t[g] : (PT)0;
}

// vector load helpers: 16 bytes of the row and of x
__device__ __forceinline__ float dot16(const float* a, const float* x) {
  float4 u = *reinterpret_cast<const float4*>(a);
  float4 v = *reinterpret_cast<const float4*>(x);
  return u.x * v.x + u.y * v.y + u.z * v.z + u.w * v.w;
}
__device__ __forceinline__ double dot16(const double* a, const double* x) {
  double2 u = *reinterpret_cast<const double2*>(a);
  double2 v = *reinterpret_cast<const double2*>(x);
  return u.x * v.x + u.y * v.y;
}
__device__ __forceinline__ float dot16(const __nv_bfloat16* a, const float* x) {
  uint4 raw = *reinterpret_cast<const uint4*>(a);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
  float4 v0 = *reinterpret_cast<const float4*>(x);
  float4 v1 = *reinterpret_cast<const float4*>(x + 4);
  float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
  float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
  return f0.x * v0.x + f0.y * v0.y + f1.x * v0.z + f1.y * v0.w + f2.x * v1.x + f2.y * v1.y + f3.x * v1.z +
         f3.y * v1.w;
}
template <typename ST> struct VecW { static constexpr int n = 16 / sizeof(ST); };

// Batched local solve z = X_i t_i for every block of a set in one persistent launch: the work items are
// binned by block size (largest blocks first) and each item carries its bin's shape, L lanes per row
// (8, 16 or 32; 256 / L rows in flight per CTA) and its row count (chosen per bin by pns_autotune).  CTAs
// take items from a global counter until the list is exhausted.  Item = (block, first row, rows, L).
// Output (FP64) by `mode`: 0 z[idx[row]] = y, 1 z[idx[row]] += y (atomic: overlapping dual grids),
// 2 packed zp[row] = y, 3 packed zp[row] += y.  The dot products run in the packed type PT (FP32 for the
// FP32/BF16 inverses): per-lane partial sums, the lane partials added in FP64.
template <typename ST, typename PT>
__global__ void __launch_bounds__(256) k_local_gemv_p(const int4* __restrict__ items, int nitems,
                                                      int* __restrict__ counter, const int* __restrict__ idx,
                                                      const long long* __restrict__ ioff, const int* __restrict__ bld,
                                                      const long long* __restrict__ moff, const ST* __restrict__ mat,
                                                      const PT* __restrict__ pk, double* __restrict__ z, int mode) {
  __shared__ int s_item;
  constexpr int W = VecW<ST>::n;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= nitems) return;
    const int4 it = items[i];
    const int L = it.w;
    const int groups = 256 / L;
    const int g = threadIdx.x / L, lane = threadIdx.x % L;
    const int b = it.x;
    const int ld = bld[b];
    const PT* x = pk + ioff[b];
    const ST* M = mat + moff[b];
    const int end = it.y + it.z;
    // the trip count is uniform within a warp (all its lane groups step together) so that the shuffles
    // below see every lane
    for (int base = it.y; base < end; base += groups) {
      const int r = base + g;
      PT acc = (PT)0;
      if (r < end) {
        const ST* row = M + (long long)r * ld;
        for (int c = lane * W; c < ld; c += L * W) acc += dot16(row + c, x + c);
      }
      double a = (double)acc;
      for (int o = L >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, L);
      if (lane == 0 && r < end) {
        const long long slot = ioff[b] + r;
        if (mode == 0) z[idx[slot]] = a;
        else if (mode == 1) atomicAdd(z + idx[slot], a);
        else if (mode == 2) z[slot] = a;
        else z[slot] += a;
      }
    }
  }
}

// Local residual of the apply-time refinement, per packed slot of a block set:
// out[slot] = t[g] - sum_{c in block} A_b[g, c] zp[slot(c)]  (FP64 from the exact stencil row of g;
// padding slots get 0).  The second pass of the local GEMV then adds X * out to zp.
template <typename PT>
__global__ void k_local_residual(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                                 int nblk, const long long* __restrict__ ioff, const int* __restrict__ bn,
                                 const int* __restrict__ idx, long long n_total, const double* __restrict__ t,
                                 const double* __restrict__ zp, PT* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_total) return;
  const int b = find_block(ioff, nblk, i);
  const int r = (int)(i - ioff[b]);
  const int n = bn[b];
  if (r >= n) {
    out[i] = (PT)0;
    return;
  }
  const int* bidx = idx + ioff[b];
  const double* zb = zp + ioff[b];
  const int g = bidx[r];
  RowList L;
  L.n = 0;
  any_row<double>(G, P, fl, op, st, g, L);
  double acc = t[g];
  for (int k = 0; k < L.n; ++k) {
    int lc = lower_idx(bidx, n, L.col[k]);
    if (lc < n && bidx[lc] == L.col[k]) acc -= L.val[k] * zb[lc];
  }
  out[i] = (PT)acc;
}

// z[idx[slot]] = zp[slot] (add: atomicAdd) for the real slots of a block set
__global__ void k_scatter_packed(const int* __restrict__ idx, long long n_total, const double* __restrict__ zp,
                                 double* __restrict__ z, int add) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_total) return;
  const int g = idx[i];
  if (g < 0) return;
  if (add) atomicAdd(z + g, zp[i]);
  else z[g] = zp[i];
}

// ------------------------------------------------------------------------------ refinement
// Newton-Schulz step X <- X + X (I - A X) for blocks whose residual exceeds a threshold.  The
// residual is formed in FP64 from the exact stencil coefficients of A (sparse rows), so the refined
// inverse is accurate to the storage precision even when the Gauss-Jordan pass was run in FP32.
//
// Work lists address a subset of a BlockSet: entry e -> block lst[e], scratch offset soff[e].

// R[r][:] = e_r - sum_k a_rk X[k][:]  (stored in the scratch of entry e, compute type AT); also
// rmax[e] = max |R| of the block (as float bits, atomicMax on non-negative floats)
template <typename ST, typename RT>
__global__ void k_ns_residual(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                              const int* __restrict__ owner, int closure, const int* __restrict__ lst,
                              const long long* __restrict__ rowpre, int nent, const long long* __restrict__ ioff,
                              const int* __restrict__ bn, const int* __restrict__ bld,
                              const long long* __restrict__ moff, const int* __restrict__ idx,
                              const ST* __restrict__ mat, const long long* __restrict__ soff, RT* __restrict__ R,
                              unsigned int* __restrict__ rmax) {
  __shared__ int scol[32];
  __shared__ double sval[32];
  __shared__ int sn;
  long long w = blockIdx.x;
  int e = find_block(rowpre, nent, w);
  int b = lst[e];
  int r = (int)(w - rowpre[e]);
  int n = bn[b], ld = bld[b];
  const int* bidx = idx + ioff[b];
  if (threadIdx.x == 0) {
    RowList L;
    L.n = 0;
    int g = bidx[r];
    any_row<double>(G, P, fl, op, st, g, L);
    int me = closure ? owner[g] : -100;
    double extra = 0.0;
    int m = 0;
    int diagpos = -1;
    for (int k = 0; k < L.n; ++k) {
      int lc = lower_idx(bidx, n, L.col[k]);
      if (lc < n && bidx[lc] == L.col[k]) {
        scol[m] = lc;
        sval[m] = L.val[k];
        if (lc == r) diagpos = m;
        ++m;
      } else if (closure) {
        int o = owner[L.col[k]];
        if (o == -3 || (o >= 0 && o != me)) extra += L.val[k];
      }
    }
    if (closure && extra != 0.0) {
      if (diagpos < 0) { scol[m] = r; sval[m] = extra; ++m; }
      else sval[diagpos] += extra;
    }
    sn = m;
  }
  __syncthreads();
  const ST* X = mat + moff[b];
  RT* Rr = R + soff[e] + (long long)r * ld;
  float lmax = 0.f;
  for (int j = threadIdx.x; j < ld; j += blockDim.x) {
    double acc = (j == r) ? 1.0 : 0.0;
    if (j < n)
      for (int k = 0; k < sn; ++k) acc -= sval[k] * (double)X[(long long)scol[k] * ld + j];
    else
      acc = 0.0;
    Rr[j] = (RT)acc;
    lmax = fmaxf(lmax, (float)fabs(acc));
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(rmax + e, __float_as_uint(lmax));
}

// T = X * R per entry (n x n), 64x64 tiles, K in steps of 64; compute type AT
template <typename ST, typename RT, typename AT>
__global__ void k_ns_gemm(const int* __restrict__ lst, const long long* __restrict__ tilepre, int nent,
                          const int* __restrict__ bn, const int* __restrict__ bld, const long long* __restrict__ moff,
                          const ST* __restrict__ mat, const long long* __restrict__ soff, const RT* __restrict__ R,
                          AT* __restrict__ Tout) {
  extern __shared__ unsigned char smraw[];
  AT(*As)[TB + 1] = (AT(*)[TB + 1])smraw;
  AT(*Bs)[TB + 1] = (AT(*)[TB + 1])(smraw + sizeof(AT) * TB * (TB + 1));
  long long w = blockIdx.x;
  int e = find_block(tilepre, nent, w);
  int b = lst[e];
  int n = bn[b], ld = bld[b];
  int T = (n + TB - 1) / TB;
  long long loc = w - tilepre[e];
  int it = (int)(loc / T), jt = (int)(loc % T);
  int i0 = it * TB, j0 = jt * TB;
  const ST* X = mat + moff[b];
  const RT* Rm = R + soff[e];
  int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  AT acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += TB) {
    __syncthreads();
    for (int q = threadIdx.x; q < TB * TB; q += blockDim.x) {
      int i = q / TB, j = q % TB;
      As[i][j] = (i0 + i < n && k0 + j < n) ? (AT)X[(long long)(i0 + i) * ld + k0 + j] : (AT)0;
      Bs[i][j] = (k0 + i < n && j0 + j < n) ? (AT)Rm[(long long)(k0 + i) * ld + j0 + j] : (AT)0;
    }
    __syncthreads();
    for (int kk = 0; kk < TB; ++kk) {
      AT a[4], bb[4];
      for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][kk];
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
  }
  AT* To = Tout + soff[e];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int r = i0 + ty * 4 + i, c = j0 + tx * 4 + j;
      if (r < n && c < n) To[(long long)r * ld + c] = acc[i][j];
    }
}

// X += T for every entry (flat over n*ld elements of each entry)
template <typename ST, typename AT>
__global__ void k_ns_add(const int* __restrict__ lst, const long long* __restrict__ elpre, int nent,
                         const int* __restrict__ bn, const int* __restrict__ bld, const long long* __restrict__ moff,
                         ST* __restrict__ mat, const long long* __restrict__ soff, const AT* __restrict__ T) {
  long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (w >= elpre[nent]) return;
  int e = find_block(elpre, nent, w);
  int b = lst[e];
  long long loc = w - elpre[e];
  int ld = bld[b];
  int r = (int)(loc / ld), c = (int)(loc % ld);
  if (r >= bn[b] || c >= bn[b]) return;
  ST* x = mat + moff[b] + loc;
  *x = (ST)((AT)*x + T[soff[e] + loc]);
}

// closure-block residual for the basis solves: res = rhs - Abar * S (FP64, n x kc per block)
__global__ void k_closure_residual(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                                   const int* __restrict__ owner, int nblk, const long long* __restrict__ ioff,
                                   const int* __restrict__ bn, const int* __restrict__ idx, long long n_total,
                                   const long long* __restrict__ roff, const int* __restrict__ kcv,
                                   const double* __restrict__ rhs, const double* __restrict__ S,
                                   double* __restrict__ res) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int b = find_block(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  int n = bn[b];
  if (r >= n) return;
  const int* bidx = idx + ioff[b];
  int g = bidx[r];
  int kc = kcv[b];
  RowList L;
  L.n = 0;
  any_row<double>(G, P, fl, op, st, g, L);
  int me = owner[g];
  const double* Sb = S + roff[b];
  double* out = res + roff[b] + (long long)r * kc;
  const double* in = rhs + roff[b] + (long long)r * kc;
  for (int q = 0; q < kc; ++q) out[q] = in[q];
  double extra = 0.0;
  for (int k = 0; k < L.n; ++k) {
    int lc = lower_idx(bidx, n, L.col[k]);
    if (lc < n && bidx[lc] == L.col[k]) {
      for (int q = 0; q < kc; ++q) out[q] -= L.val[k] * Sb[(long long)lc * kc + q];
    } else {
      int o = owner[L.col[k]];
      if (o == -3 || (o >= 0 && o != me)) extra += L.val[k];
    }
  }
  if (extra != 0.0)
    for (int q = 0; q < kc; ++q) out[q] -= extra * Sb[(long long)r * kc + q];
}

__global__ void k_add_vec(double* __restrict__ a, const double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] += b[i];
}

// ------------------------------------------------------------------------------ Woodbury closure
// The closure block Abar = A_p + E_K diag(delta) E_K^T differs from the primary block A_p only on the
// diagonal entries K of rows coupled to interface faces or other primary grids (Eqs. 6, 9), so
// Abar^{-1} R = X R - X_{:,K} (diag(delta)^{-1} + X_KK)^{-1} (X R)_K with X = A_p^{-1} already built.

// extra[t] = sum of A_b couplings of primary row t to f faces and other primary grids
__global__ void k_closure_extras(Geo G, Phy P, const uint8_t* __restrict__ fl, int op, const double* __restrict__ st,
                                 const int* __restrict__ owner, int nblk, const long long* __restrict__ ioff,
                                 const int* __restrict__ bn, const int* __restrict__ idx, long long n_total,
                                 double* __restrict__ extra) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_total) return;
  int b = find_block(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  if (r >= bn[b]) { extra[t] = 0.0; return; }
  int g = idx[t];
  RowList L;
  L.n = 0;
  any_row<double>(G, P, fl, op, st, g, L);
  int me = owner[g];
  double e = 0.0;
  for (int k = 0; k < L.n; ++k) {
    int o = owner[L.col[k]];
    if (o == -3 || (o >= 0 && o != me)) e += L.val[k];
  }
  extra[t] = e;
}

// Cap_b[i][j] = X_b[K_i][K_j] + (i == j) / delta_i, the Woodbury capacitance matrix of block b (k x k, row
// stride cld[b], in the storage precision of X); one thread per entry over the prefix epre of k^2
template <typename ST>
__global__ void k_cap_assemble(const long long* __restrict__ epre, int nb, const int* __restrict__ kv,
                               const long long* __restrict__ koff, const long long* __restrict__ cmoff,
                               const int* __restrict__ cld, const int* __restrict__ Klist,
                               const double* __restrict__ delta, const int* __restrict__ bld,
                               const long long* __restrict__ moff, const ST* __restrict__ X, ST* __restrict__ cap) {
  long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (w >= epre[nb]) return;
  int b = find_block(epre, nb, w);
  long long loc = w - epre[b];
  int k = kv[b];
  int i = (int)(loc / k), j = (int)(loc % k);
  const int* K = Klist + koff[b];
  double v = (double)X[moff[b] + (long long)K[i] * bld[b] + K[j]];
  if (i == j) v += 1.0 / delta[koff[b] + i];
  cap[cmoff[b] + (long long)i * cld[b] + j] = (ST)v;
}

// W[b] (k x kc) = Y[b][K, :]
__global__ void k_gather_rows(int nb, const long long* __restrict__ rpre, const int* __restrict__ kv,
                              const long long* __restrict__ koff, const int* __restrict__ Klist,
                              const long long* __restrict__ roff, const long long* __restrict__ woff,
                              const int* __restrict__ kcv, const double* __restrict__ Y, double* __restrict__ W) {
  long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (w >= rpre[nb]) return;
  int b = find_block(rpre, nb, w);
  int m = (int)(w - rpre[b]);
  int kc = kcv[b];
  int r = Klist[koff[b] + m];
  for (int q = 0; q < kc; ++q) W[woff[b] + (long long)m * kc + q] = Y[roff[b] + (long long)r * kc + q];
}

// Z[b] (k x kc) = Cinv[b] (k x k) * W[b]   (warp per row; FP64 accumulation)
template <typename ST>
__global__ void k_cap_mm(int nb, const long long* __restrict__ rpre, const int* __restrict__ kv,
                         const long long* __restrict__ cmoff, const int* __restrict__ cld, const ST* __restrict__ Cinv,
                         const long long* __restrict__ woff, const int* __restrict__ kcv, const double* __restrict__ W,
                         double* __restrict__ Z) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= rpre[nb]) return;
  int b = find_block(rpre, nb, w);
  int m = (int)(w - rpre[b]);
  int k = kv[b], kc = kcv[b];
  const ST* C = Cinv + cmoff[b] + (long long)m * cld[b];
  for (int q0 = 0; q0 < kc; q0 += 16) {
    int qn = min(16, kc - q0);
    double acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int j = lane; j < k; j += 32) {
      double c = (double)C[j];
      const double* wr = W + woff[b] + (long long)j * kc + q0;
      for (int q = 0; q < qn; ++q) acc[q] += c * wr[q];
    }
    for (int q = 0; q < qn; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) Z[woff[b] + (long long)m * kc + q0 + q] = v;
    }
  }
}

// S[b][r][:] = Y[b][r][:] - sum_m X_b[r][K_m] Z[b][m][:]   (warp per row of every primary block)
template <typename ST>
__global__ void k_woodbury_update(int nblk, const long long* __restrict__ ioff, const int* __restrict__ bn,
                                  const int* __restrict__ bld, const long long* __restrict__ moff,
                                  const ST* __restrict__ X, long long n_total, const int* __restrict__ kv,
                                  const long long* __restrict__ koff, const int* __restrict__ Klist,
                                  const long long* __restrict__ roff, const long long* __restrict__ woff,
                                  const int* __restrict__ kcv, const double* __restrict__ Y,
                                  const double* __restrict__ Z, double* __restrict__ S) {
  long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= n_total) return;
  int b = find_block(ioff, nblk, t);
  int r = (int)(t - ioff[b]);
  if (r >= bn[b]) return;
  int k = kv[b], kc = kcv[b];
  const ST* xr = X + moff[b] + (long long)r * bld[b];
  const int* K = Klist + koff[b];
  for (int q0 = 0; q0 < kc; q0 += 16) {
    int qn = min(16, kc - q0);
    double acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int m = lane; m < k; m += 32) {
      double xv = (double)xr[K[m]];
      const double* zr = Z + woff[b] + (long long)m * kc + q0;
      for (int q = 0; q < qn; ++q) acc[q] += xv * zr[q];
    }
    for (int q = 0; q < qn; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) {
        long long at = roff[b] + (long long)r * kc + q0 + q;
        S[at] = Y[at] - v;
      }
    }
  }
}

}  // namespace

// ================================================================================ launchers
// Temporary device buffers of one host-side step; every allocation is checked, and everything is freed
// when the object goes out of scope.
struct TmpDev {
  std::vector<void*> ptrs;
  TmpDev() = default;
  TmpDev(const TmpDev&) = delete;
  TmpDev& operator=(const TmpDev&) = delete;
  ~TmpDev() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T** out, size_t bytes) {
    *out = nullptr;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) return e;
    ptrs.push_back(p);
    *out = (T*)p;
    return cudaSuccess;
  }
};

template <typename ST>
cudaError_t launch_assemble(const Ctx& C, const BlockSet& B, int op, const double* state, ST* mat, int closure) {
  if (B.nblk == 0) return cudaSuccess;
  int thr = 128;
  long long blk = (B.n_total + thr - 1) / thr;
  { pns::count_launch(); k_assemble<ST><<<(unsigned)blk, thr, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state, C.owner.as<int>(),
                                                      B.nblk, B.d_ioff.as<long long>(), B.d_n.as<int>(),
                                                      B.d_ld.as<int>(), B.d_moff.as<long long>(), B.idx.as<int>(),
                                                      B.n_total, mat, closure); }
  return cudaGetLastError();
}
template cudaError_t launch_assemble<double>(const Ctx&, const BlockSet&, int, const double*, double*, int);
template cudaError_t launch_assemble<float>(const Ctx&, const BlockSet&, int, const double*, float*, int);

template <typename ST> struct GjPanel;
template <> struct GjPanel<double> { static constexpr int tb = 64; };
template <> struct GjPanel<float> { static constexpr int tb = MT; };

template <typename ST>
cudaError_t launch_gj_invert(const BlockSet& B, ST* mat, int* d_bad, cudaStream_t s, GjTimer* timer, int tensor_cores) {
  if (B.nblk == 0) return cudaSuccess;
  constexpr int TBK = GjPanel<ST>::tb;
  std::vector<cudaEvent_t> evs;
  double flops = 0, bytes = 0;
  long long tiles = 0;
  // order blocks by tile count (descending): the active set at step k is a prefix
  std::vector<int> order(B.nblk);
  for (int i = 0; i < B.nblk; ++i) order[i] = i;
  std::vector<int> T(B.nblk);
  for (int i = 0; i < B.nblk; ++i) T[i] = (B.n[i] + TBK - 1) / TBK;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return T[a] > T[b]; });
  std::vector<long long> pre1(B.nblk + 1, 0), pre2(B.nblk + 1, 0);
  for (int s2 = 0; s2 < B.nblk; ++s2) {
    long long t = T[order[s2]] - 1;
    pre1[s2 + 1] = pre1[s2] + t;
    pre2[s2 + 1] = pre2[s2] + t * t;
  }
  int *d_order = nullptr;
  long long *d_pre1 = nullptr, *d_pre2 = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&d_order, sizeof(int) * B.nblk)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&d_pre1, sizeof(long long) * (B.nblk + 1))) != cudaSuccess) { cudaFree(d_order); return e; }
  if ((e = cudaMalloc(&d_pre2, sizeof(long long) * (B.nblk + 1))) != cudaSuccess) {
    cudaFree(d_order); cudaFree(d_pre1); return e;
  }
  cudaMemcpyAsync(d_order, order.data(), sizeof(int) * B.nblk, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_pre1, pre1.data(), sizeof(long long) * (B.nblk + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_pre2, pre2.data(), sizeof(long long) * (B.nblk + 1), cudaMemcpyHostToDevice, s);
  const size_t smem = 2 * sizeof(ST) * TBK * (TBK + 1);
  const size_t smem_mm = sizeof(MmSmem);
  cudaFuncSetAttribute(k_gj_rowpanel<ST, TBK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_gj_colpanel<ST, TBK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (std::is_same<ST, float>::value) {
    cudaFuncSetAttribute(k_mm128_gj_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_mm);
    cudaFuncSetAttribute(k_mm128_gj_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_mm);
  }
  else
    cudaFuncSetAttribute(k_gj_update<ST, TBK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // tensor_cores 2 / 3: the update on the 5th-generation tensor cores (FP32 inverses only), persistent /
  // one CTA per tile
  GjTc tc5;
  const bool use_tc5 = std::is_same<ST, float>::value && tensor_cores >= 2;
  if (use_tc5) {
    if ((e = tc5.setup(B, (float*)mat, s, tensor_cores == 2)) != cudaSuccess) {
      cudaFree(d_order); cudaFree(d_pre1); cudaFree(d_pre2);
      return e;
    }
  }
  int Tmax = T[order[0]];
  int cnt = B.nblk;
  for (int k = 0; k < Tmax; ++k) {
    while (cnt > 0 && T[order[cnt - 1]] <= k) --cnt;
    { pns::count_launch(); k_gj_diag<ST, TBK><<<cnt, 256, 0, s>>>(k, d_order, B.d_n.as<int>(), B.d_ld.as<int>(),
                                                                         B.d_moff.as<long long>(), mat, d_bad); }
    if (pre1[cnt] > 0) {
      { pns::count_launch(); k_gj_rowpanel<ST, TBK><<<(unsigned)pre1[cnt], 256, smem, s>>>(k, cnt, d_order, d_pre1, B.d_n.as<int>(),
                                                               B.d_ld.as<int>(), B.d_moff.as<long long>(), mat); }
      if (pre2[cnt] > 0) {
        if constexpr (std::is_same<ST, float>::value) {
          if (timer) {
            cudaEvent_t a, b2;
            if ((e = cudaEventCreate(&a)) != cudaSuccess) break;
            if ((e = cudaEventCreate(&b2)) != cudaSuccess) { cudaEventDestroy(a); break; }
            evs.push_back(a);
            evs.push_back(b2);
            cudaEventRecord(a, s);
            for (int q = 0; q < cnt; ++q) {
              const int n = B.n[order[q]];
              const int nb = std::min(TBK, n - k * TBK);
              flops += 2.0 * (double)(n - nb) * (double)(n - nb) * (double)nb;
              bytes += 8.0 * (double)(n - nb) * (double)(n - nb) + 8.0 * (double)(n - nb) * (double)nb;
            }
            tiles += pre2[cnt];
          }
          if (use_tc5) {
            if ((e = tc5.step(B, (float*)mat, k, cnt, d_order, d_pre2, pre2[cnt], order, d_bad, s)) != cudaSuccess)
              break;
          } else if (tensor_cores) {
            pns::count_launch();
            k_mm128_gj_update_tc<<<(unsigned)pre2[cnt], 256, smem_mm, s>>>(k, cnt, d_order, d_pre2, B.d_n.as<int>(),
                                                                           B.d_ld.as<int>(), B.d_moff.as<long long>(),
                                                                           mat);
          } else {
            pns::count_launch();
            k_mm128_gj_update<<<(unsigned)pre2[cnt], 256, smem_mm, s>>>(k, cnt, d_order, d_pre2, B.d_n.as<int>(),
                                                                        B.d_ld.as<int>(), B.d_moff.as<long long>(), mat);
          }
          if (timer) cudaEventRecord(evs.back(), s);
        } else {
          pns::count_launch();
          k_gj_update<ST, TBK><<<(unsigned)pre2[cnt], 256, smem, s>>>(k, cnt, d_order, d_pre2, B.d_n.as<int>(),
                                                                      B.d_ld.as<int>(), B.d_moff.as<long long>(), mat);
        }
      }
      { pns::count_launch(); k_gj_colpanel<ST, TBK><<<(unsigned)pre1[cnt], 256, smem, s>>>(k, cnt, d_order, d_pre1, B.d_n.as<int>(),
                                                               B.d_ld.as<int>(), B.d_moff.as<long long>(), mat); }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
  }
  cudaStreamSynchronize(s);
  if (timer) {
    for (size_t q = 0; q + 1 < evs.size(); q += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, evs[q], evs[q + 1]) == cudaSuccess) timer->ms += ms;
    }
    timer->flops += flops;
    timer->bytes += bytes;
    timer->tiles += tiles;
    timer->launches += (long long)(evs.size() / 2);
  }
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  cudaFree(d_order);
  cudaFree(d_pre1);
  cudaFree(d_pre2);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template cudaError_t launch_gj_invert<double>(const BlockSet&, double*, int*, cudaStream_t, GjTimer*, int);
template cudaError_t launch_gj_invert<float>(const BlockSet&, float*, int*, cudaStream_t, GjTimer*, int);

cudaError_t launch_closure_rhs(const Ctx& C, const BlockSet& B, int op, const double* state, const int* d_colbase,
                               const int* d_cols, const long long* d_roff, const int* d_kc, double* rhs) {
  if (B.nblk == 0) return cudaSuccess;
  int thr = 128;
  long long blk = (B.n_total + thr - 1) / thr;
  { pns::count_launch(); k_closure_rhs<<<(unsigned)blk, thr, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state,
                                                     C.cell_iface.as<int>(), B.nblk, B.d_ioff.as<long long>(),
                                                     B.d_n.as<int>(), B.idx.as<int>(), B.n_total, d_colbase, d_cols,
                                                     d_roff, d_kc, rhs); }
  return cudaGetLastError();
}

template <typename ST, typename AT>
cudaError_t launch_block_mm(const BlockSet& B, const ST* mat, const double* rhs, const long long* d_roff,
                            const int* d_kc, const std::vector<int>& kc, double* out, cudaStream_t s) {
  static_assert(std::is_same<ST, AT>::value, "the closure product accumulates in the storage precision");
  if (B.nblk == 0) return cudaSuccess;
  // three column widths of R: kc <= 8 (64 rows per CTA), <= 16 (32 rows), else chunks of 32 (16 rows)
  std::vector<int4> items[3];
  const int kq[3] = {8, 16, 32}, rows[3] = {64, 32, 16};
  for (int b = 0; b < B.nblk; ++b) {
    const int bin = kc[b] <= 8 ? 0 : kc[b] <= 16 ? 1 : 2;
    for (int q0 = 0; q0 < kc[b]; q0 += kq[bin])
      for (int r0 = 0; r0 < B.n[b]; r0 += rows[bin]) items[bin].push_back(make_int4(b, r0, q0, 0));
  }
  TmpDev tmp;
  cudaError_t e = cudaSuccess;
  for (int bin = 0; bin < 3; ++bin) {
    if (items[bin].empty()) continue;
    int4* d_items = nullptr;
    if ((e = tmp.get(&d_items, sizeof(int4) * items[bin].size())) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_items, items[bin].data(), sizeof(int4) * items[bin].size(), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
      return e;
    const unsigned grid = (unsigned)items[bin].size();
    pns::count_launch();
    if (bin == 0)
      k_block_mm_s<ST, 8, 8><<<grid, 256, 0, s>>>(d_items, B.d_n.as<int>(), B.d_ld.as<int>(), B.d_moff.as<long long>(),
                                                  mat, rhs, d_roff, d_kc, out);
    else if (bin == 1)
      k_block_mm_s<ST, 16, 4><<<grid, 256, 0, s>>>(d_items, B.d_n.as<int>(), B.d_ld.as<int>(),
                                                   B.d_moff.as<long long>(), mat, rhs, d_roff, d_kc, out);
    else
      k_block_mm_s<ST, 32, 2><<<grid, 256, 0, s>>>(d_items, B.d_n.as<int>(), B.d_ld.as<int>(),
                                                   B.d_moff.as<long long>(), mat, rhs, d_roff, d_kc, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(s);   // the item lists are freed on return
}
template cudaError_t launch_block_mm<double, double>(const BlockSet&, const double*, const double*, const long long*,
                                                     const int*, const std::vector<int>&, double*, cudaStream_t);
template cudaError_t launch_block_mm<float, float>(const BlockSet&, const float*, const double*, const long long*,
                                                   const int*, const std::vector<int>&, double*, cudaStream_t);

// One persistent launch of the binned local GEMV over a block set (items and counter built by
// build_gemv_items): a grid of a few CTAs per SM that drain the item list.
template <typename ST, typename PT>
cudaError_t launch_local_gemv_p(const BlockSet& B, const ST* mat, const PT* pk, double* z, int mode, cudaStream_t s) {
  if (B.nitems_p == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(B.counter.p, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_local_gemv_p<float, float>, 256, 0);
    grid = sms * std::max(1, per);
  }
  pns::count_launch();
  k_local_gemv_p<ST, PT><<<(unsigned)std::min(grid, B.nitems_p), 256, 0, s>>>(
      B.items_p.as<int4>(), B.nitems_p, B.counter.as<int>(), B.idx.as<int>(), B.d_ioff.as<long long>(),
      B.d_ld.as<int>(), B.d_moff.as<long long>(), mat, pk, z, mode);
  return cudaGetLastError();
}
template cudaError_t launch_local_gemv_p<double, double>(const BlockSet&, const double*, const double*, double*, int,
                                                         cudaStream_t);
template cudaError_t launch_local_gemv_p<float, float>(const BlockSet&, const float*, const float*, double*, int,
                                                       cudaStream_t);
template cudaError_t launch_local_gemv_p<__nv_bfloat16, float>(const BlockSet&, const __nv_bfloat16*, const float*,
                                                               double*, int, cudaStream_t);

template <typename ST, typename PT>
cudaError_t launch_local_solve(const BlockSet& B, const ST* mat, const double* t, double* z, PT* pk_x, int add,
                               cudaStream_t s) {
  if (B.nblk == 0) return cudaSuccess;
  int thr = 256;
  long long blk = (B.n_total + thr - 1) / thr;
  { pns::count_launch(); k_gather<PT><<<(unsigned)blk, thr, 0, s>>>(B.idx.as<int>(), B.n_total, t, pk_x); }
  cudaError_t e = launch_local_gemv_p<ST, PT>(B, mat, pk_x, z, add ? 1 : 0, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Local solve with one step of iterative refinement against the block's own matrix A_b[idx, idx]:
// zp = X t, zp += X (t - A zp) (residual in FP64 from the stencil), then z[idx] (+)= zp.  With an
// inverse accurate to eps this leaves an error of order eps^2, at the cost of a second pass over X.
template <typename ST, typename PT>
cudaError_t launch_local_solve_refined(const Ctx& C, const BlockSet& B, int op, const double* state, const ST* mat,
                                       const double* t, double* z, PT* pk_x, double* zp, int add, cudaStream_t s) {
  if (B.nblk == 0) return cudaSuccess;
  int thr = 256;
  unsigned blk = (unsigned)((B.n_total + thr - 1) / thr);
  { pns::count_launch(); k_gather<PT><<<blk, thr, 0, s>>>(B.idx.as<int>(), B.n_total, t, pk_x); }
  cudaError_t e = launch_local_gemv_p<ST, PT>(B, mat, pk_x, zp, 2, s);
  if (e != cudaSuccess) return e;
  { pns::count_launch(); k_local_residual<PT><<<blk, thr, 0, s>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state, B.nblk,
                                                B.d_ioff.as<long long>(), B.d_n.as<int>(), B.idx.as<int>(), B.n_total,
                                                t, zp, pk_x); }
  e = launch_local_gemv_p<ST, PT>(B, mat, pk_x, zp, 3, s);
  if (e != cudaSuccess) return e;
  { pns::count_launch(); k_scatter_packed<<<blk, thr, 0, s>>>(B.idx.as<int>(), B.n_total, zp, z, add); }
  return cudaGetLastError();
}
template cudaError_t launch_local_solve_refined<float, float>(const Ctx&, const BlockSet&, int, const double*,
                                                              const float*, const double*, double*, float*, double*,
                                                              int, cudaStream_t);
template cudaError_t launch_local_solve_refined<__nv_bfloat16, float>(const Ctx&, const BlockSet&, int, const double*,
                                                                      const __nv_bfloat16*, const double*, double*,
                                                                      float*, double*, int, cudaStream_t);
template cudaError_t launch_local_solve<double, double>(const BlockSet&, const double*, const double*, double*,
                                                        double*, int, cudaStream_t);
template cudaError_t launch_local_solve<float, float>(const BlockSet&, const float*, const double*, double*, float*,
                                                      int, cudaStream_t);
template cudaError_t launch_local_solve<__nv_bfloat16, float>(const BlockSet&, const __nv_bfloat16*, const double*,
                                                              double*, float*, int, cudaStream_t);

// Refine the inverses of a block set: blocks whose max |I - A X| exceeds `thresh` get `steps`
// Newton-Schulz steps.  Scratch is bounded by `budget_bytes` (blocks processed in chunks).
template <typename ST, typename AT>
cudaError_t launch_ns_refine(const Ctx& C, const BlockSet& B, int op, const double* state, int closure, ST* mat,
                             int steps, double thresh, size_t budget_bytes, double* max_before, double* max_after) {
  if (B.nblk == 0 || steps <= 0) return cudaSuccess;
  cudaStream_t s = C.stream;
  cudaError_t e = cudaSuccess;
  *max_before = 0;
  if (max_after) *max_after = 0;
  constexpr bool f32 = std::is_same<ST, float>::value && std::is_same<AT, float>::value;
  constexpr int NT = f32 ? MT : TB;   // tile edge of the product T = X R
  size_t smem = f32 ? sizeof(MmSmem) : 2 * sizeof(AT) * TB * (TB + 1);
  if (f32) cudaFuncSetAttribute(k_mm128_ns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else cudaFuncSetAttribute(k_ns_gemm<ST, AT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // chunks of consecutive blocks whose R and T fit the budget
  int b0 = 0;
  while (b0 < B.nblk && e == cudaSuccess) {
    std::vector<int> lst;
    std::vector<long long> soff(1, 0);
    size_t used = 0;
    int b = b0;
    while (b < B.nblk) {
      size_t need = 2 * sizeof(AT) * (size_t)B.ld[b] * B.ld[b];
      if (!lst.empty() && used + need > budget_bytes) break;
      lst.push_back(b);
      used += need;
      soff.push_back(soff.back() + (long long)B.ld[b] * B.ld[b]);
      ++b;
    }
    b0 = b;
    int nent = (int)lst.size();
    std::vector<double> prev(nent, 1e300);
    for (int step = 0; step < steps && e == cudaSuccess; ++step) {
      std::vector<long long> rowpre(nent + 1, 0);
      for (int q = 0; q < nent; ++q) rowpre[q + 1] = rowpre[q] + B.n[lst[q]];
      int *d_lst = nullptr;
      long long *d_pre = nullptr, *d_soff = nullptr;
      unsigned int* d_rmax = nullptr;
      AT *R = nullptr, *T = nullptr;
      TmpDev tmp;
      if ((e = tmp.get(&d_lst, sizeof(int) * nent)) != cudaSuccess) break;
      if ((e = tmp.get(&d_pre, sizeof(long long) * (nent + 1))) != cudaSuccess) break;
      if ((e = tmp.get(&d_soff, sizeof(long long) * (nent + 1))) != cudaSuccess) break;
      if ((e = tmp.get(&d_rmax, sizeof(unsigned int) * nent)) != cudaSuccess) break;
      if ((e = tmp.get(&R, sizeof(AT) * soff[nent])) != cudaSuccess) break;
      if ((e = tmp.get(&T, sizeof(AT) * soff[nent])) != cudaSuccess) break;
      cudaMemsetAsync(T, 0, sizeof(AT) * soff[nent], s);
      cudaMemcpyAsync(d_lst, lst.data(), sizeof(int) * nent, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(d_pre, rowpre.data(), sizeof(long long) * (nent + 1), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(d_soff, soff.data(), sizeof(long long) * (nent + 1), cudaMemcpyHostToDevice, s);
      cudaMemsetAsync(d_rmax, 0, sizeof(unsigned int) * nent, s);
      cudaMemsetAsync(R, 0, sizeof(AT) * soff[nent], s);
      { pns::count_launch(); k_ns_residual<ST, AT><<<(unsigned)rowpre[nent], 256, 0, s>>>(
          C.G, C.P, C.flags.as<uint8_t>(), op, state, C.owner.as<int>(), closure, d_lst, d_pre, nent,
          B.d_ioff.as<long long>(), B.d_n.as<int>(), B.d_ld.as<int>(), B.d_moff.as<long long>(), B.idx.as<int>(), mat,
          d_soff, R, d_rmax); }
      std::vector<unsigned int> rm(nent);
      cudaMemcpyAsync(rm.data(), d_rmax, sizeof(unsigned int) * nent, cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      // refine only the blocks above the threshold
      std::vector<int> sel;
      std::vector<long long> ssoff;
      for (int q = 0; q < nent; ++q) {
        float v;
        memcpy(&v, &rm[q], sizeof v);
        if (step == 0) *max_before = std::max(*max_before, (double)v);
        // refine while the residual is above the floor and still falls fast (quadratic phase);
        // once it stalls it sits at the storage-rounding floor cond * eps and further steps are moot
        bool go = v > thresh && (step == 0 || v < 0.25 * prev[q]);
        prev[q] = v;
        if (go) { sel.push_back(lst[q]); ssoff.push_back(soff[q]); }
      }
      if (e == cudaSuccess && !sel.empty()) {
        int ns = (int)sel.size();
        std::vector<long long> tpre(ns + 1, 0), epre(ns + 1, 0);
        for (int q = 0; q < ns; ++q) {
          long long Tt = (B.n[sel[q]] + NT - 1) / NT;
          tpre[q + 1] = tpre[q] + Tt * Tt;
          epre[q + 1] = epre[q] + (long long)B.ld[sel[q]] * B.ld[sel[q]];
        }
        ssoff.push_back(0);
        int* d_sel = nullptr;
        long long *d_tpre = nullptr, *d_epre = nullptr, *d_ssoff = nullptr;
        TmpDev tsel;
        if ((e = tsel.get(&d_sel, sizeof(int) * ns)) != cudaSuccess) break;
        if ((e = tsel.get(&d_tpre, sizeof(long long) * (ns + 1))) != cudaSuccess) break;
        if ((e = tsel.get(&d_epre, sizeof(long long) * (ns + 1))) != cudaSuccess) break;
        if ((e = tsel.get(&d_ssoff, sizeof(long long) * (ns + 1))) != cudaSuccess) break;
        cudaMemcpyAsync(d_sel, sel.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_tpre, tpre.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_epre, epre.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_ssoff, ssoff.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, s);
        if constexpr (f32) {
          pns::count_launch();
          k_mm128_ns<<<(unsigned)tpre[ns], 256, smem, s>>>(d_sel, d_tpre, ns, B.d_n.as<int>(), B.d_ld.as<int>(),
                                                           B.d_moff.as<long long>(), mat, d_ssoff, R, T);
        } else {
          pns::count_launch();
          k_ns_gemm<ST, AT, AT><<<(unsigned)tpre[ns], 256, smem, s>>>(d_sel, d_tpre, ns, B.d_n.as<int>(),
                                                                     B.d_ld.as<int>(), B.d_moff.as<long long>(), mat,
                                                                     d_ssoff, R, T);
        }
        { pns::count_launch(); k_ns_add<ST, AT><<<(unsigned)((epre[ns] + 255) / 256), 256, 0, s>>>(
            d_sel, d_epre, ns, B.d_n.as<int>(), B.d_ld.as<int>(), B.d_moff.as<long long>(), mat, d_ssoff, T); }
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
      }
      if (sel.empty()) break;
    }
  }
  // final residual of every block (report, only when asked for)
  if (e == cudaSuccess && max_after) {
    int nent = B.nblk;
    std::vector<int> lst(nent);
    std::vector<long long> rowpre(nent + 1, 0), soff(nent + 1, 0);
    size_t maxm = 0;
    for (int q = 0; q < nent; ++q) {
      lst[q] = q;
      rowpre[q + 1] = rowpre[q] + B.n[q];
      maxm = std::max(maxm, (size_t)B.ld[q] * B.ld[q]);
    }
    // one block at a time through a single scratch slot, residual max only
    AT* R = nullptr;
    int* d_lst = nullptr;
    long long *d_pre = nullptr, *d_soff = nullptr;
    unsigned int* d_rmax = nullptr;
    TmpDev tmp;
    if ((e = tmp.get(&R, sizeof(AT) * maxm)) == cudaSuccess && (e = tmp.get(&d_lst, sizeof(int))) == cudaSuccess &&
        (e = tmp.get(&d_pre, sizeof(long long) * 2)) == cudaSuccess &&
        (e = tmp.get(&d_soff, sizeof(long long) * 2)) == cudaSuccess &&
        (e = tmp.get(&d_rmax, sizeof(unsigned int))) == cudaSuccess) {
      long long zero2[2] = {0, 0};
      cudaMemcpyAsync(d_soff, zero2, sizeof zero2, cudaMemcpyHostToDevice, s);
      for (int q = 0; q < nent && e == cudaSuccess; ++q) {
        long long pre[2] = {0, B.n[q]};
        cudaMemcpyAsync(d_lst, &q, sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_pre, pre, sizeof pre, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_rmax, 0, sizeof(unsigned int), s);
        { pns::count_launch(); k_ns_residual<ST, AT><<<(unsigned)B.n[q], 256, 0, s>>>(
            C.G, C.P, C.flags.as<uint8_t>(), op, state, C.owner.as<int>(), closure, d_lst, d_pre, 1,
            B.d_ioff.as<long long>(), B.d_n.as<int>(), B.d_ld.as<int>(), B.d_moff.as<long long>(), B.idx.as<int>(),
            mat, d_soff, R, d_rmax); }
        unsigned int rmv = 0;
        cudaMemcpyAsync(&rmv, d_rmax, sizeof rmv, cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        float v;
        memcpy(&v, &rmv, sizeof v);
        *max_after = std::max(*max_after, (double)v);
      }
    }
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template cudaError_t launch_ns_refine<float, float>(const Ctx&, const BlockSet&, int, const double*, int, float*, int,
                                                   double, size_t, double*, double*);
template cudaError_t launch_ns_refine<double, double>(const Ctx&, const BlockSet&, int, const double*, int, double*,
                                                     int, double, size_t, double*, double*);

cudaError_t launch_closure_residual(const Ctx& C, const BlockSet& B, int op, const double* state,
                                    const long long* d_roff, const int* d_kc, const double* rhs, const double* S,
                                    double* res) {
  if (B.nblk == 0) return cudaSuccess;
  long long blk = (B.n_total + 127) / 128;
  { pns::count_launch(); k_closure_residual<<<(unsigned)blk, 128, 0, C.stream>>>(C.G, C.P, C.flags.as<uint8_t>(), op, state,
                                                         C.owner.as<int>(), B.nblk, B.d_ioff.as<long long>(),
                                                         B.d_n.as<int>(), B.idx.as<int>(), B.n_total, d_roff, d_kc,
                                                         rhs, S, res); }
  return cudaGetLastError();
}

cudaError_t launch_add_vec(double* a, const double* b, long long n, cudaStream_t s) {
  { pns::count_launch(); k_add_vec<<<2048, 256, 0, s>>>(a, b, n); }
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------- Woodbury driver
// Woodbury data of one closure build: per primary block b the rows K_b whose diagonal the closure
// modifies (k_b of them, with their extra delta), and the inverses of the capacitance matrices, kept as a
// block set of the blocks with k_b > 0 so that the Gauss-Jordan inverse of the local blocks inverts them
// (cmoff / cld: each original block's offset and row stride in that set's storage, 0 when k_b = 0).
struct WoodburyImpl {
  int nblk = 0;
  std::vector<int> k;
  DevBuf d_k, d_koff, d_cmoff, d_cld, d_Klist, d_delta, d_rpre, d_woff;
  std::vector<long long> koff, cmoff, rpre, woff;
  BlockSet cb;
};

Woodbury::Woodbury() : impl(new WoodburyImpl) {}
Woodbury::~Woodbury() { delete impl; }

static cudaError_t upload_ll(DevBuf& b, const std::vector<long long>& v, cudaStream_t s) {
  b.release();
  cudaError_t e = cudaMalloc(&b.p, sizeof(long long) * std::max<size_t>(1, v.size()));
  if (e != cudaSuccess) return e;
  b.bytes = sizeof(long long) * std::max<size_t>(1, v.size());
  return cudaMemcpyAsync(b.p, v.data(), sizeof(long long) * v.size(), cudaMemcpyHostToDevice, s);
}
static cudaError_t upload_i(DevBuf& b, const std::vector<int>& v, cudaStream_t s) {
  b.release();
  cudaError_t e = cudaMalloc(&b.p, sizeof(int) * std::max<size_t>(1, v.size()));
  if (e != cudaSuccess) return e;
  b.bytes = sizeof(int) * std::max<size_t>(1, v.size());
  return cudaMemcpyAsync(b.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s);
}

template <typename ST>
cudaError_t Woodbury::setup(const Ctx& C, const BlockSet& B, int op, const double* state, const ST* X,
                            const std::vector<int>& kc, int* d_bad) {
  cudaStream_t s = C.stream;
  WoodburyImpl& W = *impl;
  W.nblk = B.nblk;
  cudaError_t e;
  // closure extras per primary row -> K lists
  double* d_extra = nullptr;
  if ((e = cudaMalloc(&d_extra, sizeof(double) * std::max(1LL, B.n_total))) != cudaSuccess) return e;
  cudaMemsetAsync(d_extra, 0, sizeof(double) * std::max(1LL, B.n_total), s);
  { pns::count_launch(); k_closure_extras<<<(unsigned)((B.n_total + 127) / 128), 128, 0, s>>>(
      C.G, C.P, C.flags.as<uint8_t>(), op, state, C.owner.as<int>(), B.nblk, B.d_ioff.as<long long>(),
      B.d_n.as<int>(), B.idx.as<int>(), B.n_total, d_extra); }
  std::vector<double> ex(B.n_total);
  cudaMemcpyAsync(ex.data(), d_extra, sizeof(double) * B.n_total, cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  cudaFree(d_extra);
  if (e != cudaSuccess) return e;
  W.k.assign(B.nblk, 0);
  W.koff.assign(B.nblk + 1, 0);
  W.cmoff.assign(B.nblk + 1, 0);
  W.rpre.assign(B.nblk + 1, 0);
  W.woff.assign(B.nblk + 1, 0);
  std::vector<int> Kl, cld(B.nblk, 0);
  std::vector<double> dl;
  std::vector<long long> epre(B.nblk + 1, 0);
  BlockSet& cb = W.cb;   // a Woodbury object is set up once
  for (int b = 0; b < B.nblk; ++b) {
    for (int r = 0; r < B.n[b]; ++r) {
      double v = ex[B.ioff[b] + r];
      if (v != 0.0) { Kl.push_back(r); dl.push_back(v); }
    }
    const int kb = (int)(Kl.size() - W.koff[b]);
    W.k[b] = kb;
    W.koff[b + 1] = (long long)Kl.size();
    W.rpre[b + 1] = W.rpre[b] + kb;
    W.woff[b + 1] = W.woff[b] + (long long)kb * kc[b];
    epre[b + 1] = epre[b] + (long long)kb * kb;
    W.cmoff[b] = cb.m_total;
    if (kb > 0) {
      const int ld = (kb + 7) / 8 * 8;
      cld[b] = ld;
      cb.n.push_back(kb);
      cb.ld.push_back(ld);
      cb.ioff.push_back(cb.n_total);
      cb.moff.push_back(cb.m_total);
      cb.n_total += ld;
      cb.m_total += (long long)ld * ld;
      cb.sum_n2 += (double)kb * kb;
      cb.nmax = std::max(cb.nmax, kb);
    }
  }
  W.cmoff[B.nblk] = cb.m_total;
  cb.nblk = (int)cb.n.size();
  cb.ioff.push_back(cb.n_total);
  cb.moff.push_back(cb.m_total);
  if ((e = upload_i(W.d_k, W.k, s)) != cudaSuccess) return e;
  if ((e = upload_ll(W.d_koff, W.koff, s)) != cudaSuccess) return e;
  if ((e = upload_ll(W.d_cmoff, W.cmoff, s)) != cudaSuccess) return e;
  if ((e = upload_i(W.d_cld, cld, s)) != cudaSuccess) return e;
  if ((e = upload_i(W.d_Klist, Kl, s)) != cudaSuccess) return e;
  W.d_delta.release();
  if ((e = cudaMalloc(&W.d_delta.p, sizeof(double) * std::max<size_t>(1, dl.size()))) != cudaSuccess) return e;
  W.d_delta.bytes = sizeof(double) * std::max<size_t>(1, dl.size());
  if ((e = cudaMemcpyAsync(W.d_delta.p, dl.data(), sizeof(double) * dl.size(), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = upload_ll(W.d_rpre, W.rpre, s)) != cudaSuccess) return e;
  if ((e = upload_ll(W.d_woff, W.woff, s)) != cudaSuccess) return e;
  if (cb.nblk == 0) return cudaStreamSynchronize(s);
  if ((e = upload_i(cb.d_n, cb.n, s)) != cudaSuccess) return e;
  if ((e = upload_i(cb.d_ld, cb.ld, s)) != cudaSuccess) return e;
  if ((e = upload_ll(cb.d_ioff, std::vector<long long>(cb.ioff.begin(), cb.ioff.end() - 1), s)) != cudaSuccess)
    return e;
  if ((e = upload_ll(cb.d_moff, std::vector<long long>(cb.moff.begin(), cb.moff.end() - 1), s)) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&cb.mat.p, sizeof(ST) * (size_t)cb.m_total)) != cudaSuccess) return e;
  cb.mat.bytes = sizeof(ST) * (size_t)cb.m_total;
  if ((e = cudaMemsetAsync(cb.mat.p, 0, cb.mat.bytes, s)) != cudaSuccess) return e;
  DevBuf d_epre;
  if ((e = upload_ll(d_epre, epre, s)) != cudaSuccess) return e;
  { pns::count_launch(); k_cap_assemble<ST><<<(unsigned)((epre[B.nblk] + 255) / 256), 256, 0, s>>>(
      d_epre.as<long long>(), B.nblk, W.d_k.as<int>(), W.d_koff.as<long long>(), W.d_cmoff.as<long long>(),
      W.d_cld.as<int>(), W.d_Klist.as<int>(), W.d_delta.as<double>(), B.d_ld.as<int>(), B.d_moff.as<long long>(), X,
      cb.mat.as<ST>()); }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the capacitance inverses, by the same blocked Gauss-Jordan (no pivoting) as the local inverses: on the
  // tensor cores in the FP32 build; a zero or non-finite pivot raises the build's singular flag
  if ((e = launch_gj_invert<ST>(cb, cb.mat.as<ST>(), d_bad, s, nullptr, C.opt.gj_tensor_cores)) != cudaSuccess)
    return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// S = Abar^{-1} R for every primary block (R, S: n x kc per block at offsets roff, FP64)
template <typename ST>
cudaError_t Woodbury::apply(const Ctx& C, const BlockSet& B, const ST* X, const double* R, double* S, double* Y,
                            const long long* d_roff, const int* d_kc, const std::vector<int>& kc) {
  cudaStream_t s = C.stream;
  WoodburyImpl& W = *impl;
  cudaError_t e = launch_block_mm<ST, ST>(B, X, R, d_roff, d_kc, kc, Y, s);
  if (e != cudaSuccess) return e;
  long long wtot = W.woff[B.nblk];
  double *Wm = nullptr, *Z = nullptr;
  if ((e = cudaMalloc(&Wm, sizeof(double) * std::max(1LL, wtot))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&Z, sizeof(double) * std::max(1LL, wtot))) != cudaSuccess) { cudaFree(Wm); return e; }
  cudaMemsetAsync(Wm, 0, sizeof(double) * std::max(1LL, wtot), s);
  cudaMemsetAsync(Z, 0, sizeof(double) * std::max(1LL, wtot), s);
  if (W.rpre[B.nblk] > 0) {
    { pns::count_launch(); k_gather_rows<<<(unsigned)((W.rpre[B.nblk] + 127) / 128), 128, 0, s>>>(
        B.nblk, W.d_rpre.as<long long>(), W.d_k.as<int>(), W.d_koff.as<long long>(), W.d_Klist.as<int>(), d_roff,
        W.d_woff.as<long long>(), d_kc, Y, Wm); }
    { pns::count_launch(); k_cap_mm<ST><<<(unsigned)((W.rpre[B.nblk] * 32 + 255) / 256), 256, 0, s>>>(
        B.nblk, W.d_rpre.as<long long>(), W.d_k.as<int>(), W.d_cmoff.as<long long>(), W.d_cld.as<int>(),
        W.cb.mat.as<ST>(),
        W.d_woff.as<long long>(), d_kc, Wm, Z); }
  }
  { pns::count_launch(); k_woodbury_update<ST><<<(unsigned)((B.n_total * 32 + 255) / 256), 256, 0, s>>>(
      B.nblk, B.d_ioff.as<long long>(), B.d_n.as<int>(), B.d_ld.as<int>(), B.d_moff.as<long long>(), X, B.n_total,
      W.d_k.as<int>(), W.d_koff.as<long long>(), W.d_Klist.as<int>(), d_roff, W.d_woff.as<long long>(), d_kc, Y, Z,
      S); }
  e = cudaStreamSynchronize(s);
  cudaFree(Wm);
  cudaFree(Z);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template cudaError_t Woodbury::setup<float>(const Ctx&, const BlockSet&, int, const double*, const float*,
                                            const std::vector<int>&, int*);
template cudaError_t Woodbury::setup<double>(const Ctx&, const BlockSet&, int, const double*, const double*,
                                             const std::vector<int>&, int*);
template cudaError_t Woodbury::apply<float>(const Ctx&, const BlockSet&, const float*, const double*, double*,
                                            double*, const long long*, const int*, const std::vector<int>&);
template cudaError_t Woodbury::apply<double>(const Ctx&, const BlockSet&, const double*, const double*, double*,
                                             double*, const long long*, const int*, const std::vector<int>&);

}  // namespace pns
