// Gauss-Jordan trailing update of the FP32 local inverses on the 5th-generation tensor cores
// (tcgen05, sm_103a): A[I, J] -= A[I, P] * A[P, J] for every 128 x 128 tile I != k, J != k of every
// active block at panel step k (the dominant work of the local-inverse build of Eq. 25).
//
// FP32 accuracy from TF32 units: each operand is split as x = hi + lo, hi = x rounded to TF32 and
// lo = (x - hi) rounded to TF32, and the tile product accumulates hi*hi + hi*lo + lo*hi in FP32 (the
// dropped lo*lo term is ~2^-22 of the product).
//
// Data flow of one step:
//  * k_gj_panels writes both panels of the step, already split, into K-major panel buffers:
//      PA[row(b, i)][c] = A_b[i][p0 + c]      (the column panel, before the column-panel update),
//      PB[row(b, j)][c] = A_b[p0 + c][j]      (the row panel after D^{-1} was applied, transposed),
//    row(b, i) = packed offset of block b + i, c < 128 (zero for c >= the panel width);
//  * k_gj_update_tc, one CTA per output tile (4 warps): thread 0 loads the C tile (four 32-column
//    boxes) and the four operand tiles of each 32-wide K chunk with TMA into 128-byte-swizzled shared
//    memory (two stages), thread 32 issues tcgen05.mma kind::tf32 (M = N = 128, K = 8) into a
//    128-column TMEM accumulator, and all four warps read the accumulator back with tcgen05.ld,
//    subtract it from the C tile in shared memory, and thread 0 stores the tile with TMA.  Ragged
//    edges: the per-block tensor map of the matrix has the block's true size, so loads past it read
//    zero and stores past it are dropped.
// Every wait on an mbarrier is bounded (~1 s of clock); on a timeout the kernel sets bit 2 of the
// error flag, skips its store, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc5.cuh"

namespace pns {

namespace {

using namespace tc5;

constexpr int TT = 128;          // tile edge (M = N) and panel width
constexpr int KCH = 32;          // K chunk: 32 FP32 = one 128-byte swizzle row
constexpr int NST = 2;           // operand stages
// tcgen05.mma kind::tf32, D FP32, A and B TF32 K-major, M = N = 128
constexpr uint32_t IDESC_TF32 = idesc(FMT_TF32, TT, TT);

struct __align__(1024) TcSmem {
  float c[4][TT][KCH];           // C tile, 4 boxes of 32 columns (64 KB)
  float a_hi[NST][TT][KCH];      // 16 KB each
  float a_lo[NST][TT][KCH];
  float b_hi[NST][TT][KCH];
  float b_lo[NST][TT][KCH];
  unsigned long long full[NST], empty[NST], cbar, done;
  uint32_t tmem;
  int fail;
};

__device__ __forceinline__ int find_blk(const long long* __restrict__ off, int nb, long long t) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int skip_k(int t, int k) { return t + (t >= k); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// --------------------------------------------------------------------------------- panels
// One CTA (256 threads) per 128-row chunk q of an active block: PA rows [q*128, q*128 + 128) and PB rows
// (columns j of the row panel) of the same range, split into hi / lo.  Rows past the block size are left
// as they are (they only feed C rows and columns that the tensor-map bounds drop).
__global__ void __launch_bounds__(256) k_gj_panels(int k, int cnt, const int* __restrict__ order,
                                                   const long long* __restrict__ preT, const int* __restrict__ bn,
                                                   const int* __restrict__ bld, const long long* __restrict__ moff,
                                                   const long long* __restrict__ ioff, const float* __restrict__ mat,
                                                   float* __restrict__ pa_hi, float* __restrict__ pa_lo,
                                                   float* __restrict__ pb_hi, float* __restrict__ pb_lo) {
  __shared__ float tr[32][TT + 1];
  const long long w = blockIdx.x;
  const int s = find_blk(preT, cnt, w);
  const int b = order[s];
  const int n = bn[b], ld = bld[b];
  const int q = (int)(w - preT[s]);
  const int p0 = k * TT, nb = min(TT, n - p0);
  const int r0 = q * TT, nr = min(TT, n - r0);
  const float* A = mat + moff[b];
  const long long prow = ioff[b] + r0;
  // column panel: PA[r][c] = A[r0 + r][p0 + c]
  for (int e = threadIdx.x; e < TT * TT; e += blockDim.x) {
    const int r = e / TT, c = e % TT;
    if (r >= nr) break;
    const float x = c < nb ? A[(long long)(r0 + r) * ld + p0 + c] : 0.f;
    const float hi = tf32_round(x);
    const long long o = (prow + r) * TT + c;
    pa_hi[o] = hi;
    pa_lo[o] = tf32_round(x - hi);
  }
  // row panel, transposed through shared memory in slabs of 32 panel rows: PB[j][c] = A[p0 + c][r0 + j]
  for (int c0 = 0; c0 < TT; c0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * TT; e += blockDim.x) {
      const int cc = e / TT, j = e % TT;
      const int c = c0 + cc;
      tr[cc][j] = (c < nb && j < nr) ? A[(long long)(p0 + c) * ld + r0 + j] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * TT; e += blockDim.x) {
      const int j = e / 32, cc = e % 32;
      if (j >= nr) break;
      const float x = tr[cc][j];
      const float hi = tf32_round(x);
      const long long o = (prow + j) * TT + c0 + cc;
      pb_hi[o] = hi;
      pb_lo[o] = tf32_round(x - hi);
    }
  }
}

// --------------------------------------------------------------------------------- update
__global__ void __launch_bounds__(128, 1) k_gj_update_tc(int k, int cnt, const int* __restrict__ order,
                                                         const long long* __restrict__ pre2,
                                                         const int* __restrict__ bn,
                                                         const long long* __restrict__ ioff,
                                                         const CUtensorMap* __restrict__ mat_maps,
                                                         const __grid_constant__ CUtensorMap pa_hi,
                                                         const __grid_constant__ CUtensorMap pa_lo,
                                                         const __grid_constant__ CUtensorMap pb_hi,
                                                         const __grid_constant__ CUtensorMap pb_lo,
                                                         int* __restrict__ flag) {
  extern __shared__ unsigned char smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long w = blockIdx.x;
  const int s = find_blk(pre2, cnt, w);
  const int b = order[s];
  const int n = bn[b];
  const int T = (n + TT - 1) / TT;
  const long long loc = w - pre2[s];
  const int i0 = skip_k((int)(loc / (T - 1)), k) * TT, j0 = skip_k((int)(loc % (T - 1)), k) * TT;
  const int rowA = (int)(ioff[b] + i0), rowB = (int)(ioff[b] + j0);
  const CUtensorMap* cmap = mat_maps + b;

  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) {
      mbar_init(&S.full[st], 1);
      mbar_init(&S.empty[st], 1);
    }
    mbar_init(&S.cbar, 1);
    mbar_init(&S.done, 1);
    S.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                 "r"(TT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;

  if (threadIdx.x == 0) {
    // producer: the C tile, then the operand chunks through the two stages
    mbar_expect_tx(&S.cbar, (uint32_t)sizeof(S.c));
    for (int q = 0; q < 4; ++q) tma_load_2d(&S.c[q][0][0], cmap, j0 + q * KCH, i0, &S.cbar);
    for (int c = 0; c < TT / KCH; ++c) {
      const int st = c % NST;
      if (c >= NST && !mbar_wait(&S.empty[st], ((c - NST) / NST) & 1)) {
        atomicOr(&S.fail, 1);
        break;
      }
      mbar_expect_tx(&S.full[st], 4u * TT * KCH * 4u);
      tma_load_2d(&S.a_hi[st][0][0], &pa_hi, c * KCH, rowA, &S.full[st]);
      tma_load_2d(&S.a_lo[st][0][0], &pa_lo, c * KCH, rowA, &S.full[st]);
      tma_load_2d(&S.b_hi[st][0][0], &pb_hi, c * KCH, rowB, &S.full[st]);
      tma_load_2d(&S.b_lo[st][0][0], &pb_lo, c * KCH, rowB, &S.full[st]);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: per chunk 4 K-steps of 8, three products each
    for (int c = 0; c < TT / KCH; ++c) {
      const int st = c % NST;
      if (!mbar_wait(&S.full[st], (c / NST) & 1)) {
        atomicOr(&S.fail, 1);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < KCH / 8; ++kk) {
        const uint32_t kb = kk * 32;
        const uint64_t ah = sw128_desc(&S.a_hi[st][0][0], kb), al = sw128_desc(&S.a_lo[st][0][0], kb);
        const uint64_t bh = sw128_desc(&S.b_hi[st][0][0], kb), bl = sw128_desc(&S.b_lo[st][0][0], kb);
        mma_tf32(tmem, ah, bh, IDESC_TF32, (c | kk) != 0);
        mma_tf32(tmem, ah, bl, IDESC_TF32, 1);
        mma_tf32(tmem, al, bh, IDESC_TF32, 1);
      }
      mma_commit(&S.empty[st]);
    }
    mma_commit(&S.done);
  }
  __syncwarp();
  // epilogue: C -= accumulator, row r = 32 warp + lane of the tile, in the swizzled C boxes
  bool ok = mbar_wait(&S.cbar, 0);
  ok = mbar_wait(&S.done, 0) && ok;
  tc_fence_after();
  if (!ok) atomicOr(&S.fail, 1);
  __syncthreads();
  const bool good = S.fail == 0;
  if (good) {
    const int r = warp * 32 + lane;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * KCH), v);
      float* crow = &S.c[q][r][0];
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) {
        float4* p = reinterpret_cast<float4*>(crow + ((ch ^ (r & 7)) * 4));
        float4 x = *p;
        x.x -= v[ch * 4 + 0];
        x.y -= v[ch * 4 + 1];
        x.z -= v[ch * 4 + 2];
        x.w -= v[ch * 4 + 3];
        *p = x;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (good) {
      for (int q = 0; q < 4; ++q) tma_store_2d(cmap, j0 + q * KCH, i0, &S.c[q][0][0]);
      asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
    } else {
      atomicOr(flag, 2);
    }
  }
  __syncwarp();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TT) : "memory");
  }
}

// --------------------------------------------------------------------------------- persistent update
// The same update as k_gj_update_tc, persistent and warp-specialised so that the C traffic of consecutive
// tiles never stops: one CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
//  * warp 0 (one thread) streams the operand chunks of each tile through NST stages;
//  * warp 6 (one thread) streams the C boxes (128 rows x 32 columns, four per tile) through a ring of NCS
//    slots, so that the loads of the next tile's C run while the current tile is written back;
//  * warp 1 (one thread) issues the MMAs of each tile into one of two 128-column TMEM accumulators;
//  * warps 2-5 read an accumulator back (warp w owns TMEM lanes 32 (w % 4) ..), subtract it from each C
//    box in shared memory as the box arrives, and store the box with TMA; a slot is handed back to the
//    C loader once the store of the box after it has been issued and its own store has read the slot.
// The tile's update is HBM-bound (its C tile is read and written once per step; the panels stay in L2),
// so the point is to keep loads and stores in flight on every SM at all times.  A wait that times out
// raises the CTA's abort flag, which ends every role's loop; the roles then wait (bounded) for their own
// copies and MMAs in flight before the TMEM is freed.
constexpr int NCS = 6;           // C box slots (16 KB each)
struct __align__(1024) TcpSmem {
  float c[NCS][TT][KCH];         // ring of C boxes (96 KB)
  float a_hi[NST][TT][KCH];
  float a_lo[NST][TT][KCH];
  float b_hi[NST][TT][KCH];
  float b_lo[NST][TT][KCH];
  unsigned long long full[NST], empty[NST], c_full[NCS], c_empty[NCS], acc_full[2], acc_empty[2], drain;
  uint32_t tmem;
  volatile int abort;
};
static_assert(sizeof(TcpSmem) + 1024 <= 232448, "shared memory of the persistent update");

__device__ __forceinline__ bool wait_or_abort(unsigned long long* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// barrier over the 128 epilogue threads that also ORs a predicate across them: every thread gets the same
// answer, so the epilogue warps always leave their loop together
__device__ __forceinline__ bool epi_any(bool q) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)q)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void tile_of(long long w, int k, int cnt, const int* __restrict__ order,
                                        const long long* __restrict__ pre2, const int* __restrict__ bn,
                                        const long long* __restrict__ ioff, int& b, int& i0, int& j0, int& rowA,
                                        int& rowB) {
  const int s = find_blk(pre2, cnt, w);
  b = order[s];
  const int n = bn[b];
  const int T = (n + TT - 1) / TT;
  const long long loc = w - pre2[s];
  i0 = skip_k((int)(loc / (T - 1)), k) * TT;
  j0 = skip_k((int)(loc % (T - 1)), k) * TT;
  rowA = (int)(ioff[b] + i0);
  rowB = (int)(ioff[b] + j0);
}

__global__ void __launch_bounds__(224, 1) k_gj_update_tcp(int k, int cnt, long long ntiles,
                                                          const int* __restrict__ order,
                                                          const long long* __restrict__ pre2,
                                                          const int* __restrict__ bn,
                                                          const long long* __restrict__ ioff,
                                                          const CUtensorMap* __restrict__ mat_maps,
                                                          const __grid_constant__ CUtensorMap pa_hi,
                                                          const __grid_constant__ CUtensorMap pa_lo,
                                                          const __grid_constant__ CUtensorMap pb_hi,
                                                          const __grid_constant__ CUtensorMap pb_lo,
                                                          int* __restrict__ flag) {
  extern __shared__ unsigned char smraw[];
  TcpSmem& S = *reinterpret_cast<TcpSmem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) {
      mbar_init(&S.full[st], 1);
      mbar_init(&S.empty[st], 1);
    }
    for (int sl = 0; sl < NCS; ++sl) {
      mbar_init(&S.c_full[sl], 1);
      mbar_init(&S.c_empty[sl], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&S.acc_full[q], 1);
      mbar_init(&S.acc_empty[q], 128);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&S.tmem, 2 * TT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;

  if (warp == 0) {
    if (lane == 0) {
      // operand producer
      long long q = 0;
      for (long long w = blockIdx.x; w < ntiles && !S.abort; w += gridDim.x) {
        int b, i0, j0, rowA, rowB;
        tile_of(w, k, cnt, order, pre2, bn, ioff, b, i0, j0, rowA, rowB);
        for (int c = 0; c < TT / KCH; ++c) {
          const int st = (int)(q % NST);
          if (q >= NST && !wait_or_abort(&S.empty[st], (uint32_t)(((q - NST) / NST) & 1), &S.abort)) break;
          mbar_expect_tx(&S.full[st], 4u * TT * KCH * 4u);
          tma_load_2d(&S.a_hi[st][0][0], &pa_hi, c * KCH, rowA, &S.full[st]);
          tma_load_2d(&S.a_lo[st][0][0], &pa_lo, c * KCH, rowA, &S.full[st]);
          tma_load_2d(&S.b_hi[st][0][0], &pb_hi, c * KCH, rowB, &S.full[st]);
          tma_load_2d(&S.b_lo[st][0][0], &pb_lo, c * KCH, rowB, &S.full[st]);
          ++q;
        }
      }
      if (S.abort)   // the chunks still in flight land before the CTA ends (the latest phase of each stage)
        for (long long qq = q > NST ? q - NST : 0; qq < q; ++qq)
          mbar_wait(&S.full[qq % NST], (uint32_t)((qq / NST) & 1));
    }
  } else if (warp == 6) {
    if (lane == 0) {
      // C producer: box g of the CTA = box g % 4 of its tile g / 4, in slot g % NCS
      long long g = 0;
      for (long long w = blockIdx.x; w < ntiles && !S.abort; w += gridDim.x) {
        int b, i0, j0, rowA, rowB;
        tile_of(w, k, cnt, order, pre2, bn, ioff, b, i0, j0, rowA, rowB);
        for (int qq = 0; qq < 4; ++qq) {
          const int sl = (int)(g % NCS);
          if (g >= NCS && !wait_or_abort(&S.c_empty[sl], (uint32_t)(((g - NCS) / NCS) & 1), &S.abort)) break;
          mbar_expect_tx(&S.c_full[sl], (uint32_t)(TT * KCH * sizeof(float)));
          tma_load_2d(&S.c[sl][0][0], mat_maps + b, j0 + qq * KCH, i0, &S.c_full[sl]);
          ++g;
        }
      }
      if (S.abort)
        for (long long gg = g > NCS ? g - NCS : 0; gg < g; ++gg)
          mbar_wait(&S.c_full[gg % NCS], (uint32_t)((gg / NCS) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      long long q = 0;
      int it = 0;
      bool issued = false;
      for (long long w = blockIdx.x; w < ntiles && !S.abort; w += gridDim.x, ++it) {
        const int ab = it & 1;
        if (it >= 2 && !wait_or_abort(&S.acc_empty[ab], (uint32_t)(((it - 2) >> 1) & 1), &S.abort)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(ab * TT);
        bool ok = true;
        for (int c = 0; c < TT / KCH; ++c, ++q) {
          const int st = (int)(q % NST);
          if (!wait_or_abort(&S.full[st], (uint32_t)((q / NST) & 1), &S.abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < KCH / 8; ++kk) {
            const uint32_t kb = kk * 32;
            const uint64_t ah = sw128_desc(&S.a_hi[st][0][0], kb), al = sw128_desc(&S.a_lo[st][0][0], kb);
            const uint64_t bh = sw128_desc(&S.b_hi[st][0][0], kb), bl = sw128_desc(&S.b_lo[st][0][0], kb);
            mma_tf32(acc, ah, bh, IDESC_TF32, (c | kk) != 0);
            mma_tf32(acc, ah, bl, IDESC_TF32, 1);
            mma_tf32(acc, al, bh, IDESC_TF32, 1);
          }
          issued = true;
          mma_commit(&S.empty[st]);
        }
        if (!ok) break;
        mma_commit(&S.acc_full[ab]);
      }
      if (S.abort && issued) {   // every MMA this thread issued has finished before the TMEM is freed
        mma_commit(&S.drain);
        mbar_wait(&S.drain, 0);
      }
    }
  } else {
    // epilogue: warps 2..5, TMEM lane quarter warp % 4
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;
    const bool leader = warp == 2 && lane == 0;
    long long g = 0;
    int it = 0;
    bool stop = false;
    for (long long w = blockIdx.x; w < ntiles && !stop; w += gridDim.x, ++it) {
      int b, i0, j0, rowA, rowB;
      tile_of(w, k, cnt, order, pre2, bn, ioff, b, i0, j0, rowA, rowB);
      const int ab = it & 1;
      const bool ok = wait_or_abort(&S.acc_full[ab], (uint32_t)((it >> 1) & 1), &S.abort);
      if (epi_any(!ok || S.abort)) break;
      tc_fence_after();
      const uint32_t acc = tmem + (uint32_t)(ab * TT) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int qq = 0; qq < 4; ++qq, ++g) {
        const int sl = (int)(g % NCS);
        float v[32];
        tmem_ld32(acc + (uint32_t)(qq * KCH), v);
        if (qq == 3) {   // the accumulator is read out: the MMAs of the tile after next may use it
          tc_fence_before();
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&S.acc_empty[ab])) : "memory");
        }
        const bool okc = wait_or_abort(&S.c_full[sl], (uint32_t)((g / NCS) & 1), &S.abort);
        if (epi_any(!okc || S.abort)) {
          stop = true;
          break;
        }
        float* crow = &S.c[sl][r][0];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          float4* p = reinterpret_cast<float4*>(crow + ((ch ^ (r & 7)) * 4));
          float4 x = *p;
          x.x -= v[ch * 4 + 0];
          x.y -= v[ch * 4 + 1];
          x.z -= v[ch * 4 + 2];
          x.w -= v[ch * 4 + 3];
          *p = x;
        }
        fence_async_smem();
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (leader) {
          tma_store_2d(mat_maps + b, j0 + qq * KCH, i0, &S.c[sl][0][0]);
          asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
          // every store but the newest has read its slot: hand the previous box's slot back
          asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
          if (g > 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&S.c_empty[(g - 1) % NCS]))
                         : "memory");
        }
      }
    }
    if (leader) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && S.abort) atomicOr(flag, 2);
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, 2 * TT);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D FP32 tensor map: width x height elements, row pitch `pitch` elements, 32 x 128 boxes, 128-byte swizzle
bool make_map(CUtensorMap* m, const float* base, long long width, long long height, long long pitch) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  cuuint32_t box[2] = {KCH, TT};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct GjTcImpl {
  float* panels = nullptr;       // pa_hi | pa_lo | pb_hi | pb_lo, rows x 128 each
  CUtensorMap* d_maps = nullptr; // one matrix map per block
  long long rows = 0;
  CUtensorMap pa_hi, pa_lo, pb_hi, pb_lo;
  long long* d_preT = nullptr;
  int sms = 148;
  bool persistent = true;
  ~GjTcImpl() {
    if (panels) cudaFree(panels);
    if (d_maps) cudaFree(d_maps);
    if (d_preT) cudaFree(d_preT);
  }
};

GjTc::GjTc() : impl(nullptr) {}
GjTc::~GjTc() { delete impl; }

cudaError_t GjTc::setup(const BlockSet& B, float* mat, cudaStream_t s, bool persistent) {
  delete impl;
  impl = new GjTcImpl;
  GjTcImpl& I = *impl;
  I.persistent = persistent;
  I.rows = std::max<long long>(B.n_total, 1);
  cudaError_t e = cudaMalloc(&I.panels, sizeof(float) * (size_t)I.rows * TT * 4);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&I.d_maps, sizeof(CUtensorMap) * std::max(1, B.nblk));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&I.d_preT, sizeof(long long) * (B.nblk + 1));
  if (e != cudaSuccess) return e;
  std::vector<CUtensorMap> maps(std::max(1, B.nblk));
  for (int b = 0; b < B.nblk; ++b)
    if (!make_map(&maps[b], mat + B.moff[b], B.n[b], B.n[b], B.ld[b])) return cudaErrorInvalidValue;
  const size_t pn = (size_t)I.rows * TT;
  if (!make_map(&I.pa_hi, I.panels, TT, I.rows, TT) || !make_map(&I.pa_lo, I.panels + pn, TT, I.rows, TT) ||
      !make_map(&I.pb_hi, I.panels + 2 * pn, TT, I.rows, TT) || !make_map(&I.pb_lo, I.panels + 3 * pn, TT, I.rows, TT))
    return cudaErrorInvalidValue;
  e = cudaMemcpyAsync(I.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(I.panels, 0, sizeof(float) * pn * 4, s);
  if (e != cudaSuccess) return e;
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(k_gj_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(TcSmem) + 1024));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gj_update_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(TcpSmem) + 1024));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&impl->sms, cudaDevAttrMultiProcessorCount, dev);
  return cudaSuccess;
}

cudaError_t GjTc::step(const BlockSet& B, float* mat, int k, int cnt, const int* d_order, const long long* d_pre2,
                       long long ntiles, const std::vector<int>& order, int* d_bad, cudaStream_t s) {
  GjTcImpl& I = *impl;
  // panels: one CTA per 128-row chunk of every active block
  std::vector<long long> preT(cnt + 1, 0);
  for (int q = 0; q < cnt; ++q) preT[q + 1] = preT[q] + (B.n[order[q]] + TT - 1) / TT;
  cudaError_t e = cudaMemcpyAsync(I.d_preT, preT.data(), sizeof(long long) * (cnt + 1), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  pns::count_launch();
  k_gj_panels<<<(unsigned)preT[cnt], 256, 0, s>>>(k, cnt, d_order, I.d_preT, B.d_n.as<int>(), B.d_ld.as<int>(),
                                                   B.d_moff.as<long long>(), B.d_ioff.as<long long>(), mat,
                                                   I.panels, I.panels + (size_t)I.rows * TT,
                                                   I.panels + 2 * (size_t)I.rows * TT,
                                                   I.panels + 3 * (size_t)I.rows * TT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ntiles > 0 && I.persistent) {
    pns::count_launch();
    const unsigned grid = (unsigned)std::min<long long>(ntiles, I.sms);
    k_gj_update_tcp<<<grid, 224, sizeof(TcpSmem) + 1024, s>>>(k, cnt, ntiles, d_order, d_pre2, B.d_n.as<int>(),
                                                               B.d_ioff.as<long long>(), I.d_maps, I.pa_hi, I.pa_lo,
                                                               I.pb_hi, I.pb_lo, d_bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (ntiles > 0) {
    pns::count_launch();
    k_gj_update_tc<<<(unsigned)ntiles, 128, sizeof(TcSmem) + 1024, s>>>(
        k, cnt, d_order, d_pre2, B.d_n.as<int>(), B.d_ioff.as<long long>(), I.d_maps, I.pa_hi, I.pa_lo, I.pb_hi,
        I.pb_lo, d_bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pns
