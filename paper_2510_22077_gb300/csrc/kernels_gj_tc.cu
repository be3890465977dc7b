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

namespace pns {

namespace {

constexpr int TT = 128;          // tile edge (M = N) and panel width
constexpr int KCH = 32;          // K chunk: 32 FP32 = one 128-byte swizzle row
constexpr int NST = 2;           // operand stages
constexpr long long WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity to complete; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle layout: rows of
// 128 bytes, 8-row swizzle atoms 1024 bytes apart (stride byte offset), descriptor version 1, layout
// type 2 (SWIZZLE_128B).  The tile base is 1024-byte aligned; the K offset inside the atom is added to
// the start address.
__device__ __forceinline__ uint64_t sw128_desc(const void* tile, uint32_t kbyte) {
  const uint32_t a = smem_u32(tile) + kbyte;
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused by swizzled K-major layouts)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
  return d;
}

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32, A and B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TT >> 3) << 17) |
                                ((uint32_t)(TT >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC_TF32), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 32 columns of 32 bits: lane (32 w + t) of warp w goes to thread t
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

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
        mma_tf32(tmem, ah, bh, (c | kk) != 0);
        mma_tf32(tmem, ah, bl, 1);
        mma_tf32(tmem, al, bh, 1);
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
  ~GjTcImpl() {
    if (panels) cudaFree(panels);
    if (d_maps) cudaFree(d_maps);
    if (d_preT) cudaFree(d_preT);
  }
};

GjTc::GjTc() : impl(nullptr) {}
GjTc::~GjTc() { delete impl; }

cudaError_t GjTc::setup(const BlockSet& B, float* mat, cudaStream_t s) {
  delete impl;
  impl = new GjTcImpl;
  GjTcImpl& I = *impl;
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
    attr = true;
  }
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
  if (ntiles > 0) {
    pns::count_launch();
    k_gj_update_tc<<<(unsigned)ntiles, 128, sizeof(TcSmem) + 1024, s>>>(
        k, cnt, d_order, d_pre2, B.d_n.as<int>(), B.d_ioff.as<long long>(), I.d_maps, I.pa_hi, I.pa_lo, I.pb_hi,
        I.pb_lo, d_bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pns
