// Learned Newton initial guess (include/pns_unet.h): a 3D U-Net trained and run on the GPU with
// hand-written BF16 kernels on the 5th-generation tensor cores.
//
// Layout: activations are BF16, channels-last (N, D, H, W, C) with a channel stride that is a multiple of
// 8 (16-byte rows of 8 channels; padding channels stay zero), so a view of a buffer is (pointer, channel
// stride, channel offset).  The decoder's concatenation is a buffer whose first channels are written by
// the upsampling and whose last channels are written directly by the encoder's second convolution.
//
// Convolutions are implicit GEMMs on tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator in TMEM):
//  * k_conv_tc -- forward and data gradient: D[voxel][o] = sum_k im2col(x)[voxel][k] W[o][k] with
//    k = tap * cin_p + c (taps in (dz, dy, dx) order, channels padded to cin_p); 128 voxels per CTA,
//    N = the padded output channels; all 128 threads gather the im2col tile and the weight tile of each
//    64-wide K chunk into 128-byte-swizzled shared memory (two stages), thread 0 issues the MMAs, and the
//    epilogue adds the bias, applies ReLU or the data-gradient mask (the forward input > 0) and stores.
//    The data gradient is the same GEMM with the weights flipped in space and transposed in channels.
//  * k_wgrad_tc -- weight gradient: D[k][o] = sum_voxel im2col(x)[voxel][k] g[voxel][o], 128 rows of k per
//    CTA, the voxels split over CTAs (split-K), the operand tiles transposed on their way into shared
//    memory, partial sums added to an FP32 buffer with atomics.
// Every mbarrier wait is bounded; a timeout sets bit 2 of the error flag and the kernel returns after
// freeing its TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/pns.h"
#include "../../include/pns_unet.h"
#include "tc5.cuh"

namespace pns {
void count_launch();
}

namespace {

using namespace pns::tc5;
using bf16 = __nv_bfloat16;

constexpr int CM = 128;   // voxels (GEMM rows) per CTA of k_conv_tc; k rows per CTA of k_wgrad_tc
constexpr int CK = 64;    // K chunk: 64 BF16 = one 128-byte swizzle row

int r8(int c) { return (c + 7) / 8 * 8; }
int r16(int c) { return (c + 15) / 16 * 16; }
int r64(int c) { return (c + 63) / 64 * 64; }

__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

// ------------------------------------------------------------------------------------------ conv
struct ConvP {
  const bf16* x;
  int x_cs, x_coff, cin_p, taps;  // input view; K = taps * cin_p
  const bf16* wt;
  int kpad, npad, cout;           // packed weights [npad][kpad]; real output channels
  const float* bias;              // may be null
  int relu;
  const bf16* mask;               // output *= (mask > 0) (data gradient), may be null
  int m_cs, m_coff;
  bf16* y;                        // BF16 channels-last output view (may be null)
  int y_cs, y_coff;
  float* y32;                     // FP32 (N, C, D, H, W) output (may be null)
  int n, d, h, w;
  int* flag;
};

struct __align__(1024) ConvSmem {
  bf16 a[2][CM][CK];
  bf16 b[2][128][CK];
  unsigned long long empty[2], done;
  uint32_t tmem;
};

__device__ __forceinline__ void st_chunk(bf16* tile, int row, int chunk, uint4 v) {
  *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(tile) + (row >> 3) * 1024 + (row & 7) * 128 +
                            (((chunk ^ row) & 7) << 4)) = v;
}

__global__ void __launch_bounds__(128) k_conv_tc(ConvP P) {
  extern __shared__ unsigned char smraw[];
  ConvSmem& S = *reinterpret_cast<ConvSmem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long nvox = (long long)P.n * P.d * P.h * P.w;
  const long long m0 = (long long)blockIdx.x * CM;
  const uint32_t ncols = P.npad <= 32 ? 32 : (P.npad <= 64 ? 64 : 128);
  if (tid == 0) {
    mbar_init(&S.empty[0], 1);
    mbar_init(&S.empty[1], 1);
    mbar_init(&S.done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&S.tmem, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  // rows gathered by this thread: r = (tid >> 3) + 16 q, 16-byte chunk jj = tid & 7 of the K chunk
  const int jj = tid & 7;
  int vn[8], vz[8], vy[8], vx[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    long long v = m0 + (tid >> 3) + 16 * q;
    if (v >= nvox) {
      vn[q] = -1;
      vz[q] = vy[q] = vx[q] = 0;
      continue;
    }
    vx[q] = (int)(v % P.w);
    v /= P.w;
    vy[q] = (int)(v % P.h);
    v /= P.h;
    vz[q] = (int)(v % P.d);
    vn[q] = (int)(v / P.d);
  }
  const int nk = P.kpad / CK;
  const uint32_t id = idesc(FMT_BF16, CM, P.npad);
  bool failed = false;
  for (int c = 0; c < nk; ++c) {
    const int st = c & 1;
    if (c >= 2) {
      const bool ok = mbar_wait(&S.empty[st], ((c - 2) >> 1) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    // im2col tile: row = voxel, 8 channels of one tap per 16-byte chunk
    const int k0 = c * CK + jj * 8;
    const int tap = k0 / P.cin_p, ch = k0 - tap * P.cin_p;
    const int dz = P.taps == 27 ? tap_dz(tap) : 0, dy = P.taps == 27 ? tap_dy(tap) : 0,
              dx = P.taps == 27 ? tap_dx(tap) : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = (tid >> 3) + 16 * q;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (vn[q] >= 0 && tap < P.taps) {
        const int z = vz[q] + dz, yy = vy[q] + dy, xx = vx[q] + dx;
        if (z >= 0 && z < P.d && yy >= 0 && yy < P.h && xx >= 0 && xx < P.w) {
          const long long nb = (((long long)vn[q] * P.d + z) * P.h + yy) * P.w + xx;
          val = *reinterpret_cast<const uint4*>(P.x + nb * P.x_cs + P.x_coff + ch);
        }
      }
      st_chunk(&S.a[st][0][0], r, jj, val);
    }
    // weight tile: row = output channel
    for (int e = tid; e < P.npad * 8; e += 128) {
      const int o = e >> 3, j = e & 7;
      const uint4 val = *reinterpret_cast<const uint4*>(P.wt + (long long)o * P.kpad + c * CK + j * 8);
      st_chunk(&S.b[st][0][0], o, j, val);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < CK / 16; ++kk)
        mma_f16(tmem, sw128_desc(&S.a[st][0][0], kk * 32), sw128_desc(&S.b[st][0][0], kk * 32), id, (c | kk) != 0);
      mma_commit(&S.empty[st]);
    }
  }
  if (tid == 0) mma_commit(&S.done);
  const bool okd = mbar_wait(&S.done, 0);
  tc_fence_after();
  failed = __syncthreads_or(failed || !okd);
  if (!failed) {
    const long long v = m0 + tid;
    const bool valid = v < nvox;
    long long vv = v;
    const int x = (int)(vv % P.w);
    vv /= P.w;
    const int yq = (int)(vv % P.h);
    vv /= P.h;
    const int z = (int)(vv % P.d);
    const int nn = (int)(vv / P.d);
    for (int c0 = 0; c0 < P.npad; c0 += 16) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      if (!valid) continue;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int o = c0 + q;
        float r = acc[q];
        if (P.bias && o < P.cout) r += P.bias[o];
        if (P.relu) r = fmaxf(r, 0.f);
        if (P.mask && o < P.cout && !((float)P.mask[v * P.m_cs + P.m_coff + o] > 0.f)) r = 0.f;
        acc[q] = r;
      }
      if (P.y) {
        bf16* yp = P.y + v * P.y_cs + P.y_coff + c0;
        if (c0 + 16 <= P.cout) {
          __align__(16) bf16 tmp[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) tmp[q] = __float2bfloat16_rn(acc[q]);
          reinterpret_cast<uint4*>(yp)[0] = reinterpret_cast<const uint4*>(tmp)[0];
          reinterpret_cast<uint4*>(yp)[1] = reinterpret_cast<const uint4*>(tmp)[1];
        } else {
          for (int q = 0; q < 16 && c0 + q < P.cout; ++q) yp[q] = __float2bfloat16_rn(acc[q]);
        }
      }
      if (P.y32) {
        const long long plane = (long long)P.d * P.h * P.w;
        const long long sp = ((long long)z * P.h + yq) * P.w + x;
        for (int q = 0; q < 16 && c0 + q < P.cout; ++q)
          P.y32[((long long)nn * P.cout + c0 + q) * plane + sp] = acc[q];
      }
    }
  } else if (tid == 0) {
    atomicOr(P.flag, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, ncols);
  }
}

// ------------------------------------------------------------------------------------------ wgrad
struct WgP {
  const bf16* x;
  int x_cs, x_coff, cin_p, taps;  // forward input view
  const bf16* g;
  int g_cs, g_coff, npad, cout;   // gradient of the pre-activation (channels-last)
  int kreal;                      // taps * cin_p
  float* gw;                      // [rows >= kreal][npad] FP32, accumulated with atomics
  int n, d, h, w;
  long long vchunk;               // voxels per CTA (multiple of 64)
  int* flag;
};

struct __align__(1024) WgSmem {
  bf16 a[2][CM][CK];
  bf16 b[2][128][CK];
  unsigned long long empty[2], done;
  uint32_t tmem;
};

__device__ __forceinline__ void st_elem(bf16* tile, int row, int col, bf16 v) {
  *reinterpret_cast<bf16*>(reinterpret_cast<unsigned char*>(tile) + sw128_offset(row, col, 2)) = v;
}

__global__ void __launch_bounds__(128) k_wgrad_tc(WgP P) {
  extern __shared__ unsigned char smraw[];
  WgSmem& S = *reinterpret_cast<WgSmem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long nvox = (long long)P.n * P.d * P.h * P.w;
  const int k0 = blockIdx.x * CM;
  const long long v0 = (long long)blockIdx.y * P.vchunk;
  const long long v1 = min(nvox, v0 + P.vchunk);
  const uint32_t ncols = P.npad <= 32 ? 32 : (P.npad <= 64 ? 64 : 128);
  if (tid == 0) {
    mbar_init(&S.empty[0], 1);
    mbar_init(&S.empty[1], 1);
    mbar_init(&S.done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&S.tmem, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const int nk = (int)((v1 - v0 + CK - 1) / CK);
  const uint32_t id = idesc(FMT_BF16, CM, P.npad);
  bool failed = false;
  for (int c = 0; c < nk; ++c) {
    const int st = c & 1;
    if (c >= 2) {
      const bool ok = mbar_wait(&S.empty[st], ((c - 2) >> 1) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    const long long vb = v0 + (long long)c * CK;
    // A^T tile: row = k (8 rows of one tap per item), column = voxel
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 128 * q;
      const int kg = e >> 6, j = e & 63;
      const int kk = k0 + kg * 8;
      const long long v = vb + j;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (kk < P.kreal && v < v1) {
        const int tap = kk / P.cin_p, ch = kk - tap * P.cin_p;
        long long t = v;
        const int x = (int)(t % P.w);
        t /= P.w;
        const int yq = (int)(t % P.h);
        t /= P.h;
        const int z = (int)(t % P.d);
        const int nn = (int)(t / P.d);
        const int zz = z + (P.taps == 27 ? tap_dz(tap) : 0), yy = yq + (P.taps == 27 ? tap_dy(tap) : 0),
                  xx = x + (P.taps == 27 ? tap_dx(tap) : 0);
        if (zz >= 0 && zz < P.d && yy >= 0 && yy < P.h && xx >= 0 && xx < P.w) {
          const long long nb = (((long long)nn * P.d + zz) * P.h + yy) * P.w + xx;
          val = *reinterpret_cast<const uint4*>(P.x + nb * P.x_cs + P.x_coff + ch);
        }
      }
      const bf16* h = reinterpret_cast<const bf16*>(&val);
#pragma unroll
      for (int i = 0; i < 8; ++i) st_elem(&S.a[st][0][0], kg * 8 + i, j, h[i]);
    }
    // B^T tile: row = output channel, column = voxel
    for (int e = tid; e < P.npad * 8; e += 128) {
      const int og = e >> 6, j = e & 63;
      const long long v = vb + j;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v < v1 && og * 8 < P.cout) val = *reinterpret_cast<const uint4*>(P.g + v * P.g_cs + P.g_coff + og * 8);
      const bf16* h = reinterpret_cast<const bf16*>(&val);
#pragma unroll
      for (int i = 0; i < 8; ++i) st_elem(&S.b[st][0][0], og * 8 + i, j, h[i]);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < CK / 16; ++kk)
        mma_f16(tmem, sw128_desc(&S.a[st][0][0], kk * 32), sw128_desc(&S.b[st][0][0], kk * 32), id, (c | kk) != 0);
      mma_commit(&S.empty[st]);
    }
  }
  if (tid == 0) mma_commit(&S.done);
  const bool okd = mbar_wait(&S.done, 0);
  tc_fence_after();
  failed = __syncthreads_or(failed || !okd);
  if (!failed && nk > 0) {
    const int k = k0 + tid;
    for (int c0 = 0; c0 < P.npad; c0 += 16) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      if (k >= P.kreal) continue;
      for (int q = 0; q < 16 && c0 + q < P.cout; ++q) atomicAdd(P.gw + (long long)k * P.npad + c0 + q, acc[q]);
    }
  } else if (failed && tid == 0) {
    atomicOr(P.flag, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, ncols);
  }
}

// ------------------------------------------------------------------------------------------ small kernels
// bias gradient: gb[o] += sum over voxels of g[v][o]  (block: one thread per channel, a range of voxels)
__global__ void k_bias_grad(const bf16* __restrict__ g, int cs, int coff, int cout, long long nvox, long long chunk,
                            float* __restrict__ gb) {
  const int o = threadIdx.x;
  if (o >= cout) return;
  const long long v0 = (long long)blockIdx.x * chunk, v1 = min(nvox, v0 + chunk);
  float acc = 0.f;
  for (long long v = v0; v < v1; ++v) acc += (float)g[v * cs + coff + o];
  atomicAdd(gb + o, acc);
}

// FP32 (N, C, D, H, W) -> BF16 channels-last view (channels [0, C) of the view)
__global__ void k_to_cl(const float* __restrict__ x, int C, long long plane, long long nvox, bf16* __restrict__ y,
                        int cs, int coff) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox * C) return;
  const long long v = i / C;
  const int c = (int)(i - v * C);
  const long long n = v / plane, sp = v - n * plane;
  y[v * cs + coff + c] = __float2bfloat16_rn(x[(n * C + c) * plane + sp]);
}

// 2x2x2 max-pool of a channels-last view; arg = first maximum in (dz, dy, dx) order
__global__ void k_pool(const bf16* __restrict__ x, int x_cs, int x_coff, int C, int n, int d, int h, int w,
                       bf16* __restrict__ y, int y_cs, uint8_t* __restrict__ arg) {
  const int d2 = d / 2, h2 = h / 2, w2 = w / 2;
  const long long tot = (long long)n * d2 * h2 * w2 * C;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  long long v = i / C;
  const int X = (int)(v % w2);
  v /= w2;
  const int Y = (int)(v % h2);
  v /= h2;
  const int Z = (int)(v % d2);
  const int nn = (int)(v / d2);
  float best = -INFINITY;
  int ba = 0;
  for (int t = 0; t < 8; ++t) {
    const int z = 2 * Z + (t >> 2), yy = 2 * Y + ((t >> 1) & 1), xx = 2 * X + (t & 1);
    const long long src = (((long long)nn * d + z) * h + yy) * w + xx;
    const float val = (float)x[src * x_cs + x_coff + c];
    if (val > best) {
      best = val;
      ba = t;
    }
  }
  const long long dst = i / C;
  y[dst * y_cs + c] = __float2bfloat16_rn(best);
  arg[i] = (uint8_t)ba;
}

// gradient of the pool: g_x[child] += g_y[parent] where child is the parent's argmax (no atomics: each
// child element reads its own parent)
__global__ void k_pool_bwd(const bf16* __restrict__ gy, int gy_cs, const uint8_t* __restrict__ arg, int C, int n,
                           int d, int h, int w, bf16* __restrict__ gx, int gx_cs, int gx_coff) {
  const long long tot = (long long)n * d * h * w * C;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  long long v = i / C;
  const int x = (int)(v % w);
  v /= w;
  const int yy = (int)(v % h);
  v /= h;
  const int z = (int)(v % d);
  const int nn = (int)(v / d);
  const int t = ((z & 1) << 2) | ((yy & 1) << 1) | (x & 1);
  const long long par = (((long long)nn * (d / 2) + z / 2) * (h / 2) + yy / 2) * (w / 2) + x / 2;
  if (arg[par * C + c] != t) return;
  const long long dst = (i / C) * gx_cs + gx_coff + c;
  gx[dst] = __float2bfloat16_rn((float)gx[dst] + (float)gy[par * gy_cs + c]);
}

// nearest 2x upsampling into channels [0, C) of a view at twice the resolution
__global__ void k_up(const bf16* __restrict__ x, int x_cs, int C, int n, int d, int h, int w, bf16* __restrict__ y,
                     int y_cs) {
  const long long tot = (long long)n * d * h * w * 8 * C;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  long long v = i / C;   // fine voxel
  const int W2 = 2 * w, H2 = 2 * h, D2 = 2 * d;
  const int x2 = (int)(v % W2);
  v /= W2;
  const int y2 = (int)(v % H2);
  v /= H2;
  const int z2 = (int)(v % D2);
  const int nn = (int)(v / D2);
  const long long par = (((long long)nn * d + z2 / 2) * h + y2 / 2) * w + x2 / 2;
  y[(i / C) * y_cs + c] = x[par * x_cs + c];
}

// gradient of the upsampling: g_x[parent] = sum of the 8 children of channels [0, C) of the fine view
__global__ void k_up_bwd(const bf16* __restrict__ gy, int gy_cs, int C, int n, int d, int h, int w,
                         bf16* __restrict__ gx, int gx_cs) {
  const long long tot = (long long)n * d * h * w * C;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  long long v = i / C;
  const int x = (int)(v % w);
  v /= w;
  const int yy = (int)(v % h);
  v /= h;
  const int z = (int)(v % d);
  const int nn = (int)(v / d);
  float s = 0.f;
  for (int t = 0; t < 8; ++t) {
    const long long ch = (((long long)nn * 2 * d + 2 * z + (t >> 2)) * 2 * h + 2 * yy + ((t >> 1) & 1)) * 2 * w + 2 * x +
                         (t & 1);
    s += (float)gy[ch * gy_cs + c];
  }
  gx[(i / C) * gx_cs + c] = __float2bfloat16_rn(s);
}

// masked MSE: loss += sum w (o - t)^2 / sum w (FP64 atomics); g = 2 w (o - t) / sum w as BF16 channels-last
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ tgt, const float* __restrict__ wgt,
                      int C, long long plane, long long nvox, double inv_wsum, double* __restrict__ loss,
                      bf16* __restrict__ g, int g_cs, float* __restrict__ g32) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < nvox * C) {
    const long long n = i / (C * plane), rem = i - n * C * plane;
    const int c = (int)(rem / plane);
    const long long sp = rem - (long long)c * plane;
    const float wv = wgt[n * plane + sp];
    const float dlt = out[i] - tgt[i];
    l = (double)wv * dlt * dlt * inv_wsum;
    const float gv = (float)(2.0 * wv * dlt * inv_wsum);
    if (g) g[(n * plane + sp) * g_cs + c] = __float2bfloat16_rn(gv);
    if (g32) g32[i] = gv;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

__global__ void k_sum(const float* __restrict__ a, long long n, double* __restrict__ out) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Adam on the flat FP32 parameters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// pack w[o][c][tap] (flat FP32) into the forward weights Wf[o][tap * cin_p + c] and the data-gradient
// weights Wd[c][tap' * cout_p + o] = w[o][c][taps - 1 - tap'] (BF16, zero padding)
__global__ void k_pack(const float* __restrict__ w, int cout, int cin, int taps, int cin_p, int cout_p,
                       bf16* __restrict__ wf, int kpad_f, bf16* __restrict__ wd, int kpad_d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)cout * cin * taps) return;
  const int tap = (int)(i % taps);
  const int c = (int)((i / taps) % cin);
  const int o = (int)(i / ((long long)taps * cin));
  const bf16 v = __float2bfloat16_rn(w[i]);
  wf[(long long)o * kpad_f + tap * cin_p + c] = v;
  if (wd) wd[(long long)c * kpad_d + (taps - 1 - tap) * cout_p + o] = v;
}

// gw[k][o] (k = tap * cin_p + c) -> flat gradient g[o][c][tap]
__global__ void k_unpack_grad(const float* __restrict__ gw, int npad, int cout, int cin, int taps, int cin_p,
                              float* __restrict__ g) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)cout * cin * taps) return;
  const int tap = (int)(i % taps);
  const int c = (int)((i / taps) % cin);
  const int o = (int)(i / ((long long)taps * cin));
  g[i] = gw[(long long)(tap * cin_p + c) * npad + o];
}

// --- encodings of the learned initial guess
// max |u| over the velocity blocks and max |p| over the pressure block of a full-layout FP64 vector
__global__ void k_absmax(const double* __restrict__ x, long long nc, int dim, unsigned long long* __restrict__ out) {
  double mu = 0.0, mp = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)(dim + 1) * nc;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(x[i]);
    if (i < (long long)dim * nc) mu = fmax(mu, a);
    else mp = fmax(mp, a);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(mu));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(mp));
  }
}

__global__ void k_features(const uint8_t* __restrict__ mask, const double* __restrict__ xs, long long nc, double U,
                           double Pp, float lre, float* __restrict__ f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  f[i] = mask[i] ? 1.f : 0.f;
  for (int d = 0; d < 3; ++d) f[(1 + d) * nc + i] = (float)(xs[d * nc + i] / U);
  f[4 * nc + i] = (float)(xs[3 * nc + i] / Pp);
  f[5 * nc + i] = lre;
}

__global__ void k_targets(const uint8_t* __restrict__ mask, const double* __restrict__ xn,
                          const double* __restrict__ xs, long long nc, double U, double Pp, float* __restrict__ t,
                          float* __restrict__ w) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  for (int d = 0; d < 3; ++d) t[d * nc + i] = (float)((xn[d * nc + i] - xs[d * nc + i]) / U);
  t[3 * nc + i] = (float)((xn[3 * nc + i] - xs[3 * nc + i]) / Pp);
  if (w) w[i] = mask[i] ? 1.f : 0.f;
}

__global__ void k_proposal(const float* __restrict__ o, const double* __restrict__ xs, long long nc, double U,
                           double Pp, double* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * nc) return;
  const double s = i < 3 * nc ? U : Pp;
  x[i] = xs[i] + s * (double)o[i];
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ================================================================================================ network
struct ConvL {
  int cin, cout, taps;
  int cin_p, cout_p, npad, kpad, npad_d, kpad_d;
  long long woff, boff;           // offsets in the flat parameter vector
  bf16 *wf = nullptr, *wd = nullptr;
  float* gw = nullptr;            // [kpad][npad]
};

struct View {
  bf16* p = nullptr;
  int cs = 0, coff = 0, C = 0;
};

struct pns_unet {
  int L = 0, in_ch = 0, out_ch = 0;
  std::vector<int> ch;
  long long max_vox = 0;
  cudaStream_t s = nullptr;
  std::string err;
  std::vector<ConvL> convs;       // enc0.0, enc0.1, ..., dec{L-2}.0, dec{L-2}.1, ..., dec0.1, head
  long long np = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  long long adam_t = 0;
  std::vector<void*> allocs;
  // activations per level (l = 0 .. L-1) and their gradients
  View feat;                                   // input features (level 0 input)
  std::vector<View> in_, e0, e1, cat, d0, d1;  // in_[l] level input; cat[l] for l < L-1
  std::vector<uint8_t*> arg;                   // pool argmax (l < L-1)
  std::vector<View> g_in, g_e0, g_e1, g_cat, g_d0, g_d1;
  View gout;
  float *out32 = nullptr, *g32 = nullptr;     // output and its gradient of pns_unet_train_step
  double* dsc = nullptr;                       // device scalars (loss, sums)
  unsigned long long* dmax = nullptr;
  int* flag = nullptr;
  int n = 0, d = 0, h = 0, w = 0;              // dims of the last forward
  ~pns_unet() {
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

int fail(pns_unet* U, int code, const std::string& msg, cudaError_t e = cudaSuccess) {
  U->err = msg + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
  return code;
}

#define UCK(expr)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(U, e_ == cudaErrorMemoryAllocation ? PNS_ERR_OOM : PNS_ERR_CUDA, #expr, e_);     \
  } while (0)

template <typename T>
cudaError_t dal(pns_unet* U, T** p, size_t bytes) {
  *p = nullptr;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return e;
  U->allocs.push_back(q);
  e = cudaMemset(q, 0, std::max<size_t>(bytes, 16));
  *p = (T*)q;
  return e;
}

cudaError_t view(pns_unet* U, View& V, int C, long long vox) {
  V.C = C;
  V.cs = r8(C);
  V.coff = 0;
  return dal(U, &V.p, sizeof(bf16) * (size_t)vox * V.cs);
}

size_t conv_smem() { return sizeof(ConvSmem) + 1024; }
size_t wgrad_smem() { return sizeof(WgSmem) + 1024; }

cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem());
  if (e == cudaSuccess) done = true;
  return e;
}

// conv forward (relu) or data gradient (mask) launch
cudaError_t run_conv(pns_unet* U, const View& x, const bf16* wt, int cin_p, int taps, int kpad, int npad, int cout,
                     const float* bias, int relu, const View* mask, const View* y, float* y32) {
  ConvP P;
  P.x = x.p;
  P.x_cs = x.cs;
  P.x_coff = x.coff;
  P.cin_p = cin_p;
  P.taps = taps;
  P.wt = wt;
  P.kpad = kpad;
  P.npad = npad;
  P.cout = cout;
  P.bias = bias;
  P.relu = relu;
  P.mask = mask ? mask->p : nullptr;
  P.m_cs = mask ? mask->cs : 0;
  P.m_coff = mask ? mask->coff : 0;
  P.y = y ? y->p : nullptr;
  P.y_cs = y ? y->cs : 0;
  P.y_coff = y ? y->coff : 0;
  P.y32 = y32;
  P.n = U->n;
  P.d = U->d;
  P.h = U->h;
  P.w = U->w;
  P.flag = U->flag;
  const long long nvox = (long long)P.n * P.d * P.h * P.w;
  pns::count_launch();
  k_conv_tc<<<(unsigned)((nvox + CM - 1) / CM), 128, conv_smem(), U->s>>>(P);
  return cudaGetLastError();
}

}  // namespace

static int forward_impl(pns_unet* U, const float* x, float* out) {
  const int L = U->L;
  const long long plane = (long long)U->d * U->h * U->w;
  const long long nvox0 = U->n * plane;
  pns::count_launch();
  k_to_cl<<<blocks(nvox0 * U->in_ch), 256, 0, U->s>>>(x, U->in_ch, plane, nvox0, U->feat.p, U->feat.cs, 0);
  UCK(cudaGetLastError());
  const int saved_d = U->d, saved_h = U->h, saved_w = U->w;
  auto at_level = [&](int l) {
    U->d = saved_d >> l;
    U->h = saved_h >> l;
    U->w = saved_w >> l;
  };
  int ci = 0;
  for (int l = 0; l < L; ++l) {
    at_level(l);
    const View& in = U->in_[l];
    ConvL& c0 = U->convs[ci++];
    UCK(run_conv(U, in, c0.wf, c0.cin_p, c0.taps, c0.kpad, c0.npad, c0.cout, U->params + c0.boff, 1, nullptr,
                 &U->e0[l], nullptr));
    ConvL& c1 = U->convs[ci++];
    UCK(run_conv(U, U->e0[l], c1.wf, c1.cin_p, c1.taps, c1.kpad, c1.npad, c1.cout, U->params + c1.boff, 1, nullptr,
                 &U->e1[l], nullptr));
    if (l < L - 1) {
      const long long nout = (long long)U->n * (U->d / 2) * (U->h / 2) * (U->w / 2) * U->ch[l];
      pns::count_launch();
      k_pool<<<blocks(nout), 256, 0, U->s>>>(U->e1[l].p, U->e1[l].cs, U->e1[l].coff, U->ch[l], U->n, U->d, U->h,
                                             U->w, U->in_[l + 1].p, U->in_[l + 1].cs, U->arg[l]);
      UCK(cudaGetLastError());
    }
  }
  for (int l = L - 2; l >= 0; --l) {
    at_level(l + 1);
    const View& hs = (l + 1 == L - 1) ? U->e1[L - 1] : U->d1[l + 1];
    const long long nup = (long long)U->n * U->d * U->h * U->w * 8 * U->ch[l + 1];
    pns::count_launch();
    k_up<<<blocks(nup), 256, 0, U->s>>>(hs.p, hs.cs, U->ch[l + 1], U->n, U->d, U->h, U->w, U->cat[l].p,
                                        U->cat[l].cs);
    UCK(cudaGetLastError());
    at_level(l);
    ConvL& a = U->convs[2 * L + 2 * (L - 2 - l)];
    ConvL& b = U->convs[2 * L + 2 * (L - 2 - l) + 1];
    UCK(run_conv(U, U->cat[l], a.wf, a.cin_p, a.taps, a.kpad, a.npad, a.cout, U->params + a.boff, 1, nullptr,
                 &U->d0[l], nullptr));
    UCK(run_conv(U, U->d0[l], b.wf, b.cin_p, b.taps, b.kpad, b.npad, b.cout, U->params + b.boff, 1, nullptr,
                 &U->d1[l], nullptr));
  }
  at_level(0);
  const View& h0 = L > 1 ? U->d1[0] : U->e1[0];
  ConvL& hd = U->convs.back();
  UCK(run_conv(U, h0, hd.wf, hd.cin_p, hd.taps, hd.kpad, hd.npad, hd.cout, U->params + hd.boff, 0, nullptr, nullptr,
               out));
  return PNS_OK;
}

// gradient of one convolution: weights (split-K wgrad), bias, and optionally the data gradient of its input
// masked by (input > 0)
static int conv_backward(pns_unet* U, ConvL& c, const View& x, const View& g, const View* gx) {
  const long long nvox = (long long)U->n * U->d * U->h * U->w;
  WgP P;
  P.x = x.p;
  P.x_cs = x.cs;
  P.x_coff = x.coff;
  P.cin_p = c.cin_p;
  P.taps = c.taps;
  P.g = g.p;
  P.g_cs = g.cs;
  P.g_coff = g.coff;
  P.npad = c.npad;
  P.cout = c.cout;
  P.kreal = c.taps * c.cin_p;
  P.gw = c.gw;
  P.n = U->n;
  P.d = U->d;
  P.h = U->h;
  P.w = U->w;
  P.flag = U->flag;
  const int mt = (P.kreal + CM - 1) / CM;
  // split the voxels so that the grid fills the GPU a few times over
  long long parts = std::max<long long>(1, std::min<long long>((nvox + 1023) / 1024, 2048 / mt));
  P.vchunk = ((nvox + parts - 1) / parts + CK - 1) / CK * CK;
  parts = (nvox + P.vchunk - 1) / P.vchunk;
  pns::count_launch();
  k_wgrad_tc<<<dim3((unsigned)mt, (unsigned)parts), 128, wgrad_smem(), U->s>>>(P);
  UCK(cudaGetLastError());
  const long long chunk = 4096;
  pns::count_launch();
  k_bias_grad<<<blocks(nvox, (int)chunk), 128, 0, U->s>>>(g.p, g.cs, g.coff, c.cout, nvox, chunk,
                                                          U->grads + c.boff);
  UCK(cudaGetLastError());
  if (gx) UCK(run_conv(U, g, c.wd, c.cout_p, c.taps, c.kpad_d, c.npad_d, c.cin, nullptr, 0, &x, gx, nullptr));
  return PNS_OK;
}

static int backward_impl(pns_unet* U, const float* gout32) {
  const int L = U->L;
  const int saved_d = U->d, saved_h = U->h, saved_w = U->w;
  auto at_level = [&](int l) {
    U->d = saved_d >> l;
    U->h = saved_h >> l;
    U->w = saved_w >> l;
  };
  auto restore = [&]() {
    U->d = saved_d;
    U->h = saved_h;
    U->w = saved_w;
  };
  UCK(cudaMemsetAsync(U->grads, 0, sizeof(float) * U->np, U->s));
  for (ConvL& c : U->convs) UCK(cudaMemsetAsync(c.gw, 0, sizeof(float) * (size_t)c.kpad * c.npad, U->s));
  for (int l = 0; l + 1 < L; ++l) {
    at_level(l);
    UCK(cudaMemsetAsync(U->g_cat[l].p, 0, sizeof(bf16) * (size_t)U->n * U->d * U->h * U->w * U->g_cat[l].cs, U->s));
  }
  at_level(0);
  const long long plane = (long long)U->d * U->h * U->w;
  const long long nvox0 = U->n * plane;
  pns::count_launch();
  k_to_cl<<<blocks(nvox0 * U->out_ch), 256, 0, U->s>>>(gout32, U->out_ch, plane, nvox0, U->gout.p, U->gout.cs, 0);
  UCK(cudaGetLastError());
  // head, then the decoder from the top level down
  const View& h0 = L > 1 ? U->d1[0] : U->e1[0];
  View& g_h0 = L > 1 ? U->g_d1[0] : U->g_e1[0];
  int rc = conv_backward(U, U->convs.back(), h0, U->gout, &g_h0);
  if (rc) return rc;
  for (int l = 0; l + 1 < L; ++l) {
    at_level(l);
    ConvL& a = U->convs[2 * L + 2 * (L - 2 - l)];
    ConvL& b = U->convs[2 * L + 2 * (L - 2 - l) + 1];
    if ((rc = conv_backward(U, b, U->d0[l], U->g_d1[l], &U->g_d0[l]))) return rc;
    if ((rc = conv_backward(U, a, U->cat[l], U->g_d0[l], &U->g_cat[l]))) return rc;
    // upsampled part of the concatenation -> gradient of the next level's output
    at_level(l + 1);
    View& g_h = (l + 1 == L - 1) ? U->g_e1[L - 1] : U->g_d1[l + 1];
    const long long n1 = (long long)U->n * U->d * U->h * U->w * U->ch[l + 1];
    pns::count_launch();
    k_up_bwd<<<blocks(n1), 256, 0, U->s>>>(U->g_cat[l].p, U->g_cat[l].cs, U->ch[l + 1], U->n, U->d, U->h, U->w, g_h.p,
                                          g_h.cs);
    UCK(cudaGetLastError());
  }
  // encoder from the bottom level up
  for (int l = L - 1; l >= 0; --l) {
    at_level(l);
    const View& g1 = U->g_e1[l];
    ConvL& c0 = U->convs[2 * l];
    ConvL& c1 = U->convs[2 * l + 1];
    if ((rc = conv_backward(U, c1, U->e0[l], g1, &U->g_e0[l]))) return rc;
    if ((rc = conv_backward(U, c0, U->in_[l], U->g_e0[l], l > 0 ? &U->g_in[l] : nullptr))) return rc;
    if (l > 0) {
      // gradient of the pooled input -> the skip part of the level above (e1[l-1] lives in cat[l-1])
      at_level(l - 1);
      const long long n1 = (long long)U->n * U->d * U->h * U->w * U->ch[l - 1];
      pns::count_launch();
      k_pool_bwd<<<blocks(n1), 256, 0, U->s>>>(U->g_in[l].p, U->g_in[l].cs, U->arg[l - 1], U->ch[l - 1], U->n, U->d,
                                               U->h, U->w, U->g_e1[l - 1].p, U->g_e1[l - 1].cs,
                                               U->g_e1[l - 1].coff);
      UCK(cudaGetLastError());
    }
  }
  restore();
  for (ConvL& c : U->convs) {
    pns::count_launch();
    k_unpack_grad<<<blocks((long long)c.cout * c.cin * c.taps), 256, 0, U->s>>>(c.gw, c.npad, c.cout, c.cin, c.taps,
                                                                                c.cin_p, U->grads + c.woff);
    UCK(cudaGetLastError());
  }
  return PNS_OK;
}

static int pack_all(pns_unet* U) {
  for (ConvL& c : U->convs) {
    pns::count_launch();
    k_pack<<<blocks((long long)c.cout * c.cin * c.taps), 256, 0, U->s>>>(U->params + c.woff, c.cout, c.cin, c.taps,
                                                                         c.cin_p, c.cout_p, c.wf, c.kpad, c.wd,
                                                                         c.kpad_d);
    UCK(cudaGetLastError());
  }
  return PNS_OK;
}

static int check_flag(pns_unet* U) {
  int h = 0;
  UCK(cudaMemcpyAsync(&h, U->flag, sizeof(int), cudaMemcpyDeviceToHost, U->s));
  UCK(cudaStreamSynchronize(U->s));
  if (h & 2) return fail(U, PNS_ERR_TIMEOUT, "a device wait of a tensor-core convolution hit its limit");
  return PNS_OK;
}

static int check_dims(pns_unet* U, int batch, int nz, int ny, int nx) {
  const int q = 1 << (U->L - 1);
  if (batch < 1 || nz < 1 || ny < 1 || nx < 1 || nz % q || ny % q || nx % q)
    return fail(U, PNS_ERR_ARG, "dimensions must be positive multiples of 2^(levels-1)");
  if ((long long)batch * nz * ny * nx > U->max_vox)
    return fail(U, PNS_ERR_ARG, "batch * nz * ny * nx exceeds the size given at creation");
  U->n = batch;
  U->d = nz;
  U->h = ny;
  U->w = nx;
  return PNS_OK;
}

extern "C" {

int pns_unet_create(pns_unet** out, int levels, const int* channels, int in_ch, int out_ch, int batch, int nz, int ny,
                    int nx, uint64_t seed, void* stream) {
  if (!out || !channels || levels < 1 || levels > 5 || in_ch < 1 || in_ch > 128 || out_ch < 1 || out_ch > 128 ||
      batch < 1)
    return PNS_ERR_ARG;
  *out = nullptr;
  const int q = 1 << (levels - 1);
  if (nz < 1 || ny < 1 || nx < 1 || nz % q || ny % q || nx % q) return PNS_ERR_ARG;
  for (int l = 0; l < levels; ++l)
    if (channels[l] < 8 || channels[l] > 128 || channels[l] % 8) return PNS_ERR_ARG;
  for (int l = 0; l + 1 < levels; ++l)
    if (channels[l] + channels[l + 1] > 128) return PNS_ERR_ARG;   // the concatenation feeds an MMA of N <= 128
  pns_unet* U = new (std::nothrow) pns_unet;
  if (!U) return PNS_ERR_OOM;
  U->L = levels;
  U->ch.assign(channels, channels + levels);
  U->in_ch = in_ch;
  U->out_ch = out_ch;
  U->s = (cudaStream_t)stream;
  U->max_vox = (long long)batch * nz * ny * nx;
  int rc = PNS_OK;
  auto bail = [&](int code) {
    delete U;
    return code;
  };
  if (set_attrs() != cudaSuccess) return bail(PNS_ERR_CUDA);
  // convolutions in the flat parameter order
  long long off = 0;
  auto add = [&](int cin, int cout, int taps) {
    ConvL c;
    c.cin = cin;
    c.cout = cout;
    c.taps = taps;
    c.cin_p = r8(cin);
    c.cout_p = r8(cout);
    c.npad = r16(cout);
    c.kpad = r64(taps * c.cin_p);
    c.npad_d = r16(cin);
    c.kpad_d = r64(taps * c.cout_p);
    c.woff = off;
    off += (long long)cout * cin * taps;
    c.boff = off;
    off += cout;
    U->convs.push_back(c);
  };
  int prev = in_ch;
  for (int l = 0; l < levels; ++l) {
    add(prev, channels[l], 27);
    add(channels[l], channels[l], 27);
    prev = channels[l];
  }
  for (int l = levels - 2; l >= 0; --l) {
    add(channels[l + 1] + channels[l], channels[l], 27);
    add(channels[l], channels[l], 27);
  }
  add(channels[0], out_ch, 1);
  U->np = off;
  do {
    if (dal(U, &U->params, sizeof(float) * off) || dal(U, &U->grads, sizeof(float) * off) ||
        dal(U, &U->m, sizeof(float) * off) || dal(U, &U->v, sizeof(float) * off)) {
      rc = PNS_ERR_OOM;
      break;
    }
    for (ConvL& c : U->convs) {
      if (dal(U, &c.wf, sizeof(bf16) * (size_t)c.npad * c.kpad) ||
          dal(U, &c.wd, sizeof(bf16) * (size_t)c.npad_d * c.kpad_d) ||
          dal(U, &c.gw, sizeof(float) * (size_t)c.kpad * c.npad)) {
        rc = PNS_ERR_OOM;
        break;
      }
    }
    if (rc) break;
    U->in_.resize(levels);
    U->e0.resize(levels);
    U->e1.resize(levels);
    U->cat.resize(levels);
    U->d0.resize(levels);
    U->d1.resize(levels);
    U->arg.resize(levels, nullptr);
    U->g_in.resize(levels);
    U->g_e0.resize(levels);
    U->g_e1.resize(levels);
    U->g_cat.resize(levels);
    U->g_d0.resize(levels);
    U->g_d1.resize(levels);
    bool bad = false;
    auto chk = [&](cudaError_t e) { bad = bad || e != cudaSuccess; };
    for (int l = 0; l < levels && !bad; ++l) {
      const long long vox = U->max_vox >> (3 * l);
      const int c = channels[l];
      if (l == 0) {
        chk(view(U, U->feat, in_ch, vox));
        U->in_[0] = U->feat;
      }
      chk(view(U, U->e0[l], c, vox));
      chk(view(U, U->g_e0[l], c, vox));
      if (l < levels - 1) {
        const int cu = channels[l + 1];
        chk(view(U, U->cat[l], cu + c, vox));
        chk(view(U, U->g_cat[l], cu + c, vox));
        U->e1[l] = U->cat[l];
        U->e1[l].coff = cu;
        U->e1[l].C = c;
        U->g_e1[l] = U->g_cat[l];
        U->g_e1[l].coff = cu;
        U->g_e1[l].C = c;
        chk(view(U, U->d0[l], c, vox));
        chk(view(U, U->d1[l], c, vox));
        chk(view(U, U->g_d0[l], c, vox));
        chk(view(U, U->g_d1[l], c, vox));
        chk(dal(U, &U->arg[l], (size_t)(vox / 8) * c));
        chk(view(U, U->in_[l + 1], c, vox / 8));
        chk(view(U, U->g_in[l + 1], c, vox / 8));
      } else {
        chk(view(U, U->e1[l], c, vox));
        chk(view(U, U->g_e1[l], c, vox));
      }
    }
    chk(view(U, U->gout, out_ch, U->max_vox));
    chk(dal(U, &U->out32, sizeof(float) * (size_t)U->max_vox * out_ch));
    chk(dal(U, &U->g32, sizeof(float) * (size_t)U->max_vox * out_ch));
    chk(dal(U, &U->dsc, sizeof(double) * 8));
    chk(dal(U, &U->dmax, sizeof(unsigned long long) * 2));
    chk(dal(U, &U->flag, sizeof(int)));
    if (bad) {
      rc = PNS_ERR_OOM;
      break;
    }
    // He-normal weights, zero biases, a zero head (the untrained network proposes no correction)
    std::vector<float> p(off, 0.f);
    std::mt19937_64 gen(seed);
    for (size_t q = 0; q + 1 < U->convs.size(); ++q) {
      const ConvL& c = U->convs[q];
      std::normal_distribution<float> nd(0.f, std::sqrt(2.0f / (float)(c.cin * c.taps)));
      for (long long i = 0; i < (long long)c.cout * c.cin * c.taps; ++i) p[c.woff + i] = nd(gen);
    }
    if (cudaMemcpy(U->params, p.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = PNS_ERR_CUDA;
      break;
    }
    rc = pack_all(U);
    if (rc) break;
    if (cudaStreamSynchronize(U->s) != cudaSuccess) rc = PNS_ERR_CUDA;
  } while (0);
  if (rc) return bail(rc);
  *out = U;
  return PNS_OK;
}

void pns_unet_destroy(pns_unet* net) { delete net; }

const char* pns_unet_last_error(const pns_unet* net) { return net ? net->err.c_str() : "null network"; }

long long pns_unet_num_params(const pns_unet* net) { return net ? net->np : -1; }

int pns_unet_set_params(pns_unet* U, const float* params) {
  if (!U || !params) return PNS_ERR_ARG;
  UCK(cudaMemcpyAsync(U->params, params, sizeof(float) * U->np, cudaMemcpyHostToDevice, U->s));
  UCK(cudaMemsetAsync(U->m, 0, sizeof(float) * U->np, U->s));
  UCK(cudaMemsetAsync(U->v, 0, sizeof(float) * U->np, U->s));
  U->adam_t = 0;
  int rc = pack_all(U);
  if (rc) return rc;
  UCK(cudaStreamSynchronize(U->s));
  return PNS_OK;
}

int pns_unet_get_params(const pns_unet* net, float* params) {
  if (!net || !params) return PNS_ERR_ARG;
  if (cudaMemcpyAsync(params, net->params, sizeof(float) * net->np, cudaMemcpyDeviceToHost, net->s) != cudaSuccess ||
      cudaStreamSynchronize(net->s) != cudaSuccess)
    return PNS_ERR_CUDA;
  return PNS_OK;
}

int pns_unet_get_grads(const pns_unet* net, float* grads) {
  if (!net || !grads) return PNS_ERR_ARG;
  if (cudaMemcpyAsync(grads, net->grads, sizeof(float) * net->np, cudaMemcpyDeviceToHost, net->s) != cudaSuccess ||
      cudaStreamSynchronize(net->s) != cudaSuccess)
    return PNS_ERR_CUDA;
  return PNS_OK;
}

int pns_unet_forward(pns_unet* U, const float* x, int batch, int nz, int ny, int nx, float* out) {
  if (!U || !x || !out) return PNS_ERR_ARG;
  int rc = check_dims(U, batch, nz, ny, nx);
  if (rc) return rc;
  return forward_impl(U, x, out);
}

int pns_unet_backward(pns_unet* U, const float* gout) {
  if (!U || !gout) return PNS_ERR_ARG;
  if (U->n == 0) return fail(U, PNS_ERR_STATE, "backward before a forward");
  return backward_impl(U, gout);
}

int pns_unet_mse(pns_unet* U, const float* out, const float* target, const float* weight, int batch, int nz, int ny,
                 int nx, float* gout, double* loss) {
  if (!U || !out || !target || !weight || !loss) return PNS_ERR_ARG;
  const long long plane = (long long)nz * ny * nx, nvox = batch * plane;
  UCK(cudaMemsetAsync(U->dsc, 0, sizeof(double) * 2, U->s));
  pns::count_launch();
  k_sum<<<256, 256, 0, U->s>>>(weight, nvox, U->dsc + 1);
  UCK(cudaGetLastError());
  double wsum = 0;
  UCK(cudaMemcpyAsync(&wsum, U->dsc + 1, sizeof(double), cudaMemcpyDeviceToHost, U->s));
  UCK(cudaStreamSynchronize(U->s));
  if (!(wsum > 0)) return fail(U, PNS_ERR_ARG, "the loss weight sums to zero");
  pns::count_launch();
  k_mse<<<blocks(nvox * U->out_ch), 256, 0, U->s>>>(out, target, weight, U->out_ch, plane, nvox,
                                                     1.0 / (wsum * U->out_ch), U->dsc, nullptr, 0, gout);
  UCK(cudaGetLastError());
  UCK(cudaMemcpyAsync(loss, U->dsc, sizeof(double), cudaMemcpyDeviceToHost, U->s));
  UCK(cudaStreamSynchronize(U->s));
  return PNS_OK;
}

int pns_unet_adam(pns_unet* U, float lr, float b1, float b2, float eps) {
  if (!U) return PNS_ERR_ARG;
  U->adam_t += 1;
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)U->adam_t));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)U->adam_t));
  pns::count_launch();
  k_adam<<<blocks(U->np), 256, 0, U->s>>>(U->params, U->grads, U->m, U->v, U->np, lr, b1, b2, eps, c1, c2);
  UCK(cudaGetLastError());
  return pack_all(U);
}

int pns_unet_train_step(pns_unet* U, const float* x, const float* target, const float* weight, int batch, int nz,
                        int ny, int nx, float lr, double* loss) {
  if (!U || !x || !target || !weight || !loss) return PNS_ERR_ARG;
  int rc = check_dims(U, batch, nz, ny, nx);
  if (rc) return rc;
  rc = forward_impl(U, x, U->out32);
  if (!rc) rc = pns_unet_mse(U, U->out32, target, weight, batch, nz, ny, nx, U->g32, loss);
  if (!rc) rc = backward_impl(U, U->g32);
  if (!rc) rc = pns_unet_adam(U, lr, 0.9f, 0.999f, 1e-8f);
  if (!rc) rc = check_flag(U);
  return rc;
}

int pns_unet_features(pns_unet* U, const uint8_t* mask, const double* xs, double re, int nz, int ny, int nx, float* x,
                      int b, double* scales) {
  if (!U || !mask || !xs || !x || b < 0 || !(re > 0) || U->in_ch != 6) return PNS_ERR_ARG;
  const long long nc = (long long)nz * ny * nx;
  UCK(cudaMemsetAsync(U->dmax, 0, sizeof(unsigned long long) * 2, U->s));
  pns::count_launch();
  k_absmax<<<512, 256, 0, U->s>>>(xs, nc, 3, U->dmax);
  UCK(cudaGetLastError());
  unsigned long long hm[2];
  UCK(cudaMemcpyAsync(hm, U->dmax, sizeof hm, cudaMemcpyDeviceToHost, U->s));
  UCK(cudaStreamSynchronize(U->s));
  double Uu, Pp;
  memcpy(&Uu, &hm[0], sizeof(double));
  memcpy(&Pp, &hm[1], sizeof(double));
  Uu = std::max(Uu, 1e-300);
  if (!(Pp > 0)) Pp = 1.0;
  pns::count_launch();
  k_features<<<blocks(nc), 256, 0, U->s>>>(mask, xs, nc, Uu, Pp, (float)std::log10(re), x + (long long)b * 6 * nc);
  UCK(cudaGetLastError());
  if (scales) {
    scales[0] = Uu;
    scales[1] = Pp;
  }
  return PNS_OK;
}

int pns_unet_targets(pns_unet* U, const uint8_t* mask, const double* xn, const double* xs, double us, double ps, int nz,
                     int ny, int nx, float* t, float* w, int b) {
  if (!U || !mask || !xn || !xs || !t || b < 0 || !(us > 0) || !(ps > 0)) return PNS_ERR_ARG;
  const long long nc = (long long)nz * ny * nx;
  pns::count_launch();
  k_targets<<<blocks(nc), 256, 0, U->s>>>(mask, xn, xs, nc, us, ps, t + (long long)b * 4 * nc,
                                          w ? w + (long long)b * nc : nullptr);
  UCK(cudaGetLastError());
  return PNS_OK;
}

int pns_unet_proposal(pns_unet* U, const float* out, int b, const double* xs, double us, double ps, int nz, int ny,
                      int nx, double* x) {
  if (!U || !out || !xs || !x || b < 0 || U->out_ch != 4) return PNS_ERR_ARG;
  const long long nc = (long long)nz * ny * nx;
  pns::count_launch();
  k_proposal<<<blocks(4 * nc), 256, 0, U->s>>>(out + (long long)b * 4 * nc, xs, nc, us, ps, x);
  UCK(cudaGetLastError());
  return PNS_OK;
}

}  // extern "C"
