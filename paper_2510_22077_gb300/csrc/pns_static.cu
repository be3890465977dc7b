// pns_precond_apply_static: z = M^{-1} v without any device allocation during the call.
//
// Some callers cannot call cudaMalloc when they apply the preconditioner: code running while
// another component owns the device allocator (a host-side pool or an allocator that must not
// grow), or a caller that has to keep its device footprint fixed after start-up.  This entry point
// does exactly what pns_precond_apply does, but every scratch vector it needs lives in one
// file-scope device array of fixed size instead of in buffers of the context.
//
// Limits and behaviour:
//  * The array holds STATIC_SCRATCH_BYTES (24 MiB): five FP64 vectors of the full layout, the packed
//    local vectors of the largest block set and two coarse vectors.  Problems that need more are
//    rejected with PNS_ERR_ARG and a message; the largest full layout that fits is about 500,000
//    entries (a 2D image of ~400 x 400 or a 3D image of ~50^3).
//  * The array is shared by every call on every context of the process: calls that overlap on the
//    GPU (two streams, or two host threads) race on it.  Serialise such calls.
//  * The device address of the array is looked up once per device, on the first call made with that
//    device current; make that first call before any stream capture.
//  * Every GPU that loads the library holds the array until the process exits.
//  * The preconditioner itself (built by pns_build_precond) lives in the context as before.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(24) << 20;
__device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

__global__ void k_sum3_static(const double* __restrict__ a, const double* __restrict__ b,
                              const double* __restrict__ c, double* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = a[i] + b[i] + c[i];
}

int set_err(pns::Ctx& C, int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[400];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "%s", msg);
  C.err = buf;
  return code;
}

#define CKT(expr)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return set_err(C, PNS_ERR_CUDA, #expr, e_);                     \
  } while (0)

}  // namespace

extern "C" int pns_precond_apply_static(pns_ctx* ctx, const double* v, double* z) {
  using namespace pns;
  if (!ctx || !v || !z) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  Precond& pc = C.pc;
  if (!pc.built) return set_err(C, PNS_ERR_STATE, "preconditioner not built");
  if (pc.variant == PNS_BLOCK_SCHUR)
    return set_err(C, PNS_ERR_ARG, "pns_precond_apply_static: not available for the block comparator");
  const long long n = C.nfull;
  const size_t pkel = (size_t)std::max(pc.prim.n_total, pc.dual.n_total);
  const size_t pkb = pkel * (pc.precision == PNS_FP64 ? sizeof(double) : sizeof(float));
  const size_t vb = align256(sizeof(double) * (size_t)n);
  const size_t zpb = pc.apply_refine ? align256(sizeof(double) * std::max<size_t>(1, pkel)) : 0;
  const size_t need = 5 * vb + align256(pkb) + zpb + 2 * align256(sizeof(double) * (size_t)std::max(1, pc.n_o));
  if (need > STATIC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "pns_precond_apply_static: problem needs %zu bytes of scratch, the static array has %zu",
             need, STATIC_SCRATCH_BYTES);
    return set_err(C, PNS_ERR_ARG, msg);
  }
  void* base = nullptr;
  CKT(scratch_address(&base));
  unsigned char* p = (unsigned char*)base;
  double* zG = (double*)p; p += vb;
  double* t1 = (double*)p; p += vb;
  double* zd = (double*)p; p += vb;
  double* t2 = (double*)p; p += vb;
  double* zp = (double*)p; p += vb;
  void* pk = p; p += align256(pkb);
  double* crhs = (double*)p; p += align256(sizeof(double) * (size_t)std::max(1, pc.n_o));
  double* cx = (double*)p; p += align256(sizeof(double) * (size_t)std::max(1, pc.n_o));
  double* zpk = (double*)p;
  const cudaStream_t s = C.stream;
  int op = pc.op;
  const double* st = pc.state.as<double>();
  if (C.opt.combine == PNS_COMBINE_CURRENT && C.cur_state) {
    op = OP_NEWTON;
    st = C.cur_state;
  }
  if (pc.coarse) {
    CKT(launch_seg_sum(pc, v, 1, crhs, s));
    CKT(launch_coarse_gemv<double>(pc.ao_inv.as<double>(), pc.n_o, crhs, cx, s));
    CKT((launch_prolong<double, double>(C, pc, cx, zG)));
    CKT(launch_apply<double>(C, op, st, zG, v, t1, true));
  } else {
    CKT(cudaMemsetAsync(zG, 0, sizeof(double) * n, s));
    CKT(cudaMemcpyAsync(t1, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  CKT(cudaMemsetAsync(zd, 0, sizeof(double) * n, s));
  if (pc.precision == PNS_FP64)
    CKT((launch_local_solve<double, double>(pc.dual, pc.dual.mat.as<double>(), t1, zd, (double*)pk, 1, s)));
  else if (pc.precision == PNS_FP32 && pc.apply_refine)
    CKT((launch_local_solve_refined<float, float>(C, pc.dual, pc.op, pc.state.as<double>(), pc.dual.mat.as<float>(),
                                                  t1, zd, (float*)pk, zpk, 1, s)));
  else if (pc.precision == PNS_FP32)
    CKT((launch_local_solve<float, float>(pc.dual, pc.dual.mat.as<float>(), t1, zd, (float*)pk, 1, s)));
  else if (pc.apply_refine)
    CKT((launch_local_solve_refined<__nv_bfloat16, float>(C, pc.dual, pc.op, pc.state.as<double>(),
                                                          pc.dual.mat.as<__nv_bfloat16>(), t1, zd, (float*)pk, zpk, 1, s)));
  else
    CKT((launch_local_solve<__nv_bfloat16, float>(pc.dual, pc.dual.mat.as<__nv_bfloat16>(), t1, zd, (float*)pk, 1, s)));
  CKT(launch_apply<double>(C, op, st, zd, t1, t2, true));
  CKT(cudaMemsetAsync(zp, 0, sizeof(double) * n, s));
  if (pc.precision == PNS_FP64)
    CKT((launch_local_solve<double, double>(pc.prim, pc.prim.mat.as<double>(), t2, zp, (double*)pk, 0, s)));
  else if (pc.precision == PNS_FP32 && pc.apply_refine)
    CKT((launch_local_solve_refined<float, float>(C, pc.prim, pc.op, pc.state.as<double>(), pc.prim.mat.as<float>(),
                                                  t2, zp, (float*)pk, zpk, 0, s)));
  else if (pc.precision == PNS_FP32)
    CKT((launch_local_solve<float, float>(pc.prim, pc.prim.mat.as<float>(), t2, zp, (float*)pk, 0, s)));
  else if (pc.apply_refine)
    CKT((launch_local_solve_refined<__nv_bfloat16, float>(C, pc.prim, pc.op, pc.state.as<double>(),
                                                          pc.prim.mat.as<__nv_bfloat16>(), t2, zp, (float*)pk, zpk, 0, s)));
  else
    CKT((launch_local_solve<__nv_bfloat16, float>(pc.prim, pc.prim.mat.as<__nv_bfloat16>(), t2, zp, (float*)pk, 0, s)));
  { pns::count_launch(); k_sum3_static<<<2048, 256, 0, s>>>(zG, zd, zp, z, n); }
  CKT(cudaGetLastError());
  return PNS_OK;
}
