// pns_precond_apply_static: z = M^{-1} v without any device allocation during the call.
//
// Some callers cannot call cudaMalloc when they apply the preconditioner: code running while
// another component owns the device allocator (a host-side pool or an allocator that must not
// grow), or a caller that has to keep its device footprint fixed after start-up.  This entry point
// runs the same apply body as pns_precond_apply (precond_apply_with), but every scratch vector it
// needs lives in one file-scope device array of fixed size instead of in buffers of the context.
//
// Limits and behaviour:
//  * The array holds STATIC_SCRATCH_BYTES (24 MiB).  One apply takes
//        5 * A(8 * nfull) + A(w * max(prim, dual) packed entries) + R + 2 * A(8 * n_o)
//    bytes of it, with A(x) = x rounded up to 256, w = 8 (FP64) or 4 (FP32/BF16 preconditioners),
//    R = A(8 * max(prim, dual) packed entries) when the local solves are refined, else 0
//    (static_apply_bytes; reported by pns_get_info).  Problems that need more are rejected with
//    PNS_ERR_ARG and a message; the largest full layout that fits is about 500,000 entries.
//  * The array is shared by every call on every context of the process: calls that overlap on the
//    GPU (two streams, or two host threads) race on it.  Serialise such calls.
//  * The device address of the array is taken once per device by static_scratch_init, which
//    pns_setup calls with the context's device current.  The apply itself only reads the address
//    kept in the context.
//  * Every GPU that loads the library holds the array until the process exits.
//  * The preconditioner itself (built by pns_build_precond) lives in the context as before.
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

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int set_err(pns::Ctx& C, int code, const char* msg) {
  C.err = msg;
  return code;
}

}  // namespace

namespace pns {

// Device address of g_static_scratch on the current device, looked up once per device.  In host
// code the array's name is only a host-side stand-in: the device address comes from
// cudaGetSymbolAddress, which also loads this file's module (and with it the array) under lazy
// module loading.
cudaError_t static_scratch_init(void** out) {
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

size_t static_scratch_capacity() { return STATIC_SCRATCH_BYTES; }

size_t static_apply_bytes(const Ctx& C) {
  const Precond& pc = C.pc;
  const size_t pkel = (size_t)std::max<long long>(1, std::max(pc.prim.n_total, pc.dual.n_total));
  const size_t pkb = pkel * (pc.precision == PNS_FP64 ? sizeof(double) : sizeof(float));
  const size_t vb = align256(sizeof(double) * (size_t)C.nfull);
  const size_t zpb = pc.apply_refine ? align256(sizeof(double) * pkel) : 0;
  return 5 * vb + align256(pkb) + zpb + 2 * align256(sizeof(double) * (size_t)std::max(1, pc.n_o));
}

}  // namespace pns

extern "C" int pns_precond_apply_static(pns_ctx* ctx, const double* v, double* z) {
  using namespace pns;
  if (!ctx || !v || !z) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  Precond& pc = C.pc;
  if (!pc.built) return set_err(C, PNS_ERR_STATE, "preconditioner not built");
  if (pc.variant == PNS_BLOCK_SCHUR)
    return set_err(C, PNS_ERR_ARG, "pns_precond_apply_static: not available for the block comparator");
  if (!C.static_scratch) {
    std::string m = "pns_precond_apply_static: no static scratch on this device (" + C.static_err + ")";
    return set_err(C, PNS_ERR_STATE, m.c_str());
  }
  const size_t need = static_apply_bytes(C);
  if (need > STATIC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "pns_precond_apply_static: problem needs %zu bytes of scratch, the static array has %zu",
             need, STATIC_SCRATCH_BYTES);
    return set_err(C, PNS_ERR_ARG, msg);
  }
  const size_t pkel = (size_t)std::max<long long>(1, std::max(pc.prim.n_total, pc.dual.n_total));
  const size_t pkb = pkel * (pc.precision == PNS_FP64 ? sizeof(double) : sizeof(float));
  const size_t vb = align256(sizeof(double) * (size_t)C.nfull);
  const size_t cb = align256(sizeof(double) * (size_t)std::max(1, pc.n_o));
  unsigned char* p = (unsigned char*)C.static_scratch;
  ApplyScratch W;
  W.zG = (double*)p; p += vb;
  W.t1 = (double*)p; p += vb;
  W.zd = (double*)p; p += vb;
  W.t2 = (double*)p; p += vb;
  W.zp = (double*)p; p += vb;
  W.pk = p; p += align256(pkb);
  W.crhs = (double*)p; p += cb;
  W.cx = (double*)p; p += cb;
  W.zpk = pc.apply_refine ? (double*)p : nullptr;
  W.timed = false;   // no CUDA events: the call creates no resource of any kind
  // every vector the body reads is written earlier in the same call (z_G / t1 / z_d / z_p are zeroed
  // or overwritten before use), so the contents left by the previous call do not matter
  return precond_apply_with(C, pc, v, z, W);
}
