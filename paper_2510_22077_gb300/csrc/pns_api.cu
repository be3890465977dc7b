// C ABI of libpns (include/pns.h): context setup, preconditioner build and apply (Secs. 3-4),
// flexible GMRES and Newton (Sec. 8), the Stokes initial iterate.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>

#include "internal.h"

using namespace pns;

#include <atomic>
namespace pns {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace pns

namespace {


int fail(Ctx& C, int code, const char* what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "%s", what);
  C.err = buf;
  return code;
}

#define CK(expr)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(C, e_ == cudaErrorMemoryAllocation ? PNS_ERR_OOM : PNS_ERR_CUDA, #expr, e_);     \
  } while (0)

#define CKS(expr)                     \
  do {                                \
    int s_ = (expr);                  \
    if (s_ != PNS_OK) return s_;      \
  } while (0)

// Device allocation, zero-filled: no buffer of the library is ever read before it is written, but a
// zero fill makes any such mistake deterministic instead of depending on recycled memory.
cudaError_t dalloc(DevBuf& b, size_t bytes) {
  b.release();
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) {
    b.bytes = bytes;
    e = cudaMemset(b.p, 0, bytes);
  } else {
    b.p = nullptr;
  }
  return e;
}

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = dalloc(b, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  e = cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int vt_bytes(int precision) { return precision == PNS_FP64 ? 8 : 4; }
int st_bytes(int precision) { return precision == PNS_FP64 ? 8 : (precision == PNS_FP32 ? 4 : 2); }

// --------------------------------------------------------------------------- block sets
// Binned work list of the persistent local GEMV: blocks in descending size, each cut into items of its
// bin's row count and tagged with its bin's lanes per row (tune[bin] = config id).
int build_gemv_items(Ctx& C, BlockSet& B, const int* tune) {
  std::vector<int> order(B.nblk);
  for (int b = 0; b < B.nblk; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B.n[a] > B.n[b]; });
  std::vector<int4> items;
  for (int b : order) {
    const int cfg = tune[tune_bin(B.n[b])];
    const int R = TUNE_ROWS[cfg], L = TUNE_LANES[cfg];
    for (int r = 0; r < B.n[b]; r += R) items.push_back(make_int4(b, r, std::min(R, B.n[b] - r), L));
  }
  B.nitems_p = (int)items.size();
  if (B.nblk == 0) return PNS_OK;
  CK(upload(B.items_p, items, C.stream));
  if (!B.counter.p) CK(dalloc(B.counter, sizeof(int)));
  return PNS_OK;
}

int make_blockset(Ctx& C, BlockSet& B, const std::vector<std::vector<int>>& lists) {
  B.nblk = (int)lists.size();
  B.n.resize(B.nblk);
  B.ld.resize(B.nblk);
  B.ioff.resize(B.nblk + 1);
  B.moff.resize(B.nblk + 1);
  B.n_total = 0;
  B.m_total = 0;
  B.sum_n2 = 0;
  B.nmax = 0;
  for (int b = 0; b < B.nblk; ++b) {
    int n = (int)lists[b].size();
    int np = (n + 7) / 8 * 8;
    B.n[b] = n;
    B.ld[b] = np;
    B.ioff[b] = B.n_total;
    B.moff[b] = B.m_total;
    B.n_total += np;
    B.m_total += (long long)np * np;
    B.sum_n2 += (double)n * n;
    B.nmax = std::max(B.nmax, n);
  }
  B.ioff[B.nblk] = B.n_total;
  B.moff[B.nblk] = B.m_total;
  std::vector<int> idx(B.n_total, -1);
  for (int b = 0; b < B.nblk; ++b) {
    std::copy(lists[b].begin(), lists[b].end(), idx.begin() + B.ioff[b]);
  }
  std::vector<long long> ioff(B.ioff.begin(), B.ioff.end() - 1), moff(B.moff.begin(), B.moff.end() - 1);
  if (B.nblk == 0) return PNS_OK;
  CK(upload(B.idx, idx, C.stream));
  CK(upload(B.d_n, B.n, C.stream));
  CK(upload(B.d_ld, B.ld, C.stream));
  CK(upload(B.d_ioff, ioff, C.stream));
  CK(upload(B.d_moff, moff, C.stream));
  return build_gemv_items(C, B, C.tune);
}

int op_of_variant(int variant) {
  switch (variant) {
    case PNS_APLMM_NS: return OP_NEWTON;
    case PNS_BLOCK_SCHUR: return OP_NEWTON;
    case PNS_APLMM_S: return OP_STOKES;
    default: return OP_OSEEN;
  }
}

__global__ void k_f2bf(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}
template <typename VT>
__global__ void k_sum3(const VT* __restrict__ a, const VT* __restrict__ b, const VT* __restrict__ c,
                       double* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = (double)a[i] + (double)b[i] + (double)c[i];
}
template <typename VT>
__global__ void k_from_double(const double* __restrict__ v, VT* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (VT)v[i];
}
__global__ void k_negate(const double* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = -a[i];
}
__global__ void k_unit(double* __restrict__ x, int n, int k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (i == k) ? 1.0 : 0.0;
}
__global__ void k_setcol(double* __restrict__ A, int n, int k, const double* __restrict__ col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(long long)i * n + k] = col[i];
}
__global__ void k_unitrow(double* __restrict__ A, int n, int k) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) A[(long long)k * n + j] = (j == k) ? 1.0 : 0.0;
}

// local inverses of one block set in the storage type of `precision`
int to_bf16(Ctx& C, BlockSet& B) {
  DevBuf bf;
  CK(dalloc(bf, sizeof(__nv_bfloat16) * B.m_total));
  { pns::count_launch(); k_f2bf<<<4096, 256, 0, C.stream>>>(B.mat.as<float>(), bf.as<__nv_bfloat16>(), B.m_total); }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(C.stream));
  B.mat.release();
  B.mat.p = bf.p;
  B.mat.bytes = bf.bytes;
  bf.p = nullptr;
  bf.bytes = 0;
  return PNS_OK;
}

// local inverses of one block set; with defer_bf16 the FP32 inverse is kept (converted later)
int build_local(Ctx& C, Precond& pc, BlockSet& B, int* d_bad, bool defer_bf16 = false) {
  if (B.nblk == 0) return PNS_OK;
  const cudaStream_t s = C.stream;
  if (pc.precision == PNS_FP64) {
    CK(dalloc(B.mat, sizeof(double) * B.m_total));
    CK(cudaMemsetAsync(B.mat.p, 0, B.mat.bytes, s));
    CK(launch_assemble<double>(C, B, pc.op, pc.state.as<double>(), B.mat.as<double>(), 0));
    CK(launch_gj_invert<double>(B, B.mat.as<double>(), d_bad, s));
  } else {
    DevBuf& F = B.mat;
    CK(dalloc(F, sizeof(float) * B.m_total));
    CK(cudaMemsetAsync(F.p, 0, F.bytes, s));
    CK(launch_assemble<float>(C, B, pc.op, pc.state.as<double>(), F.as<float>(), 0));
    CK(launch_gj_invert<float>(B, F.as<float>(), d_bad, s, C.opt.timing ? &C.gj : nullptr, C.opt.gj_tensor_cores));
    // Newton-Schulz refinement with FP64 residuals (refine_steps > 0): the FP32 Gauss-Jordan error
    // (~cond * eps32) drops to the FP32 rounding of the exact inverse.  By default the refinement is
    // done in the apply instead (one step of iterative refinement per local solve, pc.apply_refine),
    // which costs a second pass over X per apply rather than a 2 n^3 product per block and build.
    int steps = C.opt.refine_steps > 0 ? C.opt.refine_steps : 0;
    if (steps > 0) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      size_t budget = std::max<size_t>(fr / 2, (size_t)1 << 28);
      double before = 0;
      CK((launch_ns_refine<float, float>(C, B, pc.op, pc.state.as<double>(), 0, F.as<float>(), steps, 1e-5,
                                          budget, &before, nullptr)));
      pc.ns_residual_before = std::max(pc.ns_residual_before, before);
    }
    if (pc.precision == PNS_BF16 && !defer_bf16) CKS(to_bf16(C, B));
  }
  return PNS_OK;
}

// restriction segments: interface cells then primary unknowns
int build_segments(Ctx& C, Precond& pc) {
  const Maps& M = C.M;
  std::vector<int> idx;
  std::vector<long long> off(1, 0);
  std::vector<int2> items;
  auto add_seg = [&](const std::vector<int>& list, bool cells) {
    int sidx = (int)off.size() - 1;
    for (int v : list) idx.push_back(cells ? C.G.dim * C.G.ncell + v : v);
    long long len = (long long)list.size();
    for (long long q = 0; q * 2048 < len; ++q) items.push_back(make_int2(sidx, (int)q));
    off.push_back((long long)idx.size());
  };
  for (int j : M.coarse_ifaces) add_seg(M.iface_cells[j], true);
  for (int i = 0; i < M.n_prim; ++i) add_seg(M.prim_unk[i], false);
  pc.nseg_items = (int)items.size();
  CK(upload(pc.seg_idx, idx, C.stream));
  CK(upload(pc.seg_off, off, C.stream));
  CK(upload(pc.seg_items, items, C.stream));
  return PNS_OK;
}

// shape/correction vectors (closure blocks, Eqs. 6, 9, 15, 17) and the coarse matrix (Remark 1)
template <typename SB>
int build_coarse_t(Ctx& C, Precond& pc, int* d_bad) {
  const Maps& M = C.M;
  const cudaStream_t s = C.stream;
  BlockSet& B = pc.prim;
  // per-primary RHS layout
  std::vector<int> kc(M.n_prim), colbase(M.n_prim), cols, colid, coloff(M.n_prim);
  std::vector<long long> roff(M.n_prim + 1, 0);
  for (int i = 0; i < M.n_prim; ++i) {
    kc[i] = (int)M.C[i].size() + 1;
    colbase[i] = (int)cols.size();
    coloff[i] = (int)colid.size();
    for (int j : M.C[i]) { cols.push_back(j); colid.push_back(M.coarse_of_iface[j]); }
    colid.push_back(pc.n_cif + i);
    roff[i + 1] = roff[i] + (long long)B.n[i] * kc[i];
  }
  pc.kcols = kc;
  pc.boff.assign(roff.begin(), roff.end() - 1);
  DevBuf d_kc, d_colbase, d_cols, d_roff;
  CK(upload(d_kc, kc, s));
  CK(upload(d_colbase, colbase, s));
  CK(upload(d_cols, cols, s));
  std::vector<long long> roffv(roff.begin(), roff.end() - 1);
  CK(upload(d_roff, roffv, s));
  CK(upload(pc.d_kcols, kc, s));
  CK(upload(pc.d_colid, colid, s));
  CK(upload(pc.d_coloff, coloff, s));
  CK(upload(pc.d_boff, roffv, s));
  long long rtot = roff[M.n_prim];
  const double tc0 = now_ms();
  DevBuf rhs, out;
  CK(dalloc(rhs, sizeof(double) * std::max(1LL, rtot)));
  CK(dalloc(out, sizeof(double) * std::max(1LL, rtot)));
  CK(cudaMemsetAsync(rhs.p, 0, rhs.bytes, s));
  CK(launch_closure_rhs(C, B, pc.op, pc.state.as<double>(), d_colbase.as<int>(), d_cols.as<int>(),
                        d_roff.as<long long>(), d_kc.as<int>(), rhs.as<double>()));
  {
    // closure blocks Abar = A_b on p_i plus the row sums of its couplings to f faces and other
    // primary grids (Eqs. 6, 9): solved by the Woodbury identity on the primary-block inverses (the
    // capacitance inverses in the same precision), then iterative refinement with FP64 residuals of Abar:
    // at least two steps, more while the residual norm still falls by 2x per step and is above 1e-14 of
    // the right-hand side's (at most six)
    Woodbury WB;
    CK(WB.setup<SB>(C, B, pc.op, pc.state.as<double>(), B.mat.as<SB>(), kc, d_bad));
    DevBuf Y, res, ds, dn;
    CK(dalloc(Y, sizeof(double) * std::max(1LL, rtot)));
    CK(dalloc(res, sizeof(double) * std::max(1LL, rtot)));
    CK(dalloc(ds, sizeof(double) * std::max(1LL, rtot)));
    CK(dalloc(dn, sizeof(double) * (1 + 1024)));   // the norm, then the dot product's block partials
    CK(WB.apply<SB>(C, B, B.mat.as<SB>(), rhs.as<double>(), out.as<double>(), Y.as<double>(),
                    d_roff.as<long long>(), d_kc.as<int>(), kc));
    auto sq_norm = [&](const double* v, double& out_v) -> cudaError_t {
      cudaError_t e2 = launch_dot(v, v, rtot, dn.as<double>() + 1, dn.as<double>(), s);
      if (e2 != cudaSuccess) return e2;
      e2 = cudaMemcpyAsync(&out_v, dn.p, sizeof(double), cudaMemcpyDeviceToHost, s);
      return e2 != cudaSuccess ? e2 : cudaStreamSynchronize(s);
    };
    double rhs2 = 0, prev2 = -1;
    CK(sq_norm(rhs.as<double>(), rhs2));
    for (int it = 0; it < 6; ++it) {
      CK(launch_closure_residual(C, B, pc.op, pc.state.as<double>(), d_roff.as<long long>(), d_kc.as<int>(),
                                 rhs.as<double>(), out.as<double>(), res.as<double>()));
      double r2 = 0;
      CK(sq_norm(res.as<double>(), r2));
      if (it >= 2 && (r2 <= 1e-28 * rhs2 || (prev2 >= 0 && r2 > 0.25 * prev2))) break;
      prev2 = r2;
      CK(WB.apply<SB>(C, B, B.mat.as<SB>(), res.as<double>(), ds.as<double>(), Y.as<double>(),
                      d_roff.as<long long>(), d_kc.as<int>(), kc));
      CK(launch_add_vec(out.as<double>(), ds.as<double>(), rtot, s));
    }
    CK(cudaStreamSynchronize(s));
  }
  // The basis stays FP64 in every precision (Sum_i n_i (|C_i| + 1) values, ~0.1 GB for a 96^3 pack).
  // The coarse matrix has a near-null mode (the constant interface pressure, pinned through one cell
  // only): rounding the basis to FP32 perturbs A^o by ~1e-7 |A^o|, above its smallest singular value,
  // and the coarse solve then amplifies the rounding along that mode.
  CK(dalloc(pc.basis, sizeof(double) * std::max(1LL, rtot)));
  CK(cudaMemcpyAsync(pc.basis.p, out.p, sizeof(double) * rtot, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  const double tc1 = now_ms();
  // coarse matrix A^o = R^ A_b P^ column by column (prolong e_k, apply A_b, restrict)
  const int no = pc.n_o;
  // A primary grid on which b_B = rho b vanishes (no face unknown along a nonzero component of b) has
  // a zero correction vector, hence a zero column of P^ and of A^o.  It has no coarse unknown: its row
  // and column of A^o are replaced by those of the identity, which leaves the solution of the other
  // coarse unknowns unchanged and multiplies the zero vector in the prolongation.
  std::vector<char> no_source(M.n_prim, 1);
  for (int i = 0; i < M.n_prim; ++i)
    for (int u : M.prim_unk[i])
      if (u < C.G.dim * C.G.ncell && C.P.rho * C.P.b[u / C.G.ncell] != 0.0) {
        no_source[i] = 0;
        break;
      }
  DevBuf Ao, ek, zf, yf, col, work, perm;
  CK(dalloc(Ao, sizeof(double) * (size_t)no * no));
  CK(dalloc(ek, sizeof(double) * no));
  CK(dalloc(zf, sizeof(double) * C.nfull));
  CK(dalloc(yf, sizeof(double) * C.nfull));
  CK(dalloc(col, sizeof(double) * no));
  for (int k = 0; k < no; ++k) {
    if (k >= pc.n_cif && no_source[k - pc.n_cif]) {
      { pns::count_launch(); k_unit<<<(no + 255) / 256, 256, 0, s>>>(col.as<double>(), no, k); }
      { pns::count_launch(); k_setcol<<<(no + 255) / 256, 256, 0, s>>>(Ao.as<double>(), no, k, col.as<double>()); }
      CK(cudaGetLastError());
      continue;
    }
    { pns::count_launch(); k_unit<<<(no + 255) / 256, 256, 0, s>>>(ek.as<double>(), no, k); }
    CK((launch_prolong<double, double>(C, pc, ek.as<double>(), zf.as<double>())));
    CK(launch_apply<double>(C, pc.op, pc.state.as<double>(), zf.as<double>(), nullptr, yf.as<double>(), true));
    CK(launch_seg_sum(pc, yf.p, 1, col.as<double>(), s));
    { pns::count_launch(); k_setcol<<<(no + 255) / 256, 256, 0, s>>>(Ao.as<double>(), no, k, col.as<double>()); }
    CK(cudaGetLastError());
  }
  for (int i = 0; i < M.n_prim; ++i)
    if (no_source[i]) { pns::count_launch(); k_unitrow<<<(no + 255) / 256, 256, 0, s>>>(Ao.as<double>(), no, pc.n_cif + i); }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  const double tc2 = now_ms();
  CK(dalloc(work, sizeof(double) * no));
  CK(dalloc(perm, sizeof(int) * no));
  CK(launch_coarse_invert(Ao.as<double>(), no, work.as<double>(), perm.as<int>(), d_bad, s));
  // the coarse inverse stays FP64 in every precision: it is small (N_o^2 entries) and the coarse
  // matrix can be ill-conditioned (cond ~1e8 on a 96^3 sphere pack), which FP32 storage would ruin
  pc.ao_inv.release();
  pc.ao_inv.p = Ao.p;
  pc.ao_inv.bytes = Ao.bytes;
  Ao.p = nullptr;
  Ao.bytes = 0;
  CK(cudaStreamSynchronize(s));
  C.t_mg_parts[0] = tc1 - tc0;
  C.t_mg_parts[1] = tc2 - tc1;
  C.t_mg_parts[2] = now_ms() - tc2;
  return PNS_OK;
}

int ensure_scratch(Ctx& C, const Precond& pc) {
  const int precision = pc.precision;
  size_t vb = sizeof(double) * C.nfull;
  DevBuf* ws[5] = {&C.w0, &C.w1, &C.w2, &C.w3, &C.w4};
  for (DevBuf* w : ws)
    if (w->bytes < vb) CK(dalloc(*w, vb));
  long long pk = std::max(pc.prim.n_total, pc.dual.n_total);
  size_t pb = (size_t)vt_bytes(precision) * std::max(1LL, pk);
  if (C.pk_x.bytes < pb) CK(dalloc(C.pk_x, pb));
  if (pc.apply_refine) {
    size_t zb = sizeof(double) * std::max(1LL, pk);
    if (C.zpk.bytes < zb) CK(dalloc(C.zpk, zb));
  }
  size_t cb = sizeof(double) * std::max(1, pc.n_o);
  if (C.coarse_rhs.bytes < cb) CK(dalloc(C.coarse_rhs, cb));
  if (C.coarse_x.bytes < cb) CK(dalloc(C.coarse_x, cb));
  return PNS_OK;
}

// --------------------------------------------------------------------------- block comparator
// Block-triangular Schur-complement preconditioner (Sec. 1, M_B with the scaled BFBt X of Eq. 4).
// Pore partition: a face unknown belongs to the pore of the cell on its high side (the cell that
// stores it), a cell to its own pore; pinned cells are left out of L.
template <typename ST>
int build_block_t(Ctx& C, Precond& pc, int* d_bad) {
  BlockSchurData& S = pc.bs;
  const cudaStream_t s = C.stream;
  const Maps& M = C.M;
  const int nc = C.G.ncell, dim = C.G.dim;
  int maxlab = 0;
  for (int c = 0; c < nc; ++c) maxlab = std::max(maxlab, M.label[c]);
  std::vector<int> pid(maxlab + 1, -1);
  int np = 0;
  for (int c = 0; c < nc; ++c)
    if ((M.flags[c] & FL_VOID) && pid[M.label[c]] < 0) pid[M.label[c]] = np++;
  std::vector<std::vector<int>> lf(np), lc(np);
  for (int d = 0; d < dim; ++d)
    for (int c = 0; c < nc; ++c)
      if (M.flags[c] & fl_face(d)) lf[pid[M.label[c]]].push_back(d * nc + c);
  for (int c = 0; c < nc; ++c)
    if ((M.flags[c] & FL_VOID) && !(M.flags[c] & FL_PIN)) lc[pid[M.label[c]]].push_back(dim * nc + c);
  auto drop_empty = [](std::vector<std::vector<int>>& l) {
    l.erase(std::remove_if(l.begin(), l.end(), [](const std::vector<int>& v) { return v.empty(); }), l.end());
  };
  drop_empty(lf);
  drop_empty(lc);
  CKS(make_blockset(C, S.bf, lf));
  CKS(make_blockset(C, S.bl, lc));
  CK(dalloc(S.D, sizeof(double) * C.nfull));
  CK(launch_diag_F(C, OP_NEWTON, pc.state.as<double>(), S.D.as<double>()));
  if (S.bf.nblk) {
    CK(dalloc(S.bf.mat, sizeof(ST) * S.bf.m_total));
    CK(launch_assemble<ST>(C, S.bf, OP_NEWTON, pc.state.as<double>(), S.bf.mat.as<ST>(), 0));
    CK(launch_gj_invert<ST>(S.bf, S.bf.mat.as<ST>(), d_bad, s, nullptr, C.opt.gj_tensor_cores));
  }
  if (S.bl.nblk) {
    CK(dalloc(S.bl.mat, sizeof(ST) * S.bl.m_total));
    CK(launch_assemble_L<ST>(C, S.bl, S.D.as<double>(), S.bl.mat.as<ST>()));
    CK(launch_gj_invert<ST>(S.bl, S.bl.mat.as<ST>(), d_bad, s, nullptr, C.opt.gj_tensor_cores));
  }
  S.its = C.opt.block_inner_its;
  S.tol = C.opt.block_inner_tol;
  const size_t vb = sizeof(double) * C.nfull;
  CK(dalloc(S.V, vb * (S.its + 1)));
  CK(dalloc(S.Z, vb * S.its));
  CK(dalloc(S.H, sizeof(double) * (S.its + 1) * S.its));
  CK(dalloc(S.small, sizeof(double) * (7 * (S.its + 1) + 8)));
  CK(dalloc(S.partial, sizeof(double) * 1024 * (S.its + 2)));
  for (DevBuf* t : {&S.t1, &S.t2, &S.t3, &S.t4, &S.t5}) CK(dalloc(*t, vb));
  CK(dalloc(S.pk, sizeof(ST) * std::max(1LL, std::max(S.bf.n_total, S.bl.n_total))));
  S.inner_total = 0;
  return PNS_OK;
}

int build_block(Ctx& C, Precond& pc) {
  DevBuf bad;
  CK(dalloc(bad, sizeof(int)));
  double t0 = now_ms();
  if (pc.precision == PNS_FP64) CKS(build_block_t<double>(C, pc, bad.as<int>()));
  else CKS(build_block_t<float>(C, pc, bad.as<int>()));
  CK(cudaStreamSynchronize(C.stream));
  C.t_ml_ms = now_ms() - t0;
  C.t_mg_ms = 0;
  int hbad = 0;
  CK(cudaMemcpy(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (hbad & 2) return fail(C, PNS_ERR_TIMEOUT, "a device wait of the tensor-core Gauss-Jordan update hit its limit");
  if (hbad) return fail(C, PNS_ERR_SINGULAR, "zero or non-finite pivot in a block-Jacobi factor");
  pc.local_bytes = 0;
  for (BlockSet* B : {&pc.bs.bf, &pc.bs.bl})
    for (int b = 0; b < B->nblk; ++b)
      pc.local_bytes += (double)B->n[b] * B->ld[b] * (pc.precision == PNS_FP64 ? 8 : 4) + 20.0 * B->n[b];
  pc.built = true;
  return PNS_OK;
}

// z = M^{-1} r by block Jacobi over one block set of the comparator (z zero outside the set)
int block_jacobi(Ctx& C, Precond& pc, const BlockSet& B, const double* r, double* z) {
  CK(cudaMemsetAsync(z, 0, sizeof(double) * C.nfull, C.stream));
  if (B.nblk == 0) return PNS_OK;
  if (pc.precision == PNS_FP64)
    CK((launch_local_solve<double, double>(B, B.mat.as<double>(), r, z, pc.bs.pk.as<double>(), 0, C.stream)));
  else
    CK((launch_local_solve<float, float>(B, B.mat.as<float>(), r, z, pc.bs.pk.as<float>(), 0, C.stream)));
  return PNS_OK;
}

// y = F v (faces; the cell block of v is zero, the cell block of y is zeroed)
int block_opF(Ctx& C, Precond& pc, const double* v, double* y) {
  CK(launch_apply<double>(C, OP_NEWTON, pc.state.as<double>(), v, nullptr, y, true));
  CK(launch_zero_cells(C, y));
  return PNS_OK;
}

// y = L v = B2 D^{-1} B1 v on the cells that are not pinned
int block_opL(Ctx& C, Precond& pc, const double* v, double* y) {
  double* t = pc.bs.t5.as<double>();
  CK(launch_grad(C, v, pc.bs.D.as<double>(), nullptr, 0, t));
  CK(launch_div(C, t, nullptr, 1.0, y));
  return PNS_OK;
}

// Inner GMRES (FP64 vectors, classical Gram-Schmidt twice, no restart): x ~ A^{-1} b with block
// Jacobi on the right; stops after S.its iterations or at ||b - A x|| <= S.tol ||b||.
int block_gmres(Ctx& C, Precond& pc, int which, const double* b, double* x) {
  BlockSchurData& S = pc.bs;
  const cudaStream_t s = C.stream;
  const long long n = C.nfull;
  const int m = S.its;
  double* V = S.V.as<double>();
  double* Z = S.Z.as<double>();
  double* H = S.H.as<double>();
  double* cs = S.small.as<double>();
  double* sn = cs + (m + 1);
  double* g = sn + (m + 1);
  double* outv = g + (m + 1);
  double* h1 = outv + 8;
  double* h2 = h1 + (m + 1);
  double* yv = h2 + (m + 1);
  double* nrm = yv + (m + 1);
  double* partial = S.partial.as<double>();
  const BlockSet& B = which == 0 ? S.bf : S.bl;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  CK(launch_dot(b, b, n, partial, nrm, s));
  double beta2 = 0;
  CK(cudaMemcpyAsync(&beta2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double beta = std::sqrt(beta2);
  if (!std::isfinite(beta)) return fail(C, PNS_ERR_NAN, "non-finite vector in the block comparator");
  if (beta == 0.0) return PNS_OK;
  const double tol_abs = S.tol * beta;
  std::vector<double> gh(m + 1, 0.0);
  gh[0] = beta;
  CK(cudaMemcpyAsync(g, gh.data(), sizeof(double) * (m + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)(m + 1) * m, s));
  CK(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  const double binv = 1.0 / beta;
  CK(cudaMemcpyAsync(nrm, &binv, sizeof(double), cudaMemcpyHostToDevice, s));
  CK(launch_scale(V, n, nrm, nullptr, 0, s));
  int k = 0;
  for (int j = 0; j < m; ++j) {
    double* vj = V + (size_t)j * n;
    double* zj = Z + (size_t)j * n;
    double* w = V + (size_t)(j + 1) * n;
    CKS(block_jacobi(C, pc, B, vj, zj));
    if (which == 0) CKS(block_opF(C, pc, zj, w));
    else CKS(block_opL(C, pc, zj, w));
    CK(launch_multidot(V, n, j + 1, w, n, partial, 0, h1, s));
    CK(launch_multi_axpy(w, V, n, j + 1, h1, -1.0, n, s));
    CK(launch_multidot(V, n, j + 1, w, n, partial, 0, h2, s));
    CK(launch_multi_axpy(w, V, n, j + 1, h2, -1.0, n, s));
    CK(launch_dot(w, w, n, partial, nrm, s));
    CK(launch_hcol(H, m, j, h1, h2, nrm, s));
    CK(launch_scale(w, n, nullptr, nrm, 1, s));
    CK(launch_givens(H, m, cs, sn, g, j, outv, s));
    double hres[2];
    CK(cudaMemcpyAsync(hres, outv, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    k = j + 1;
    S.inner_total++;
    if (!std::isfinite(hres[0])) return fail(C, PNS_ERR_NAN, "non-finite residual in the block comparator");
    if (hres[0] <= tol_abs) break;
  }
  CK(launch_trisolve_update(H, m, g, k, yv, Z, n, x, n, s));
  return PNS_OK;
}

// z = M_B^{-1} v:  y = X^{-1} v_p (pins: y = v),  u = F^{-1} (v_u - B1 y),  z = [u; y]
int block_apply(Ctx& C, Precond& pc, const double* v, double* z) {
  BlockSchurData& S = pc.bs;
  double *t1 = S.t1.as<double>(), *t2 = S.t2.as<double>(), *t3 = S.t3.as<double>(), *t4 = S.t4.as<double>();
  double* t5 = S.t5.as<double>();
  const double* D = S.D.as<double>();
  CK(launch_compose(C, v, nullptr, 0, t1));                    // v on the cells that are not pinned
  CKS(block_gmres(C, pc, 1, t1, t2));                          // t2 = L^{-1} v_n
  CK(launch_grad(C, t2, D, nullptr, 0, t3));                   // t3 = D^{-1} B1 t2
  CK(launch_apply<double>(C, OP_NEWTON, pc.state.as<double>(), t3, nullptr, t4, true));   // F t3 (faces)
  CK(launch_div(C, t4, D, 1.0, t1));                           // t1 = B2 D^{-1} F D^{-1} B1 t2
  CKS(block_gmres(C, pc, 1, t1, t2));                          // t2 = L^{-1} t1 = -y_n
  CK(launch_compose(C, v, t2, 1, t3));                         // t3 = y (pins: v)
  CK(launch_grad(C, t3, nullptr, v, 1, t1));                   // t1 = v_u - B1 y
  CKS(block_gmres(C, pc, 0, t1, t4));                          // t4 = F^{-1} t1
  (void)t5;
  CK(launch_compose(C, t4, t3, 2, z));                         // z = [t4; t3]
  return PNS_OK;
}

int build_precond(Ctx& C, Precond& pc, int variant, const double* x_lin) {
  const cudaStream_t s = C.stream;
  ++C.n_builds;
  if (&pc == &C.pc) C.solves_since_build = 0;
  pc.built = false;
  pc.ns_residual_before = 0;
  pc.variant = variant;
  pc.precision = C.opt.precision;
  pc.apply_refine = pc.precision != PNS_FP64 && C.opt.refine_steps < 0;
  pc.op = op_of_variant(variant);
  pc.coarse = variant != PNS_ML_ONLY;
  pc.n_cif = (int)C.M.coarse_ifaces.size();
  pc.n_o = pc.n_cif + C.M.n_prim;
  CK(dalloc(pc.state, sizeof(double) * C.nfull));
  if (x_lin) CK(cudaMemcpyAsync(pc.state.p, x_lin, sizeof(double) * C.nfull, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(pc.state.p, 0, sizeof(double) * C.nfull, s));
  if (variant == PNS_BLOCK_SCHUR) {
    pc.coarse = false;
    pc.n_o = 0;
    return build_block(C, pc);
  }
  if (pc.prim.nblk != C.M.n_prim || pc.prim.idx.p == nullptr) CKS(make_blockset(C, pc.prim, C.M.prim_unk));
  if (pc.dual.nblk != C.M.n_iface || (C.M.n_iface && pc.dual.idx.p == nullptr)) CKS(make_blockset(C, pc.dual, C.M.dual_unk));
  CKS(build_segments(C, pc));
  DevBuf bad;
  CK(dalloc(bad, sizeof(int)));
  CK(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  double t0 = now_ms();
  CKS(build_local(C, pc, pc.prim, bad.as<int>(), true));
  CKS(build_local(C, pc, pc.dual, bad.as<int>()));
  CK(cudaStreamSynchronize(s));
  double t1 = now_ms();
  C.t_ml_ms = t1 - t0;
  if (pc.coarse) {
    if (pc.precision == PNS_FP64) CKS(build_coarse_t<double>(C, pc, bad.as<int>()));
    else CKS(build_coarse_t<float>(C, pc, bad.as<int>()));
  }
  if (pc.precision == PNS_BF16) CKS(to_bf16(C, pc.prim));
  C.t_mg_ms = now_ms() - t1;
  int hbad = 0;
  CK(cudaMemcpy(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (hbad & 2) return fail(C, PNS_ERR_TIMEOUT, "a device wait of the tensor-core Gauss-Jordan update hit its limit");
  if (hbad) return fail(C, PNS_ERR_SINGULAR, "zero or non-finite pivot in a local or coarse factor");
  pc.ns_residual_before = pc.ns_residual_before;
  pc.local_bytes = 0;
  for (BlockSet* B : {&pc.prim, &pc.dual})
    for (int b = 0; b < B->nblk; ++b)
      pc.local_bytes += (pc.apply_refine ? 2.0 : 1.0) * B->n[b] * B->ld[b] * st_bytes(pc.precision) +  // inverse
                        (pc.apply_refine ? 60.0 : 20.0) * B->n[b];   // t, z, index (and the refinement vectors)
  CKS(ensure_scratch(C, pc));
  pc.built = true;
  return PNS_OK;
}

template <typename ST, typename PT>
int local_solve(Ctx& C, Precond& pc, BlockSet& B, const double* t, double* z, int add, const ApplyScratch& W) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (W.timed) {
    if (C.ev_used + 2 > C.ev_pool.size()) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      C.ev_pool.push_back(a);
      C.ev_pool.push_back(b);
    }
    e0 = C.ev_pool[C.ev_used];
    e1 = C.ev_pool[C.ev_used + 1];
    C.ev_used += 2;
    CK(cudaEventRecord(e0, C.stream));
  }
  PT* pk = (PT*)W.pk;
  if constexpr (!std::is_same<ST, double>::value) {
    if (pc.apply_refine) {
      CK((launch_local_solve_refined<ST, PT>(C, B, pc.op, pc.state.as<double>(), B.mat.as<ST>(), t, z, pk, W.zpk,
                                             add, C.stream)));
    } else {
      CK((launch_local_solve<ST, PT>(B, B.mat.as<ST>(), t, z, pk, add, C.stream)));
    }
  } else {
    CK((launch_local_solve<ST, PT>(B, B.mat.as<ST>(), t, z, pk, add, C.stream)));
  }
  if (W.timed) {
    CK(cudaEventRecord(e1, C.stream));
    C.local_launches += 1;
  }
  return PNS_OK;
}

}  // namespace

// z = M^{-1} v.  The local inverses, basis and coarse inverse are stored in the preconditioner's
// precision and the batched local solves compute in it; the vectors between the stages and the two
// stencil residual updates (v - A z_G, t - A z_d) are FP64: those differences cancel strongly when
// z_G is large (ill-conditioned coarse systems), and in FP32 their error would scale with |A z_G|.
int pns::precond_apply_with(Ctx& C, Precond& pc, const double* v, double* z, const ApplyScratch& W) {
  const cudaStream_t s = C.stream;
  const long long n = C.nfull;
  double *zG = W.zG, *t1 = W.t1, *zd = W.zd, *t2 = W.t2, *zp = W.zp;
  int op = pc.op;
  const double* st = pc.state.as<double>();
  if (C.opt.combine == PNS_COMBINE_CURRENT && C.cur_state) {
    op = OP_NEWTON;
    st = C.cur_state;
  }
  if (pc.coarse) {
    CK(launch_seg_sum(pc, v, 1, W.crhs, s));
    CK(launch_coarse_gemv<double>(pc.ao_inv.as<double>(), pc.n_o, W.crhs, W.cx, s));
    CK((launch_prolong<double, double>(C, pc, W.cx, zG)));
    CK(launch_apply<double>(C, op, st, zG, v, t1, true));           // t1 = v - A z_G
  } else {
    CK(cudaMemsetAsync(zG, 0, sizeof(double) * n, s));
    CK(cudaMemcpyAsync(t1, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaMemsetAsync(zd, 0, sizeof(double) * n, s));
  if (pc.precision == PNS_FP64) CKS((local_solve<double, double>(C, pc, pc.dual, t1, zd, 1, W)));
  else if (pc.precision == PNS_FP32) CKS((local_solve<float, float>(C, pc, pc.dual, t1, zd, 1, W)));
  else CKS((local_solve<__nv_bfloat16, float>(C, pc, pc.dual, t1, zd, 1, W)));
  CK(launch_apply<double>(C, op, st, zd, t1, t2, true));             // t2 = t1 - A z_d
  CK(cudaMemsetAsync(zp, 0, sizeof(double) * n, s));
  if (pc.precision == PNS_FP64) CKS((local_solve<double, double>(C, pc, pc.prim, t2, zp, 0, W)));
  else if (pc.precision == PNS_FP32) CKS((local_solve<float, float>(C, pc, pc.prim, t2, zp, 0, W)));
  else CKS((local_solve<__nv_bfloat16, float>(C, pc, pc.prim, t2, zp, 0, W)));
  { pns::count_launch(); k_sum3<double><<<2048, 256, 0, s>>>(zG, zd, zp, z, n); }
  CK(cudaGetLastError());
  return PNS_OK;
}

namespace {

int precond_apply(Ctx& C, Precond& pc, const double* v, double* z) {
  if (!pc.built) return fail(C, PNS_ERR_STATE, "preconditioner not built");
  if (pc.variant == PNS_BLOCK_SCHUR) return block_apply(C, pc, v, z);
  ApplyScratch W;
  W.zp = C.w0.as<double>();
  W.zG = C.w1.as<double>();
  W.t1 = C.w2.as<double>();
  W.zd = C.w3.as<double>();
  W.t2 = C.w4.as<double>();
  W.pk = C.pk_x.p;
  W.zpk = C.zpk.as<double>();
  W.crhs = C.coarse_rhs.as<double>();
  W.cx = C.coarse_x.as<double>();
  W.timed = C.opt.timing != 0;
  return precond_apply_with(C, pc, v, z, W);
}

// --------------------------------------------------------------------------- Krylov
int ensure_krylov(Ctx& C, int m) {
  if (C.m_alloc >= m) return PNS_OK;
  CK(dalloc(C.V, sizeof(double) * (size_t)(m + 1) * C.nfull));
  CK(dalloc(C.Z, sizeof(double) * (size_t)m * C.nfull));
  CK(dalloc(C.H, sizeof(double) * (size_t)(m + 1) * m));
  CK(dalloc(C.givens, sizeof(double) * (3 * (m + 1) + 8)));
  CK(dalloc(C.hvec, sizeof(double) * 4 * (m + 1)));
  CK(dalloc(C.partial, sizeof(double) * 1024 * (m + 2)));
  C.m_alloc = m;
  return PNS_OK;
}

double host_norm(Ctx& C, const double* a, int& st) {
  double* out = C.hvec.as<double>() + 3 * (C.m_alloc + 1);
  cudaError_t e = launch_dot(a, a, C.nfull, C.partial.as<double>(), out, C.stream);
  double h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, C.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(C.stream);
  st = e == cudaSuccess ? PNS_OK : fail(C, PNS_ERR_CUDA, "norm", e);
  return std::sqrt(h);
}

void harvest_events(Ctx& C);

// Solve J(op, state) dx = b with right-preconditioned FGMRES(m); dx is overwritten.
int fgmres(Ctx& C, Precond& pc, int op, const double* state, const double* b, double* dx, double tol_abs, int maxit,
           int& its_out, double& res_out) {
  const cudaStream_t s = C.stream;
  const long long n = C.nfull;
  const int m = std::max(1, C.opt.restart);
  CKS(ensure_krylov(C, m));
  double* V = C.V.as<double>();
  double* Z = C.Z.as<double>();
  double* H = C.H.as<double>();
  double* cs = C.givens.as<double>();
  double* sn = cs + (m + 1);
  double* g = sn + (m + 1);
  double* outv = g + (m + 1);
  double* h1 = C.hvec.as<double>();
  double* h2 = h1 + (m + 1);
  double* yv = h2 + (m + 1);
  double* nrm = yv + (m + 1);
  CK(cudaMemsetAsync(dx, 0, sizeof(double) * n, s));
  double* r = V;   // the residual lives in V_0 before normalisation
  CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  int st = 0;
  double beta = host_norm(C, r, st);
  CKS(st);
  int its = 0;
  while (beta > tol_abs && its < maxit) {
    if (!std::isfinite(beta)) return fail(C, PNS_ERR_NAN, "non-finite residual in FGMRES");
    // V_0 = r / beta ; g = [beta, 0, ...]
    std::vector<double> gh(m + 1, 0.0);
    gh[0] = beta;
    CK(cudaMemcpyAsync(g, gh.data(), sizeof(double) * (m + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)(m + 1) * m, s));
    double binv = 1.0 / beta;
    CK(cudaMemcpyAsync(nrm, &binv, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_scale(V, n, nrm, nullptr, 0, s));
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      CKS(precond_apply(C, pc, vj, zj));
      CK(launch_apply<double>(C, op, state, zj, nullptr, w, true));
      // CGS2
      CK(launch_multidot(V, n, j + 1, w, n, C.partial.as<double>(), 0, h1, s));
      CK(launch_multi_axpy(w, V, n, j + 1, h1, -1.0, n, s));
      CK(launch_multidot(V, n, j + 1, w, n, C.partial.as<double>(), 0, h2, s));
      CK(launch_multi_axpy(w, V, n, j + 1, h2, -1.0, n, s));
      CK(launch_dot(w, w, n, C.partial.as<double>(), nrm, s));
      CK(launch_hcol(H, m, j, h1, h2, nrm, s));
      CK(launch_scale(w, n, nullptr, nrm, 1, s));
      CK(launch_givens(H, m, cs, sn, g, j, outv, s));
      double hres[2];
      CK(cudaMemcpyAsync(hres, outv, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (C.ev_used >= 256) harvest_events(C);
      ++its;
      k = j + 1;
      if (!std::isfinite(hres[0])) return fail(C, PNS_ERR_NAN, "non-finite Givens residual");
      res_out = hres[0];
      if (hres[0] <= tol_abs || its >= maxit) break;
    }
    CK(launch_trisolve_update(H, m, g, k, yv, Z, n, dx, n, s));
    // true residual for the restart: r = b - J dx
    CK(launch_apply<double>(C, op, state, dx, b, r, true));
    beta = host_norm(C, r, st);
    CKS(st);
    res_out = beta;
  }
  its_out = its;
  return PNS_OK;
}

// Sum the local-solve event pairs recorded since the last harvest (the stream has synchronised).
void harvest_events(Ctx& C) {
  for (size_t k = 0; k + 1 < C.ev_used; k += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, C.ev_pool[k], C.ev_pool[k + 1]) == cudaSuccess) C.t_local_ms += ms;
  }
  C.ev_used = 0;
}

int newton(Ctx& C, Precond& pc, int stokes, double* x, const double* x_prev, pns_stats* stt) {
  const cudaStream_t s = C.stream;
  const long long n = C.nfull;
  CK(dalloc(C.rk, sizeof(double) * n));
  CK(dalloc(C.dx, sizeof(double) * n));
  CK(dalloc(C.xk, sizeof(double) * n));
  CKS(ensure_krylov(C, std::max(1, C.opt.restart)));
  // ||r(0)||
  CK(cudaMemsetAsync(C.xk.p, 0, sizeof(double) * n, s));
  CK(launch_residual(C, stokes, C.xk.as<double>(), nullptr, C.rk.as<double>()));
  int st = 0;
  double r0 = host_norm(C, C.rk.as<double>(), st);
  CKS(st);
  if (!(r0 > 0)) r0 = 1.0;
  pns_stats loc;
  memset(&loc, 0, sizeof loc);
  loc.r0_norm = r0;
  int op = stokes ? OP_STOKES : OP_NEWTON;
  int maxn = C.opt.max_newton;
  int code = PNS_OK;
  double tsol = 0;
  for (int k = 0;; ++k) {
    CK(launch_residual(C, stokes, x, x_prev, C.rk.as<double>()));
    double nr = host_norm(C, C.rk.as<double>(), st);
    CKS(st);
    double rel = nr / r0;
    if (k < 65) loc.res_hist[k] = rel;
    if (!std::isfinite(rel)) { code = fail(C, PNS_ERR_NAN, "non-finite Newton residual"); break; }
    if (rel < C.opt.newton_tol) break;
    if (k >= maxn) { code = fail(C, PNS_ERR_NOT_CONVERGED, "Newton iteration cap reached"); break; }
    { pns::count_launch(); k_negate<<<2048, 256, 0, s>>>(C.rk.as<double>(), C.rk.as<double>(), n); }
    CK(cudaGetLastError());
    C.cur_state = stokes ? nullptr : x;
    double t0 = now_ms();
    int its = 0;
    double res = 0;
    int fs = fgmres(C, pc, op, x, C.rk.as<double>(), C.dx.as<double>(), C.opt.inner_tol * r0, C.opt.max_fgmres, its,
                    res);
    tsol += now_ms() - t0;
    if (fs != PNS_OK) { code = fs; break; }
    if (loc.newton_its < 64) loc.fgmres_its[loc.newton_its] = its;
    loc.newton_its++;
    loc.fgmres_its_total += its;
    CK(launch_axpy(x, C.dx.as<double>(), 1.0, n, s));
  }
  C.cur_state = nullptr;
  CK(cudaStreamSynchronize(s));
  harvest_events(C);
  loc.t_sol_ms = tsol;
  loc.t_setup_ms = C.t_setup_ms;
  loc.t_mg_ms = C.t_mg_ms;
  for (int q = 0; q < 3; ++q) loc.t_mg_parts_ms[q] = C.t_mg_parts[q];
  loc.t_ml_ms = C.t_ml_ms;
  loc.t_local_ms = C.t_local_ms;
  loc.local_launches = C.local_launches;
  loc.local_bytes_per_apply = pc.local_bytes;
  loc.kernel_launches = launch_count();
  loc.refine_residual_max = pc.ns_residual_before;
  loc.t_gj_update_ms = C.gj.ms;
  loc.gj_update_flops = C.gj.flops;
  loc.gj_update_bytes = C.gj.bytes;
  loc.precond_builds = C.n_builds;
  loc.gj_update_launches = C.gj.launches;
  loc.gj_update_tiles = C.gj.tiles;
  if (stt) *stt = loc;
  return code;
}

void export_maps(const Maps& M, const Geo& G, int32_t* cell_prim, int32_t* cell_iface, int32_t* face_class,
                 uint8_t* tags, int32_t* dual_count, int32_t* pins) {
  const int nc = G.ncell, dim = G.dim;
  if (cell_prim) std::copy(M.cell_prim.begin(), M.cell_prim.end(), cell_prim);
  if (cell_iface) std::copy(M.cell_iface.begin(), M.cell_iface.end(), cell_iface);
  if (face_class) std::copy(M.face_class.begin(), M.face_class.end(), face_class);
  if (tags)
    for (int d = 0; d < dim; ++d)
      for (int c = 0; c < nc; ++c) tags[(size_t)d * nc + c] = (M.flags[c] & fl_tag(d)) ? 1 : 0;
  if (dual_count) {
    std::fill(dual_count, dual_count + (size_t)(dim + 1) * nc, 0);
    for (auto& v : M.dual_unk)
      for (int g : v) dual_count[g]++;
  }
  if (pins) std::copy(M.pins.begin(), M.pins.end(), pins);
}

int check_ctx(const pns_ctx* ctx) { return ctx ? PNS_OK : PNS_ERR_ARG; }

}  // namespace

// ============================================================================ C ABI
extern "C" {

void pns_default_options(pns_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->periodic[0] = 1;
  o->variant = PNS_GPLMM;
  o->precision = PNS_FP64;
  o->combine = PNS_COMBINE_BUILD;
  o->n_dilate = 1;
  o->n_tag = 1;
  o->restart = 100;
  o->max_fgmres = 2000;
  o->max_newton = 30;
  o->inner_tol = 1e-9;
  o->newton_tol = 1e-8;
  o->refine_steps = -1;
  o->timing = 0;
  o->stream = nullptr;
  o->block_inner_its = 20;
  o->block_inner_tol = 1e-2;
  o->gj_tensor_cores = 2;
  o->rebuild_every = 0;
}

int pns_setup(pns_ctx** out, int nz, int ny, int nx, const uint8_t* mask, const int32_t* labels, double rho,
              double mu, const double b[3], double dt, const pns_options* opt) {
  if (!out || !mask || !labels || !b || nz < 1 || ny < 1 || nx < 1) return PNS_ERR_ARG;
  if ((long long)nx * ny * nz * 4 >= (1LL << 31)) return PNS_ERR_ARG;
  *out = nullptr;
  pns_ctx* ctx = new (std::nothrow) pns_ctx;
  if (!ctx) return PNS_ERR_OOM;
  Ctx& C = ctx->c;
  double t0 = now_ms();
  if (opt) C.opt = *opt;
  else pns_default_options(&C.opt);
  if (C.opt.restart < 1 || C.opt.restart > 127 || C.opt.n_dilate < 0 || C.opt.n_tag < 1 || C.opt.precision < 0 ||
      C.opt.precision > 2 || C.opt.variant < 0 || C.opt.variant > 4 || C.opt.block_inner_its < 1 ||
      C.opt.block_inner_its > 100 || !(C.opt.block_inner_tol > 0.0) || C.opt.gj_tensor_cores < 0 ||
      C.opt.gj_tensor_cores > 3 || C.opt.rebuild_every < 0) {
    delete ctx;
    return PNS_ERR_ARG;
  }
  if (!(rho > 0) || !(mu > 0)) {
    delete ctx;
    return PNS_ERR_ARG;
  }
  C.stream = (cudaStream_t)C.opt.stream;
  C.G.nx = nx;
  C.G.ny = ny;
  C.G.nz = nz;
  C.G.dim = nz == 1 ? 2 : 3;
  C.G.ncell = nx * ny * nz;
  for (int a = 0; a < 3; ++a) C.G.per[a] = C.opt.periodic[a] ? 1 : 0;
  if (C.G.dim == 2) C.G.per[2] = 0;
  C.P.rho = rho;
  C.P.mu = mu;
  C.P.inv_dt = dt > 0 ? 1.0 / dt : 0.0;
  for (int a = 0; a < 3; ++a) C.P.b[a] = b[a];
  C.nfull = (long long)(C.G.dim + 1) * C.G.ncell;
  int rc = build_maps(C.G, mask, labels, C.opt.n_dilate, C.opt.n_tag, C.M, C.err);
  if (rc != 0) {
    delete ctx;
    return PNS_ERR_ARG;
  }
  int st = PNS_OK;
  do {
    cudaError_t e;
    if ((e = upload(C.flags, C.M.flags, C.stream)) != cudaSuccess) { st = fail(C, PNS_ERR_CUDA, "upload flags", e); break; }
    if ((e = upload(C.owner, C.M.owner, C.stream)) != cudaSuccess) { st = fail(C, PNS_ERR_CUDA, "upload owner", e); break; }
    if ((e = upload(C.cell_iface, C.M.cell_iface, C.stream)) != cudaSuccess) { st = fail(C, PNS_ERR_CUDA, "upload iface", e); break; }
    if ((e = cudaEventCreate(&C.ev0)) != cudaSuccess || (e = cudaEventCreate(&C.ev1)) != cudaSuccess) {
      st = fail(C, PNS_ERR_CUDA, "event", e);
      break;
    }
  } while (0);
  if (st != PNS_OK) {
    delete ctx;
    return st;
  }
  // device address of the fixed scratch array of pns_precond_apply_static, taken here (a call that may
  // allocate) so that the allocation-free apply only reads it; a failure only disables that entry point
  {
    cudaError_t e = static_scratch_init(&C.static_scratch);
    if (e != cudaSuccess) {
      C.static_scratch = nullptr;
      C.static_err = std::string("device address of the static scratch array: ") + cudaGetErrorString(e);
      cudaGetLastError();
    }
  }
  C.t_setup_ms = now_ms() - t0;
  *out = ctx;
  return PNS_OK;
}

void pns_destroy(pns_ctx* ctx) {
  if (!ctx) return;
  for (cudaEvent_t e : ctx->c.ev_pool) cudaEventDestroy(e);
  if (ctx->c.ev0) cudaEventDestroy(ctx->c.ev0);
  if (ctx->c.ev1) cudaEventDestroy(ctx->c.ev1);
  delete ctx;
}

const char* pns_last_error(const pns_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int pns_get_info(const pns_ctx* ctx, pns_info* info) {
  if (check_ctx(ctx) || !info) return PNS_ERR_ARG;
  const Ctx& C = ctx->c;
  memset(info, 0, sizeof *info);
  info->nx = C.G.nx;
  info->ny = C.G.ny;
  info->nz = C.G.nz;
  info->dim = C.G.dim;
  info->ncell = C.G.ncell;
  info->n_unknowns = C.M.n_unknowns;
  info->n_faces = C.M.n_faces;
  info->n_cells = C.M.n_cells;
  info->n_prim = C.M.n_prim;
  info->n_iface = C.M.n_iface;
  info->n_pins = (int)C.M.pins.size();
  info->n_dropped_labels = C.M.n_dropped;
  for (auto& v : C.M.prim_unk) {
    info->prim_unknowns_total += (long long)v.size();
    info->prim_sum_n2 += (double)v.size() * v.size();
    info->max_block = std::max(info->max_block, (int)v.size());
  }
  for (auto& v : C.M.dual_unk) {
    info->dual_unknowns_total += (long long)v.size();
    info->dual_sum_n2 += (double)v.size() * v.size();
    info->max_block = std::max(info->max_block, (int)v.size());
  }
  size_t bytes = 0;
  const DevBuf* bufs[] = {&C.flags, &C.owner, &C.cell_iface, &C.pc.prim.mat, &C.pc.dual.mat, &C.pc.basis,
                          &C.pc.ao_inv, &C.V, &C.Z, &C.w0, &C.w1, &C.w2, &C.w3, &C.w4, &C.pk_x, &C.pk_y};
  for (auto* p : bufs) bytes += p->bytes;
  info->device_bytes = bytes;
  info->static_scratch_capacity = static_scratch_capacity();
  info->static_apply_bytes = C.pc.built && C.pc.variant != PNS_BLOCK_SCHUR ? static_apply_bytes(C) : 0;
  return PNS_OK;
}

int pns_residual(pns_ctx* ctx, const double* x, const double* x_prev, double* r) {
  if (check_ctx(ctx) || !x || !r) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  CK(launch_residual(C, 0, x, x_prev, r));
  return PNS_OK;
}

int pns_jacobian_apply(pns_ctx* ctx, const double* x_lin, const double* v, double* y) {
  if (check_ctx(ctx) || !x_lin || !v || !y) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  CK(launch_apply<double>(C, OP_NEWTON, x_lin, v, nullptr, y, true));
  return PNS_OK;
}

int pns_operator_apply(pns_ctx* ctx, int variant, const double* x_lin, const double* v, double* y) {
  if (check_ctx(ctx) || !x_lin || !v || !y || variant < 0 || variant > 3) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  CK(launch_apply<double>(C, op_of_variant(variant), x_lin, v, nullptr, y, true));
  return PNS_OK;
}

int pns_build_precond(pns_ctx* ctx, const double* x_lin) {
  if (check_ctx(ctx) || !x_lin) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  // the aPLMM_S build matrix is the Stokes operator, which does not depend on x_lin: a built aPLMM_S
  // preconditioner (from pns_stokes_solve or an earlier build) is already the one asked for
  if (C.opt.variant == PNS_APLMM_S && C.pc.built && C.pc.variant == PNS_APLMM_S) return PNS_OK;
  return build_precond(C, C.pc, C.opt.variant, x_lin);
}

int pns_precond_apply(pns_ctx* ctx, const double* v, double* z) {
  if (check_ctx(ctx) || !v || !z) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  return precond_apply(C, C.pc, v, z);
}

int pns_set_tuning(pns_ctx* ctx, const int* table) {
  if (check_ctx(ctx) || !table) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  for (int b = 0; b < TUNE_BINS; ++b)
    if (table[b] < 0 || table[b] >= TUNE_CONFIGS) return fail(C, PNS_ERR_ARG, "tuning table: config id out of range");
  for (int b = 0; b < TUNE_BINS; ++b) C.tune[b] = table[b];
  for (BlockSet* B : {&C.pc.prim, &C.pc.dual, &C.pc.bs.bf, &C.pc.bs.bl})
    if (B->nblk && B->idx.p) CKS(build_gemv_items(C, *B, C.tune));
  return PNS_OK;
}

int pns_autotune(pns_ctx* ctx, int* table, double* ms) {
  if (check_ctx(ctx)) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  Precond& pc = C.pc;
  if (!pc.built || pc.variant == PNS_BLOCK_SCHUR) return fail(C, PNS_ERR_STATE, "pns_autotune needs a built PLMM preconditioner");
  const cudaStream_t s = C.stream;
  const long long pkn = std::max(1LL, std::max(pc.prim.n_total, pc.dual.n_total));
  DevBuf out, pk;
  CK(dalloc(out, sizeof(double) * pkn));
  CK(dalloc(pk, sizeof(double) * pkn));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<double> t(TUNE_BINS * TUNE_CONFIGS, 0.0);
  int saved[TUNE_BINS];
  for (int b = 0; b < TUNE_BINS; ++b) saved[b] = C.tune[b];
  int rc = PNS_OK;
  for (int bin = 0; bin < TUNE_BINS && rc == PNS_OK; ++bin) {
    for (int cfg = 0; cfg < TUNE_CONFIGS && rc == PNS_OK; ++cfg) {
      for (BlockSet* B : {&pc.prim, &pc.dual}) {
        if (B->nblk == 0) continue;
        // a work list of this bin's blocks only, in this config
        BlockSet& S = *B;
        std::vector<int> keep;
        for (int q = 0; q < S.nblk; ++q)
          if (tune_bin(S.n[q]) == bin) keep.push_back(q);
        if (keep.empty()) continue;
        std::vector<int4> items;
        for (int q : keep)
          for (int r = 0; r < S.n[q]; r += TUNE_ROWS[cfg])
            items.push_back(make_int4(q, r, std::min(TUNE_ROWS[cfg], S.n[q] - r), TUNE_LANES[cfg]));
        DevBuf saved_items;
        saved_items.p = S.items_p.p;
        saved_items.bytes = S.items_p.bytes;
        const int saved_n = S.nitems_p;
        S.items_p.p = nullptr;
        S.items_p.bytes = 0;
        cudaError_t e = upload(S.items_p, items, s);
        S.nitems_p = (int)items.size();
        float best = 1e30f;
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
          cudaEventRecord(e0, s);
          if (pc.precision == PNS_FP64)
            e = launch_local_gemv_p<double, double>(S, S.mat.as<double>(), pk.as<double>(), out.as<double>(), 2, s);
          else if (pc.precision == PNS_FP32)
            e = launch_local_gemv_p<float, float>(S, S.mat.as<float>(), pk.as<float>(), out.as<double>(), 2, s);
          else
            e = launch_local_gemv_p<__nv_bfloat16, float>(S, S.mat.as<__nv_bfloat16>(), pk.as<float>(),
                                                          out.as<double>(), 2, s);
          cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float msr = 0;
          if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&msr, e0, e1) == cudaSuccess) best = std::min(best, msr);
        }
        S.items_p.release();
        S.items_p.p = saved_items.p;
        S.items_p.bytes = saved_items.bytes;
        saved_items.p = nullptr;
        S.nitems_p = saved_n;
        if (e != cudaSuccess) {
          rc = fail(C, PNS_ERR_CUDA, "pns_autotune", e);
          break;
        }
        t[bin * TUNE_CONFIGS + cfg] += best;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int best[TUNE_BINS];
  for (int bin = 0; bin < TUNE_BINS; ++bin) {
    best[bin] = saved[bin];
    double bt = 1e300;
    for (int cfg = 0; cfg < TUNE_CONFIGS; ++cfg) {
      const double v = t[bin * TUNE_CONFIGS + cfg];
      if (v > 0 && v < bt) {
        bt = v;
        best[bin] = cfg;
      }
    }
  }
  if (table)
    for (int b = 0; b < TUNE_BINS; ++b) table[b] = best[b];
  if (ms)
    for (int q = 0; q < TUNE_BINS * TUNE_CONFIGS; ++q) ms[q] = t[q];
  return pns_set_tuning(ctx, best);
}

int pns_newton_solve(pns_ctx* ctx, double* x, const double* x_prev, pns_stats* st) {
  if (check_ctx(ctx) || !x) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  if (!C.pc.built) {
    CKS(build_precond(C, C.pc, C.opt.variant, x));
  } else if (x_prev && C.opt.rebuild_every > 0 && C.solves_since_build >= C.opt.rebuild_every &&
             C.pc.variant != PNS_APLMM_S) {
    CKS(build_precond(C, C.pc, C.opt.variant, x));   // at this time step's initial guess
  }
  if (x_prev) ++C.solves_since_build;
  return newton(C, C.pc, 0, x, x_prev, st);
}

int pns_stokes_solve(pns_ctx* ctx, double* x, pns_stats* st) {
  if (check_ctx(ctx) || !x) return PNS_ERR_ARG;
  Ctx& C = ctx->c;
  Precond tmp;
  Precond* pc = &tmp;
  if (C.opt.variant == PNS_APLMM_S) {
    // the context's own preconditioner is the aPLMM_S one: build it once and keep it for Newton
    if (!C.pc.built || C.pc.variant != PNS_APLMM_S) CKS(build_precond(C, C.pc, PNS_APLMM_S, nullptr));
    pc = &C.pc;
  } else {
    CKS(build_precond(C, tmp, PNS_APLMM_S, nullptr));
  }
  CK(cudaMemsetAsync(x, 0, sizeof(double) * C.nfull, C.stream));
  int maxn = C.opt.max_newton;
  C.opt.max_newton = std::min(maxn, 3);
  int code = newton(C, *pc, 1, x, nullptr, st);
  C.opt.max_newton = maxn;
  return code;
}

int pns_export_coarse(const pns_ctx* ctx, double* ao_inv, int* n_o) {
  if (check_ctx(ctx) || !n_o) return PNS_ERR_ARG;
  const Ctx& C = ctx->c;
  *n_o = C.pc.n_o;
  if (!C.pc.built || !C.pc.coarse) return PNS_ERR_STATE;
  if (ao_inv) {
    cudaError_t e = cudaMemcpy(ao_inv, C.pc.ao_inv.p, sizeof(double) * (size_t)C.pc.n_o * C.pc.n_o,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return PNS_ERR_CUDA;
  }
  return PNS_OK;
}

int pns_export_maps(const pns_ctx* ctx, int32_t* cell_prim, int32_t* cell_iface, int32_t* face_class, uint8_t* tags,
                    int32_t* dual_count, int32_t* pins) {
  if (check_ctx(ctx)) return PNS_ERR_ARG;
  const Ctx& C = ctx->c;
  export_maps(C.M, C.G, cell_prim, cell_iface, face_class, tags, dual_count, pins);
  return PNS_OK;
}

int pns_maps_host(int nz, int ny, int nx, const uint8_t* mask, const int32_t* labels, const int periodic[3],
                  int n_dilate, int n_tag, int32_t* cell_prim, int32_t* cell_iface, int32_t* face_class,
                  uint8_t* tags, int32_t* dual_count, int32_t* pins, int32_t counts[4]) {
  if (!mask || !labels || !periodic || nz < 1 || ny < 1 || nx < 1 || n_dilate < 0 || n_tag < 1) return PNS_ERR_ARG;
  if ((long long)nx * ny * nz * 4 >= (1LL << 31)) return PNS_ERR_ARG;
  Geo G;
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.dim = nz == 1 ? 2 : 3;
  G.ncell = nx * ny * nz;
  for (int a = 0; a < 3; ++a) G.per[a] = periodic[a] ? 1 : 0;
  if (G.dim == 2) G.per[2] = 0;
  Maps M;
  std::string err;
  if (build_maps(G, mask, labels, n_dilate, n_tag, M, err) != 0) return PNS_ERR_ARG;
  export_maps(M, G, cell_prim, cell_iface, face_class, tags, dual_count, pins);
  if (counts) {
    counts[0] = M.n_prim;
    counts[1] = M.n_iface;
    counts[2] = (int32_t)M.pins.size();
    counts[3] = M.n_dropped;
  }
  return PNS_OK;
}

}  // extern "C"
