// Internal types of libpns: device buffers, the preconditioner, the context and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pns.h"
#include "maps.h"
#include "stencil.cuh"

namespace pns {

// ---------------------------------------------------------------- device allocation helpers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return (T*)p; }
};

// Error carrier: kernels and launchers return cudaError_t; API functions map to pns_status.
struct Status {
  int code = PNS_OK;
  std::string msg;
};

// A batch of dense local blocks (primary grids, dual grids, or closure blocks).
struct BlockSet {
  int nblk = 0;
  std::vector<int> n;            // block sizes
  std::vector<int> ld;           // leading dimension of each stored matrix (row-major, padded)
  std::vector<long long> ioff;   // offset of each block's unknown list / packed local vector
  std::vector<long long> moff;   // offset (elements) of each block's matrix
  long long n_total = 0;         // sum of n
  long long m_total = 0;         // sum of n * ld
  double sum_n2 = 0;             // sum of n^2
  int nmax = 0;
  DevBuf idx;                    // int32 full indices, concatenated
  DevBuf d_n, d_ld, d_ioff, d_moff;
  DevBuf mat;                    // inverse storage (type depends on precision)
  // binned work list of the persistent GEMV: (block, first row, row count, lanes per row), largest blocks
  // first; built from the context's tuning table (build_gemv_items)
  int nitems_p = 0;
  DevBuf items_p;                // int4
  DevBuf counter;                // int: next item of the running launch
};

// Size bins and shapes of the persistent local GEMV (pns_autotune / pns_set_tuning of pns.h).
constexpr int TUNE_BINS = 6;     // n <= 64, 256, 1024, 4096, 16384, larger
constexpr int TUNE_CONFIGS = 6;  // (lanes per row, rows per item)
inline int tune_bin(int n) {
  return n <= 64 ? 0 : n <= 256 ? 1 : n <= 1024 ? 2 : n <= 4096 ? 3 : n <= 16384 ? 4 : 5;
}
constexpr int TUNE_LANES[TUNE_CONFIGS] = {8, 8, 16, 16, 32, 32};
constexpr int TUNE_ROWS[TUNE_CONFIGS] = {32, 128, 32, 128, 16, 64};
constexpr int TUNE_DEFAULT[TUNE_BINS] = {0, 0, 2, 4, 4, 4};   // pns_autotune on a GB300, 96^3 pack

// Block-triangular Schur comparator (variant PNS_BLOCK_SCHUR): pore blocks of F and L = B2 D^-1 B1 for
// block Jacobi, D = diag(F), and the workspace of its inner GMRES.
struct BlockSchurData {
  BlockSet bf, bl;               // pore blocks of F (faces) and of L (cells that are not pinned)
  DevBuf D;                      // diag(F) on faces, full layout
  int its = 20;                  // inner GMRES iterations (no restart)
  double tol = 1e-2;             // inner GMRES relative tolerance
  DevBuf V, Z, H, small, partial;
  DevBuf t1, t2, t3, t4, t5;     // full-layout temporaries
  DevBuf pk;                     // packed local vectors of the block-Jacobi solves
  long long inner_total = 0;     // inner iterations since the build
};

// Preconditioner built from one build matrix A_b (pns_build_precond / the internal Stokes solve).
struct Precond {
  bool built = false;
  int variant = PNS_GPLMM;
  int precision = PNS_FP64;
  int op = OP_OSEEN;             // stencil operator of A_b
  DevBuf state;                  // linearisation state of A_b (FP64, full layout)
  BlockSet prim, dual;
  bool coarse = true;
  int n_o = 0;                   // coarse interfaces + N^p
  int n_cif = 0;                 // coarse interfaces (adjacent to a primary grid)
  // basis: per primary grid a dense n_i x k_i matrix (k_i = |C_i| + 1), row-major, storage type
  std::vector<int> kcols;
  std::vector<long long> boff;
  DevBuf basis, d_boff, d_kcols, d_colid, d_coloff;   // colid: coarse column of each basis column
  DevBuf ao_inv;                 // N_o x N_o inverse of the coarse matrix (storage type)
  // restriction segments: interface cells (by interface) then primary unknowns (by primary grid)
  DevBuf seg_idx, seg_off;       // int32 indices, int64 offsets (n_o + 1)
  int nseg_items = 0;
  DevBuf seg_items;              // int2 (segment, chunk start) work list
  double local_bytes = 0;        // algorithmic bytes of one M_d + M_p pass
  double ns_residual_before = 0; // max |I - A X| of the local inverses before refinement
  BlockSchurData bs;             // variant PNS_BLOCK_SCHUR only
  bool apply_refine = false;     // one step of iterative refinement inside each local solve
};

// CUDA-event timing of the FP32 Gauss-Jordan update launches (cumulative; read after a synchronise)
struct GjTimer {
  double ms = 0, flops = 0, bytes = 0;   // bytes: the trailing matrix read and written once per step plus the panels
  long long launches = 0, tiles = 0;
};

struct Ctx {
  Geo G;
  Phy P;
  pns_options opt;
  cudaStream_t stream = nullptr;
  Maps M;
  std::string err;
  DevBuf flags;                  // uint8 per cell
  DevBuf owner;                  // int32 per full index
  DevBuf cell_iface;             // int32 per cell
  long long nfull = 0;
  Precond pc;
  // scratch vectors (precision-dependent types; FP64 buffers sized nfull)
  DevBuf w0, w1, w2, w3, w4;     // preconditioner internals (VT)
  DevBuf pk_x, pk_y;             // packed local vectors (VT), sized max(prim, dual) n_total
  DevBuf zpk;                    // packed FP64 local solutions of the refined local solves
  DevBuf coarse_rhs, coarse_x;   // double, n_o
  DevBuf red;                    // reduction scratch (double)
  // Krylov workspace
  int m_alloc = 0;
  DevBuf V, Z, H, givens, hvec, partial;
  DevBuf xk, rk, dx;
  // timing: event pairs around the batched local solves, read after the solve synchronises
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double t_local_ms = 0;
  long long n_builds = 0;        // preconditioner builds of this context (pns_stats.precond_builds)
  int solves_since_build = 0;    // transient Newton solves with the context's preconditioner since its build
  long long local_launches = 0;
  const double* cur_state = nullptr;   // Newton state for COMBINE_CURRENT
  double t_setup_ms = 0;
  double t_mg_ms = 0, t_ml_ms = 0;
  double t_mg_parts[3] = {0, 0, 0};  // closure solves (shape / correction vectors), A^o assembly, A^o inverse
  GjTimer gj;                    // update-kernel timing of the local-inverse builds (timing == 1)
  int tune[TUNE_BINS] = {TUNE_DEFAULT[0], TUNE_DEFAULT[1], TUNE_DEFAULT[2], TUNE_DEFAULT[3], TUNE_DEFAULT[4],
                         TUNE_DEFAULT[5]};   // config of each size bin of the persistent local GEMV
  void* static_scratch = nullptr;  // device address of the fixed scratch array of pns_precond_apply_static
  std::string static_err;        // why that address could not be taken at set-up ("" if it was)
};

// Scratch of one preconditioner apply: FP64 vectors of the full layout (zG, t1, zd, t2, zp), the packed
// local vectors in the working type (pk; max(prim, dual) n_total entries), the packed FP64 refined local
// solutions (zpk; only with apply_refine) and the two coarse vectors (n_o entries each).
struct ApplyScratch {
  double *zG = nullptr, *t1 = nullptr, *zd = nullptr, *t2 = nullptr, *zp = nullptr;
  void* pk = nullptr;
  double* zpk = nullptr;
  double *crhs = nullptr, *cx = nullptr;
  bool timed = false;            // record CUDA events around the batched local solves
};

// z = M^{-1} v (Eqs. 4a, 24, 25, 20) with the given scratch; the context's own apply and the
// allocation-free apply of pns_static.cu both run this body.
int precond_apply_with(Ctx& C, Precond& pc, const double* v, double* z, const ApplyScratch& W);

// The allocation-free apply (pns_static.cu): device address of its fixed array on the current device,
// taken once per device at context set-up; the array's size; the bytes one apply of a built
// preconditioner takes from it.
cudaError_t static_scratch_init(void** addr);
size_t static_scratch_capacity();
size_t static_apply_bytes(const Ctx& C);

// Counts every kernel launch of the library (all contexts); read through pns_stats.
void count_launch();
long long launch_count();

// ---------------------------------------------------------------- launchers (kernels_*.cu)
// stencil
cudaError_t launch_residual(const Ctx& C, int stokes, const double* x, const double* xprev, double* r);
template <typename VT>
cudaError_t launch_apply(const Ctx& C, int op, const double* state, const VT* v, const VT* b, VT* y, bool fp64_math);
cudaError_t launch_cast_d2f(const double* in, float* out, long long n, cudaStream_t s);
cudaError_t launch_cast_f2d(const float* in, double* out, long long n, cudaStream_t s);

// dense local blocks
template <typename ST>
cudaError_t launch_assemble(const Ctx& C, const BlockSet& B, int op, const double* state, ST* mat, int closure);
// Gauss-Jordan trailing update on the 5th-generation tensor cores (kernels_gj_tc.cu): per build of one
// block set, setup() makes the split-panel buffers and the tensor maps of the blocks; step() runs the
// panel split and the update of panel step k for the first cnt blocks of `order`.
struct GjTcImpl;
struct GjTc {
  GjTcImpl* impl;
  GjTc();
  ~GjTc();
  GjTc(const GjTc&) = delete;
  GjTc& operator=(const GjTc&) = delete;
  cudaError_t setup(const BlockSet& B, float* mat, cudaStream_t s, bool persistent);
  cudaError_t step(const BlockSet& B, float* mat, int k, int cnt, const int* d_order, const long long* d_pre2,
                   long long ntiles, const std::vector<int>& order, int* d_bad, cudaStream_t s);
};

template <typename ST>
cudaError_t launch_gj_invert(const BlockSet& B, ST* mat, int* d_bad, cudaStream_t s, GjTimer* timer = nullptr,
                             int tensor_cores = 0);
cudaError_t launch_closure_rhs(const Ctx& C, const BlockSet& B, int op, const double* state, const int* d_colbase,
                               const int* d_cols, const long long* d_roff, const int* d_kc, double* rhs);
template <typename ST, typename AT>
cudaError_t launch_block_mm(const BlockSet& B, const ST* mat, const double* rhs, const long long* d_roff,
                            const int* d_kc, const std::vector<int>& kc, double* out, cudaStream_t s);
template <typename ST, typename PT>
cudaError_t launch_local_solve_refined(const Ctx& C, const BlockSet& B, int op, const double* state, const ST* mat,
                                       const double* t, double* z, PT* pk_x, double* zp, int add, cudaStream_t s);
template <typename ST, typename PT>
cudaError_t launch_local_gemv_p(const BlockSet& B, const ST* mat, const PT* pk, double* z, int mode, cudaStream_t s);
template <typename ST, typename PT>
cudaError_t launch_local_solve(const BlockSet& B, const ST* mat, const double* t, double* z, PT* pk_x, int add,
                               cudaStream_t s);

template <typename ST, typename AT>
cudaError_t launch_ns_refine(const Ctx& C, const BlockSet& B, int op, const double* state, int closure, ST* mat,
                             int steps, double thresh, size_t budget_bytes, double* max_before, double* max_after);
cudaError_t launch_closure_residual(const Ctx& C, const BlockSet& B, int op, const double* state,
                                    const long long* d_roff, const int* d_kc, const double* rhs, const double* S,
                                    double* res);
cudaError_t launch_add_vec(double* a, const double* b, long long n, cudaStream_t s);

// Closure-block solves by the Woodbury identity on the primary-block inverses (see kernels_dense.cu)
struct WoodburyImpl;
struct Woodbury {
  WoodburyImpl* impl;
  Woodbury();
  ~Woodbury();
  Woodbury(const Woodbury&) = delete;
  Woodbury& operator=(const Woodbury&) = delete;
  template <typename ST>
  cudaError_t setup(const Ctx& C, const BlockSet& B, int op, const double* state, const ST* X,
                    const std::vector<int>& kc, int* d_bad);
  template <typename ST>
  cudaError_t apply(const Ctx& C, const BlockSet& B, const ST* X, const double* R, double* S, double* Y,
                    const long long* d_roff, const int* d_kc, const std::vector<int>& kc);
};

// block-triangular Schur comparator (kernels_block.cu)
cudaError_t launch_diag_F(const Ctx& C, int op, const double* state, double* D);
cudaError_t launch_grad(const Ctx& C, const double* y, const double* D, const double* v, int mode, double* t);
cudaError_t launch_div(const Ctx& C, const double* t, const double* D, double sign, double* y);
cudaError_t launch_compose(const Ctx& C, const double* a, const double* b, int mode, double* out);
cudaError_t launch_zero_cells(const Ctx& C, double* y);
template <typename ST>
cudaError_t launch_assemble_L(const Ctx& C, const BlockSet& B, const double* D, ST* mat);

// coarse
cudaError_t launch_seg_sum(const Precond& pc, const void* v, int vt_is_double, double* out, cudaStream_t s);
template <typename ST, typename VT>
cudaError_t launch_prolong(const Ctx& C, const Precond& pc, const double* xo, VT* z);
cudaError_t launch_coarse_invert(double* A, int n, double* work, int* perm, int* d_bad, cudaStream_t s);
template <typename ST>
cudaError_t launch_coarse_gemv(const ST* Ainv, int n, const double* rhs, double* x, cudaStream_t s);

// krylov (FP64)
cudaError_t launch_multidot(const double* V, long long ld, int nvec, const double* w, long long n, double* partial,
                            int nblocks, double* out, cudaStream_t s);
cudaError_t launch_multi_axpy(double* w, const double* V, long long ld, int nvec, const double* h, double sign,
                              long long n, cudaStream_t s);
cudaError_t launch_dot(const double* a, const double* b, long long n, double* partial, double* out, cudaStream_t s);
cudaError_t launch_scale(double* x, long long n, const double* num, const double* den, int invert, cudaStream_t s);
cudaError_t launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t s);
cudaError_t launch_givens(double* H, int ldh, double* cs, double* sn, double* g, int j, double* resid_out,
                          cudaStream_t s);
cudaError_t launch_hcol(double* H, int ldh, int j, const double* h1, const double* h2, const double* hnorm,
                        cudaStream_t s);
cudaError_t launch_trisolve_update(const double* H, int ldh, const double* g, int k, double* y, const double* Z,
                                   long long ld, double* x, long long n, cudaStream_t s);

}  // namespace pns

// The opaque handle of the C ABI.
struct pns_ctx {
  pns::Ctx c;
};
