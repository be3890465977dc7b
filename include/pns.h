/*
 * pns.h -- C ABI of libpns: Newton-FGMRES for MAC-discretised incompressible Navier-Stokes on a
 * voxel image, preconditioned by the pore-level multiscale preconditioners gPLMM, aPLMM_NS and
 * aPLMM_S of Li & Mehmani, "Preconditioning and Reduced-Order Modeling of Navier-Stokes Equations
 * in Complex Porous Microstructures" (arXiv 2510.22077).  Single GPU (NVIDIA GB300, sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Image: shape (nz, ny, nx), C order, x fastest; nz == 1 selects 2D.  Solver axis 0 = x, 1 = y,
 * 2 = z.  Grid spacing h = 1.
 *
 * Vectors ("full layout"): device pointers to double arrays of length (dim + 1) * ncell with
 * ncell = nx*ny*nz, blocks [u_x | u_y | (u_z) | p], each image-shaped.  The face array of axis d
 * at cell c holds the velocity on the LOW face of c along d (between c - e_d and c).  A face is an
 * unknown iff both flanking cells exist and are void (wrapping along periodic axes); a cell is an
 * unknown iff it is void.  Entries that are not unknowns are ignored on input and written as 0 on
 * output.  The caller owns every vector; the library never frees or retains caller pointers.
 *
 * Discretisation (Sec. 2 and Eq. 1 of the paper; readings where the paper is silent):
 *   momentum row of face q (axis d):  rho/dt (q - q_prev) [transient]
 *       + rho * sum_a upwind(U_a; q)          (advective (u.grad)u, first-order 3-point upwind)
 *       + mu  * sum_a (2q - q_{+a} - q_{-a})  (missing neighbour: 0 along d, ghost -q across d)
 *       + (p_c - p_{c-e_d}) - rho * b_d
 *   continuity row of cell c: sum_a (u_a(high face) - u_a(low face)); in each face-connected
 *   void component the cell with the lowest linear index is pinned instead: row = p.
 *
 * Execution: every call enqueues work on the stream given in pns_options.stream (NULL = the
 * legacy default stream) and, unless stated, returns without synchronising.
 *
 * Errors: every int-returning call returns PNS_OK (0) or a negative PNS_ERR_* code; the message
 * is kept in the context (pns_last_error).  No call aborts the process.  After PNS_ERR_CUDA the
 * context should be destroyed.
 */
#ifndef PNS_H
#define PNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque solver context; owned by the library (pns_setup creates it, pns_destroy frees it). */
typedef struct pns_ctx pns_ctx;

enum pns_status {
  PNS_OK = 0,
  PNS_ERR_ARG = -1,           /* bad argument (NULL pointer, bad size, labels inconsistent with mask) */
  PNS_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  PNS_ERR_OOM = -3,           /* device or host allocation failed */
  PNS_ERR_SINGULAR = -4,      /* zero or non-finite pivot in a local or coarse factor */
  PNS_ERR_NOT_CONVERGED = -5, /* Newton or FGMRES hit its iteration cap; outputs are still written */
  PNS_ERR_NAN = -6,           /* NaN/Inf in a residual norm */
  PNS_ERR_STATE = -7,         /* call made in the wrong state (e.g. apply before build) */
  PNS_ERR_TIMEOUT = -8        /* a device wait hit its limit */
};

/* Preconditioner family (Sec. 3-4):
 *   GPLMM    build matrix = Jacobian of the modified residual (Eq. 27): inertia w . grad u with the
 *            wind w = velocity of the linearisation state, inertia removed on tagged faces;
 *   APLMM_NS build matrix = Newton Jacobian at the linearisation state;
 *   APLMM_S  build matrix = Stokes Jacobian (inertia dropped, rho/dt kept);
 *   ML_ONLY  the dual-primary smoother alone (Eq. 24) built from the gPLMM matrix (no M_G);
 *   BLOCK_SCHUR  the block-triangular comparator of Sec. 1, M_B = [[F, B1], [0, X]] with X^{-1} the
 *            scaled BFBt approximation of the Schur complement (Eq. 4), D = diag(F); built from the
 *            Newton Jacobian at the linearisation state.  Its solves with F and with B2 D^{-1} B1 run
 *            GMRES (block_inner_its iterations at most, relative tolerance block_inner_tol) with block
 *            Jacobi over the pores (dense inverses in the storage precision; BF16 stores FP32).
 *            The preconditioner is then not a fixed linear map: FGMRES is what allows that. */
enum pns_variant { PNS_GPLMM = 0, PNS_APLMM_NS = 1, PNS_APLMM_S = 2, PNS_ML_ONLY = 3, PNS_BLOCK_SCHUR = 4 };

/* Storage / arithmetic precision of the preconditioner (local inverses, basis, coarse inverse,
 * inner residual updates).  The Newton residual, the outer Jacobian, Arnoldi and Givens are FP64. */
enum pns_precision { PNS_FP64 = 0, PNS_FP32 = 1, PNS_BF16 = 2 };

/* Which operator the residual updates inside M use (Eqs. 4a and 24):
 *   BUILD_MATRIX  the build matrix A_b (default: M is one fixed operator made from A_b);
 *   CURRENT_J     the Newton Jacobian FGMRES is solving. */
enum pns_combine { PNS_COMBINE_BUILD = 0, PNS_COMBINE_CURRENT = 1 };

typedef struct pns_options {
  int periodic[3];       /* wrap along x, y, z (default 1, 0, 0) */
  int variant;           /* enum pns_variant (default PNS_GPLMM) */
  int precision;         /* enum pns_precision (default PNS_FP64) */
  int combine;           /* enum pns_combine (default PNS_COMBINE_BUILD) */
  int n_dilate;          /* dual-grid dilations of each interface (default 1) */
  int n_tag;             /* gPLMM tag layers (default 1) */
  int restart;           /* FGMRES restart length m (default 100) */
  int max_fgmres;        /* FGMRES iterations per Newton step (default 2000) */
  int max_newton;        /* Newton iterations (default 30) */
  double inner_tol;      /* FGMRES: stop when ||J d + r|| < inner_tol * ||r(0)|| (default 1e-9) */
  double newton_tol;     /* Newton: stop when ||r(x)|| < newton_tol * ||r(0)|| (default 1e-8) */
  int refine_steps;      /* accuracy of the FP32/BF16 local solves (FP64 needs none):
                            -1 (default) one step of iterative refinement inside every local solve,
                               z = X t, z += X (t - A_b z) with an FP64 residual from the stencil
                               (a second pass over X per apply; error of order eps^2);
                             0 none (the Gauss-Jordan inverse as computed);
                             k > 0 k Newton-Schulz steps X <- X + X (I - A X) at build time on the
                               blocks whose max |I - A X| exceeds 1e-5 (2 n^3 flops per block and step) */
  int timing;            /* 1: record CUDA events around the local-solve kernels (pns_stats) */
  void* stream;          /* cudaStream_t to enqueue on (NULL = legacy default stream) */
  int block_inner_its;   /* PNS_BLOCK_SCHUR: inner GMRES iterations per solve with F or L (default 20) */
  double block_inner_tol;/* PNS_BLOCK_SCHUR: inner GMRES relative tolerance (default 1e-2) */
  int gj_tensor_cores;   /* FP32 Gauss-Jordan trailing update of the local inverses:
                            0 FP32 FMA units;
                            1 tensor cores through warp-level mma.sync, TF32 with a 3-term split (hi*hi +
                              hi*lo + lo*hi, close to FP32 accuracy);
                            2 (default) 5th-generation tensor cores (tcgen05.mma kind::tf32, accumulators in
                              TMEM, operands and C tiles moved by TMA), with the same 3-term split; one
                              persistent CTA per SM, loads, products and write-backs of consecutive tiles
                              overlapped;
                            3 the same tensor-core product with one CTA per tile and no overlap.
                            Measured on a GB300, 96^3 sphere pack: 39.8 (0) and 80.1 (3) TFLOP/s */
  int rebuild_every;     /* transient runs (pns_newton_solve with x_prev != NULL): 0 (default) keeps the
                            preconditioner built once and reuses it at every time step (Sec. 8.2); k > 0
                            rebuilds it at the initial guess of a time step once k time steps have been
                            solved with the current one.  An aPLMM_S preconditioner does not depend on the
                            state and is never rebuilt. */
} pns_options;

typedef struct pns_stats {
  int newton_its;                 /* Newton iterations taken */
  int fgmres_its_total;           /* FGMRES iterations summed over Newton steps */
  int fgmres_its[64];             /* per Newton step (first 64) */
  double res_hist[65];            /* ||r(x_k)|| / ||r(0)|| for k = 0 .. newton_its */
  double r0_norm;                 /* ||r(u=0, p=0)|| */
  double t_setup_ms;              /* maps + uploads (pns_setup) */
  double t_mg_ms;                 /* M_G build: closure/shape/correction vectors, coarse matrix */
  double t_ml_ms;                 /* M_L build: local block assembly, inversion, refinement */
  double t_sol_ms;                /* FGMRES self time (all Newton steps) */
  double t_local_ms;              /* time inside the batched local-solve kernels (timing == 1) */
  long long local_launches;       /* number of batched local-solve launches timed */
  double local_bytes_per_apply;   /* algorithmic bytes of one M_d + M_p local-solve pass */
  long long kernel_launches;      /* library-wide count of kernel launches so far (all contexts) */
  double refine_residual_max;     /* max |I - A X| of the FP32 local inverses before refinement */
  double t_gj_update_ms;          /* time inside the FP32 Gauss-Jordan update kernel (timing == 1; cumulative) */
  double gj_update_flops;         /* its algorithmic flops, 2 (n - nb)^2 nb per block and step (cumulative) */
  long long gj_update_launches;   /* its timed launches (cumulative) */
  long long gj_update_tiles;      /* 128 x 128 output tiles it processed (cumulative) */
  double t_mg_parts_ms[3];        /* t_mg of the last build split into: closure solves (shape and correction
                                     vectors), assembly of A^o, inversion of A^o */
  double gj_update_bytes;         /* algorithmic bytes of the timed update launches: the trailing matrix read and
                                     written and the two panels read, FP32, per block and step (cumulative) */
  long long precond_builds;       /* preconditioner builds of this context so far (cumulative) */
} pns_stats;

typedef struct pns_info {
  int nx, ny, nz, dim;
  long long ncell, n_unknowns, n_faces, n_cells;
  int n_prim, n_iface, n_pins, n_dropped_labels;
  long long prim_unknowns_total, dual_unknowns_total;
  double prim_sum_n2, dual_sum_n2;  /* sum of squared block sizes (dense inverse entries) */
  int max_block;
  size_t device_bytes;              /* bytes the context holds on the device */
  size_t static_scratch_capacity;   /* size of the fixed array of pns_precond_apply_static (bytes) */
  size_t static_apply_bytes;        /* bytes one pns_precond_apply_static of the built preconditioner takes
                                       from that array (0 before a build or for BLOCK_SCHUR); the call is
                                       refused when this exceeds static_scratch_capacity */
} pns_info;

/* Fill `opt` with the defaults listed above. */
void pns_default_options(pns_options* opt);

/* Create a context.  mask: HOST uint8 array (nz*ny*nx), 1 = void.  subdomain_labels: HOST int32
 * array, >= 1 on void cells, 0 on solid cells (PNS_ERR_ARG otherwise); labels need not be
 * consecutive (primary grids are numbered in ascending label order).  rho, mu > 0; b[3] body force
 * per unit mass; dt <= 0 selects the steady equations, dt > 0 backward Euler with step dt.
 * Builds the integer maps of Sec. 3.2.1-3.2.2 and Sec. 4 (pins, contact interfaces, face classes,
 * dual grids, gPLMM tags) and uploads them.  Copies its inputs.  Synchronises. */
int pns_setup(pns_ctx** out, int nz, int ny, int nx, const uint8_t* mask,
              const int32_t* subdomain_labels, double rho, double mu, const double b[3], double dt,
              const pns_options* opt);

/* Free everything the context holds.  NULL is accepted. */
void pns_destroy(pns_ctx* ctx);

/* Message of the last error on this context ("" if none).  Valid until the next call. */
const char* pns_last_error(const pns_ctx* ctx);

/* Fill the HOST struct `info` with the sizes of the context's problem: grid, unknown counts,
 * primary/dual block statistics, device bytes held.  PNS_ERR_ARG if ctx or info is NULL. */
int pns_get_info(const pns_ctx* ctx, pns_info* info);

/* r = r(x) (Eq. 3): the Newton residual in FP64.  x_prev: previous time level (device, full
 * layout) for backward Euler, or NULL (steady, or transient with u_prev = 0). */
int pns_residual(pns_ctx* ctx, const double* x, const double* x_prev, double* r);

/* y = J(x_lin) v: the Newton Jacobian of the residual of Eq. 3 at x_lin, i.e. the matrix of the linear
 * system FGMRES solves at each Newton step (Sec. 8, Eq. 3 differentiated), upwind branches frozen at
 * x_lin (FP64, matrix-free).  x_lin, v, y: device, full layout; y may not alias v.  PNS_ERR_ARG for a
 * NULL pointer. */
int pns_jacobian_apply(pns_ctx* ctx, const double* x_lin, const double* v, double* y);

/* y = A v for the build-matrix operator of a variant (enum pns_variant; ML_ONLY = GPLMM) at the
 * linearisation state x_lin (FP64).  Exposed for testing the gPLMM modified Jacobian (Eq. 27). */
int pns_operator_apply(pns_ctx* ctx, int variant, const double* x_lin, const double* v, double* y);

/* Build the preconditioner of opt.variant at the linearisation state x_lin (device, full layout):
 * local blocks of the primary and dual grids (Eq. 25) assembled densely and inverted, closure
 * blocks (Eqs. 6 and 9), shape and correction vectors (Eqs. 15 and 17), coarse matrix
 * A^o = R^ A_b P^ (Remark 1) and its inverse.  For APLMM_S the build matrix does not depend on
 * x_lin, so a built aPLMM_S preconditioner is kept and the call returns at once.  Synchronises. */
int pns_build_precond(pns_ctx* ctx, const double* x_lin);

/* z = M^{-1} v (Eqs. 4a, 24, 25, 20): FP64 in and out, internal precision opt.precision.
 * PNS_ERR_STATE before pns_build_precond. */
int pns_precond_apply(pns_ctx* ctx, const double* v, double* z);

/* z = M^{-1} v exactly as pns_precond_apply (the same apply body), but without allocating device
 * memory during the call: for callers that cannot call cudaMalloc when they apply the preconditioner
 * (a device allocator owned by someone else, or a footprint that must stay fixed after start-up).
 * The scratch vectors live in one file-scope device array of 24 MiB.  One apply takes
 *     5 * A(8 * nfull) + A(w * P) + R + 2 * A(8 * n_o)  bytes of it,
 * with nfull = (dim + 1) * ncell, P = the larger of the primary and dual packed sizes (block sizes
 * rounded up to 8, summed), A(x) = x rounded up to a multiple of 256, w = 8 for FP64 and 4 for FP32 /
 * BF16 preconditioners, R = A(8 * P) when the local solves are refined (refine_steps == -1, FP32 /
 * BF16) and 0 otherwise; pns_get_info reports the figure (static_apply_bytes).  Larger problems
 * return PNS_ERR_ARG with a message; a full layout of up to about 500,000 entries fits.
 * The array is shared by every call in the process and keeps the last call's contents (each call
 * writes every entry it reads first), so calls that overlap on the GPU race on it: serialise them.
 * Its device address is taken once per device inside pns_setup, with the context's device current;
 * the call itself only reads that address.  Under lazy module loading (the CUDA default) the code of
 * a kernel is loaded on its first launch in the process: a caller for whom even that must not happen
 * inside this call runs one pns_precond_apply first, or loads modules eagerly.
 * Every GPU that loads the library holds the array until exit.  The paper has no counterpart: this is
 * an interface of this library.  PNS_ERR_STATE before pns_build_precond, PNS_ERR_ARG for the
 * BLOCK_SCHUR variant. */
int pns_precond_apply_static(pns_ctx* ctx, const double* v, double* z);

/* Shapes of the batched local solves (Eq. 25: M_p and M_d applied as one persistent launch per block set).
 * The blocks are binned by size n: bin 0 n <= 64, 1 n <= 256, 2 n <= 1024, 3 n <= 4096, 4 n <= 16384,
 * 5 larger; each bin uses one of PNS_TUNE_CONFIGS shapes (lanes per matrix row, rows per work item):
 * 0 (8, 32), 1 (8, 128), 2 (16, 32), 3 (16, 128), 4 (32, 16), 5 (32, 64).  Default table {0, 0, 2, 4, 4, 4},
 * the choice of pns_autotune on a GB300 for the 96^3 sphere pack.
 * The paper has no counterpart: this is how this library schedules the paper's batched local solves. */
#define PNS_TUNE_BINS 6
#define PNS_TUNE_CONFIGS 6

/* Time every shape on every size bin of the built preconditioner's primary and dual blocks (CUDA events,
 * best of five launches after one warm-up, the two block sets summed) and adopt the fastest per bin.
 * table (HOST, PNS_TUNE_BINS ints, may be NULL) receives the chosen config ids; ms (HOST,
 * PNS_TUNE_BINS * PNS_TUNE_CONFIGS doubles, may be NULL) the times, ms[bin * PNS_TUNE_CONFIGS + config],
 * 0 for a bin with no block.  Allocates scratch for the duration of the call.  Synchronises.
 * PNS_ERR_STATE without a built PLMM-family preconditioner. */
int pns_autotune(pns_ctx* ctx, int* table, double* ms);

/* Adopt a tuning table (PNS_TUNE_BINS config ids, HOST), e.g. one saved from pns_autotune on the same
 * kind of GPU.  PNS_ERR_ARG for an id out of range. */
int pns_set_tuning(pns_ctx* ctx, const int* table);

/* Newton-FGMRES (Sec. 8).  x: device, full layout; initial guess on input, solution on output.
 * x_prev: previous time level (transient) or NULL.  Builds the preconditioner at the initial
 * guess if none is built.  st may be NULL.  Synchronises.  PNS_ERR_NOT_CONVERGED if max_newton is
 * reached (x holds the last iterate). */
int pns_newton_solve(pns_ctx* ctx, double* x, const double* x_prev, pns_stats* st);

/* Stokes solution (inertia dropped, rho b kept): the initial Newton iterate of Sec. 4 when no
 * nearby wind exists.  Builds an aPLMM_S preconditioner and runs FGMRES on the linear system.
 * When the context's variant is APLMM_S that preconditioner becomes the context's own (Newton then
 * uses it without a second build); otherwise it is temporary and the context's preconditioner is
 * left as it was.  x: device, output.  Synchronises. */
int pns_stokes_solve(pns_ctx* ctx, double* x, pns_stats* st);

/* Copy the inverse of the coarse matrix A^o = R^ A_b P^ (Remark 1) of the built preconditioner to a
 * HOST array of n_o * n_o doubles (row-major); *n_o receives the coarse size (coarse interfaces
 * first, then primary grids).  A primary grid on which rho b vanishes (no face unknown along a
 * nonzero component of b) has a zero correction vector and no coarse unknown: its row and column
 * are those of the identity.  ao_inv may be NULL to query n_o.  PNS_ERR_STATE before a build or
 * for ML_ONLY.  Synchronises. */
int pns_export_coarse(const pns_ctx* ctx, double* ao_inv, int* n_o);

/* Copy the integer maps to HOST arrays (for bit-exact tests).  Any pointer may be NULL.
 *   cell_prim[ncell]   primary grid of each cell (-1: interface cell or solid)
 *   cell_iface[ncell]  contact interface of each cell (-1: none)
 *   face_class[dim*ncell]  per axis: primary grid of the face, -1 interface face (f), -2 not an unknown
 *   tags[dim*ncell]    1 where the gPLMM modified residual drops the inertia
 *   dual_count[(dim+1)*ncell]  number of dual grids containing each unknown
 *   pins[n_pins]       pinned cells (ascending) */
int pns_export_maps(const pns_ctx* ctx, int32_t* cell_prim, int32_t* cell_iface, int32_t* face_class,
                    uint8_t* tags, int32_t* dual_count, int32_t* pins);

/* The same integer maps computed on the host alone, with no device and no context (Sec. 3.2.1,
 * Sec. 3.2.2, Sec. 4; the readings of pns_setup): for checks of the index maps at any size on a
 * machine without a GPU.
 *   nz, ny, nx, mask, labels   as pns_setup (HOST arrays of nz*ny*nx)
 *   periodic[3], n_dilate, n_tag   as in pns_options
 *   outputs   as pns_export_maps, HOST arrays sized by the caller (any may be NULL); pins needs
 *             room for nz*ny*nx entries
 *   counts[4] (may be NULL) receives n_prim, n_iface, n_pins, n_dropped_labels.
 * Returns PNS_ERR_ARG on bad sizes or labels inconsistent with the mask; touches no device. */
int pns_maps_host(int nz, int ny, int nx, const uint8_t* mask, const int32_t* labels, const int periodic[3],
                  int n_dilate, int n_tag, int32_t* cell_prim, int32_t* cell_iface, int32_t* face_class,
                  uint8_t* tags, int32_t* dual_count, int32_t* pins, int32_t counts[4]);

#ifdef __cplusplus
}
#endif

#endif /* PNS_H */
