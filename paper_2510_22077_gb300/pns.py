"""Python binding of libpns (include/pns.h): ctypes marshalling only.  Every step of the solver runs
inside the CUDA library; this module converts tensors to device pointers and status codes to
exceptions.  It refuses to run without the compiled library or without a CUDA device."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpns.so")

GPLMM, APLMM_NS, APLMM_S, ML_ONLY, BLOCK_SCHUR = 0, 1, 2, 3, 4
VARIANTS = {"gplmm": GPLMM, "aplmm_ns": APLMM_NS, "aplmm_s": APLMM_S, "ml_only": ML_ONLY,
            "block_schur": BLOCK_SCHUR}
FP64, FP32, BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16}
COMBINE_BUILD, COMBINE_CURRENT = 0, 1
TUNE_BINS, TUNE_CONFIGS = 6, 6
# (lanes per row, rows per work item) of each local-solve config id, and the block-size bin edges
TUNE_SHAPES = [(8, 32), (8, 128), (16, 32), (16, 128), (32, 16), (32, 64)]
TUNE_BIN_EDGES = [64, 256, 1024, 4096, 16384]

STATUS = {0: "PNS_OK", -1: "PNS_ERR_ARG", -2: "PNS_ERR_CUDA", -3: "PNS_ERR_OOM", -4: "PNS_ERR_SINGULAR",
          -5: "PNS_ERR_NOT_CONVERGED", -6: "PNS_ERR_NAN", -7: "PNS_ERR_STATE", -8: "PNS_ERR_TIMEOUT"}


class PnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("periodic", ctypes.c_int * 3), ("variant", ctypes.c_int), ("precision", ctypes.c_int),
                ("combine", ctypes.c_int), ("n_dilate", ctypes.c_int), ("n_tag", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_fgmres", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("newton_tol", ctypes.c_double), ("refine_steps", ctypes.c_int),
                ("timing", ctypes.c_int), ("stream", ctypes.c_void_p), ("block_inner_its", ctypes.c_int),
                ("block_inner_tol", ctypes.c_double), ("gj_tensor_cores", ctypes.c_int),
                ("rebuild_every", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("fgmres_its_total", ctypes.c_int),
                ("fgmres_its", ctypes.c_int * 64), ("res_hist", ctypes.c_double * 65),
                ("r0_norm", ctypes.c_double), ("t_setup_ms", ctypes.c_double), ("t_mg_ms", ctypes.c_double),
                ("t_ml_ms", ctypes.c_double), ("t_sol_ms", ctypes.c_double), ("t_local_ms", ctypes.c_double),
                ("local_launches", ctypes.c_longlong), ("local_bytes_per_apply", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("refine_residual_max", ctypes.c_double),
                ("t_gj_update_ms", ctypes.c_double), ("gj_update_flops", ctypes.c_double),
                ("gj_update_launches", ctypes.c_longlong), ("gj_update_tiles", ctypes.c_longlong),
                ("t_mg_parts_ms", ctypes.c_double * 3), ("gj_update_bytes", ctypes.c_double),
                ("precond_builds", ctypes.c_longlong)]

    def as_dict(self):
        n = self.newton_its
        return {"newton_its": n, "fgmres_its_total": self.fgmres_its_total,
                "fgmres_its": list(self.fgmres_its[:min(n, 64)]), "res_hist": list(self.res_hist[:min(n + 1, 65)]),
                "r0_norm": self.r0_norm, "t_setup_ms": self.t_setup_ms, "t_mg_ms": self.t_mg_ms,
                "t_ml_ms": self.t_ml_ms, "t_sol_ms": self.t_sol_ms, "t_local_ms": self.t_local_ms,
                "local_launches": self.local_launches, "local_bytes_per_apply": self.local_bytes_per_apply,
                "kernel_launches": self.kernel_launches, "refine_residual_max": self.refine_residual_max,
                "t_gj_update_ms": self.t_gj_update_ms, "gj_update_flops": self.gj_update_flops,
                "gj_update_launches": self.gj_update_launches, "gj_update_tiles": self.gj_update_tiles,
                "t_mg_parts_ms": list(self.t_mg_parts_ms), "gj_update_bytes": self.gj_update_bytes,
                "precond_builds": self.precond_builds}


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dim", ctypes.c_int),
                ("ncell", ctypes.c_longlong), ("n_unknowns", ctypes.c_longlong), ("n_faces", ctypes.c_longlong),
                ("n_cells", ctypes.c_longlong), ("n_prim", ctypes.c_int), ("n_iface", ctypes.c_int),
                ("n_pins", ctypes.c_int), ("n_dropped_labels", ctypes.c_int),
                ("prim_unknowns_total", ctypes.c_longlong), ("dual_unknowns_total", ctypes.c_longlong),
                ("prim_sum_n2", ctypes.c_double), ("dual_sum_n2", ctypes.c_double), ("max_block", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("static_scratch_capacity", ctypes.c_size_t),
                ("static_apply_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libpns.so (built by __graft_entry__.build()).  Raises when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpns.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "pns_default_options": (V, [ctypes.POINTER(Options)]),
        "pns_setup": (I, [ctypes.POINTER(P), I, I, I, P, P, D, D, ctypes.POINTER(D), D, ctypes.POINTER(Options)]),
        "pns_destroy": (V, [P]),
        "pns_last_error": (ctypes.c_char_p, [P]),
        "pns_get_info": (I, [P, ctypes.POINTER(Info)]),
        "pns_residual": (I, [P, P, P, P]),
        "pns_jacobian_apply": (I, [P, P, P, P]),
        "pns_operator_apply": (I, [P, I, P, P, P]),
        "pns_build_precond": (I, [P, P]),
        "pns_precond_apply": (I, [P, P, P]),
        "pns_precond_apply_static": (I, [P, P, P]),
        "pns_newton_solve": (I, [P, P, P, ctypes.POINTER(Stats)]),
        "pns_stokes_solve": (I, [P, P, ctypes.POINTER(Stats)]),
        "pns_export_maps": (I, [P, P, P, P, P, P, P]),
        "pns_export_coarse": (I, [P, P, ctypes.POINTER(ctypes.c_int)]),
        "pns_maps_host": (I, [I, I, I, P, P, P, I, I, P, P, P, P, P, P, P]),
        "pns_autotune": (I, [P, P, P]),
        "pns_set_tuning": (I, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def pns_maps_host(mask, labels, periodic=(True, False, False), n_dilate=1, n_tag=1):
    """The integer maps of pns_setup computed by the library on the host (no device needed)."""
    lib = load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    if mask.ndim != 3 or labels.shape != mask.shape:
        raise ValueError("mask and labels must be (nz, ny, nx) arrays of equal shape")
    nz, ny, nx = mask.shape
    dim = 2 if nz == 1 else 3
    nc = nx * ny * nz
    out = {"cell_prim": np.zeros(nc, np.int32), "cell_iface": np.zeros(nc, np.int32),
           "face_class": np.zeros(dim * nc, np.int32), "tags": np.zeros(dim * nc, np.uint8),
           "dual_count": np.zeros((dim + 1) * nc, np.int32), "pins": np.zeros(nc, np.int32)}
    counts = np.zeros(4, np.int32)
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.pns_maps_host(nz, ny, nx, P(mask), P(labels), ctypes.cast(per, ctypes.c_void_p), int(n_dilate),
                           int(n_tag), P(out["cell_prim"]), P(out["cell_iface"]), P(out["face_class"]),
                           P(out["tags"]), P(out["dual_count"]), P(out["pins"]), P(counts))
    if rc != 0:
        raise PnsError(rc, "pns_maps_host: bad sizes or labels inconsistent with the mask")
    out["face_class"] = out["face_class"].reshape(dim, nc)
    out["tags"] = out["tags"].reshape(dim, nc).astype(bool)
    out["pins"] = out["pins"][:counts[2]]
    out["n_prim"], out["n_iface"], out["n_pins"], out["n_dropped_labels"] = (int(c) for c in counts)
    return out


def default_options() -> Options:
    o = Options()
    load().pns_default_options(ctypes.byref(o))
    return o


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One pns context: geometry, parameters, maps and (once built) a preconditioner."""

    def __init__(self, mask, labels, rho, mu, b, dt=0.0, variant="gplmm", precision="fp64", combine="build",
                 periodic=(True, False, False), n_dilate=1, n_tag=1, restart=100, max_fgmres=2000, max_newton=30,
                 inner_tol=1e-9, newton_tol=1e-8, timing=False, stream=None, block_inner_its=20,
                 block_inner_tol=1e-2, refine_steps=-1, gj_tensor_cores=None, rebuild_every=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpns needs a CUDA device")
        self.lib = load()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        if mask.ndim != 3 or labels.shape != mask.shape:
            raise ValueError("mask and labels must be (nz, ny, nx) arrays of equal shape")
        self.shape = mask.shape
        nz, ny, nx = mask.shape
        self.dim = 2 if nz == 1 else 3
        self.ncell = nx * ny * nz
        self.nfull = (self.dim + 1) * self.ncell
        o = default_options()
        o.periodic[:] = [int(p) for p in periodic]
        o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.combine = COMBINE_BUILD if combine == "build" else COMBINE_CURRENT
        o.n_dilate, o.n_tag, o.restart = n_dilate, n_tag, restart
        o.max_fgmres, o.max_newton = max_fgmres, max_newton
        o.inner_tol, o.newton_tol = inner_tol, newton_tol
        o.timing = int(bool(timing))
        o.block_inner_its, o.block_inner_tol = int(block_inner_its), float(block_inner_tol)
        o.refine_steps = int(refine_steps)
        if gj_tensor_cores is not None:
            o.gj_tensor_cores = int(gj_tensor_cores)
        o.rebuild_every = int(rebuild_every)
        s = stream if stream is not None else torch.cuda.current_stream()
        o.stream = ctypes.c_void_p(s.cuda_stream)
        self.stream = s
        self.options = o
        bb = (ctypes.c_double * 3)(*(list(b) + [0.0] * (3 - len(b))))
        ctx = ctypes.c_void_p()
        rc = self.lib.pns_setup(ctypes.byref(ctx), nz, ny, nx, mask.ctypes.data_as(ctypes.c_void_p),
                                labels.ctypes.data_as(ctypes.c_void_p), float(rho), float(mu), bb, float(dt),
                                ctypes.byref(o))
        if rc != 0:
            raise PnsError(rc, "pns_setup failed (bad mask/labels/parameters or CUDA error)")
        self.ctx = ctx

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.pns_destroy(ctx)
            self.ctx = None

    def close(self):
        self.__del__()

    def _check(self, rc, what):
        if rc != 0:
            raise PnsError(rc, f"{what}: {self.lib.pns_last_error(self.ctx).decode()}")

    def zeros(self):
        import torch
        return torch.zeros(self.nfull, dtype=torch.float64, device="cuda")

    # --- C-ABI calls (same names as include/pns.h)
    def info(self):
        inf = Info()
        self._check(self.lib.pns_get_info(self.ctx, ctypes.byref(inf)), "pns_get_info")
        return inf.as_dict()

    def pns_residual(self, x, x_prev=None, r=None):
        """r(x), the FP64 Newton residual (steady, or backward Euler from x_prev); CUDA tensors of the full
        layout [u_x | u_y | (u_z) | p], entries that are not unknowns ignored on input, 0 on output."""
        r = self.zeros() if r is None else r
        self._check(self.lib.pns_residual(self.ctx, _ptr(x), _ptr(x_prev), _ptr(r)), "pns_residual")
        return r

    def pns_jacobian_apply(self, x_lin, v, y=None):
        """y = J(x_lin) v, the Newton Jacobian at x_lin (upwind branches frozen there)."""
        y = self.zeros() if y is None else y
        self._check(self.lib.pns_jacobian_apply(self.ctx, _ptr(x_lin), _ptr(v), _ptr(y)), "pns_jacobian_apply")
        return y

    def pns_operator_apply(self, variant, x_lin, v, y=None):
        """y = A_b v for the build matrix of `variant` at x_lin (gplmm: the modified Jacobian of the
        inertia-free tagged faces; aplmm_ns: the Newton Jacobian; aplmm_s: the Stokes operator)."""
        y = self.zeros() if y is None else y
        var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        self._check(self.lib.pns_operator_apply(self.ctx, var, _ptr(x_lin), _ptr(v), _ptr(y)), "pns_operator_apply")
        return y

    def pns_build_precond(self, x_lin):
        """Build the context's preconditioner at the linearisation state x_lin (synchronises)."""
        self._check(self.lib.pns_build_precond(self.ctx, _ptr(x_lin)), "pns_build_precond")

    def pns_precond_apply(self, v, z=None):
        """z = M^{-1} v with the built preconditioner (FP64 in and out)."""
        z = self.zeros() if z is None else z
        self._check(self.lib.pns_precond_apply(self.ctx, _ptr(v), _ptr(z)), "pns_precond_apply")
        return z

    def pns_precond_apply_static(self, v, z=None):
        """z = M^{-1} v with no device allocation inside the call (scratch in a fixed device array)."""
        z = self.zeros() if z is None else z
        self._check(self.lib.pns_precond_apply_static(self.ctx, _ptr(v), _ptr(z)), "pns_precond_apply_static")
        return z

    def pns_autotune(self):
        """Time every local-solve shape on every block-size bin of the built preconditioner and adopt the
        fastest per bin; returns (table, ms) with ms[bin][config] (0 where a bin has no block)."""
        table = (ctypes.c_int * TUNE_BINS)()
        ms = (ctypes.c_double * (TUNE_BINS * TUNE_CONFIGS))()
        self._check(self.lib.pns_autotune(self.ctx, ctypes.cast(table, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p)),
                    "pns_autotune")
        return list(table), np.array(list(ms)).reshape(TUNE_BINS, TUNE_CONFIGS)

    def pns_set_tuning(self, table):
        """Adopt a local-solve tuning table (one config id per block-size bin)."""
        t = (ctypes.c_int * TUNE_BINS)(*[int(v) for v in table])
        self._check(self.lib.pns_set_tuning(self.ctx, ctypes.cast(t, ctypes.c_void_p)), "pns_set_tuning")

    def pns_newton_solve(self, x, x_prev=None, check=True):
        """Newton-FGMRES from the initial guess x, updated in place; returns the statistics as a dict
        (status, iterations per Newton step, residual history, build and solve times).  With
        check=False a non-converged solve returns its status instead of raising."""
        st = Stats()
        rc = self.lib.pns_newton_solve(self.ctx, _ptr(x), _ptr(x_prev), ctypes.byref(st))
        if check:
            self._check(rc, "pns_newton_solve")
        d = st.as_dict()
        d["status"] = STATUS.get(rc, rc)
        return d

    def pns_stokes_solve(self, x=None, check=True):
        """The Stokes solution (the usual Newton initial guess); returns (x, statistics)."""
        x = self.zeros() if x is None else x
        st = Stats()
        rc = self.lib.pns_stokes_solve(self.ctx, _ptr(x), ctypes.byref(st))
        if check:
            self._check(rc, "pns_stokes_solve")
        d = st.as_dict()
        d["status"] = STATUS.get(rc, rc)
        return x, d

    def pns_export_coarse(self):
        """Inverse of the coarse matrix of the built preconditioner (host, n_o x n_o)."""
        n = ctypes.c_int(0)
        self._check(self.lib.pns_export_coarse(self.ctx, None, ctypes.byref(n)), "pns_export_coarse")
        a = np.zeros((n.value, n.value), np.float64)
        self._check(self.lib.pns_export_coarse(self.ctx, a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)),
                    "pns_export_coarse")
        return a

    def pns_export_maps(self):
        """The integer maps of the context (primary grid and interface of each cell, face classes, gPLMM
        tags, dual-grid multiplicity of each unknown, pinned cells) as NumPy arrays."""
        nc, dim = self.ncell, self.dim
        cell_prim = np.zeros(nc, np.int32)
        cell_iface = np.zeros(nc, np.int32)
        face_class = np.zeros(dim * nc, np.int32)
        tags = np.zeros(dim * nc, np.uint8)
        dual_count = np.zeros((dim + 1) * nc, np.int32)
        n_pins = self.info()["n_pins"]
        pins = np.zeros(max(1, n_pins), np.int32)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._check(self.lib.pns_export_maps(self.ctx, P(cell_prim), P(cell_iface), P(face_class), P(tags),
                                             P(dual_count), P(pins)), "pns_export_maps")
        return {"cell_prim": cell_prim, "cell_iface": cell_iface, "face_class": face_class.reshape(dim, nc),
                "tags": tags.reshape(dim, nc).astype(bool), "dual_count": dual_count, "pins": pins[:n_pins]}


# ------------------------------------------------------------------------------------ learned initial guess
def unet_param_names(levels):
    """Names of the flat parameter vector of pns_unet (include/pns_unet.h), in its order: each
    convolution's weight then bias, enc0.0 .. enc{L-1}.1, dec{L-2}.0 .. dec0.1, head."""
    names = []
    for l in range(levels):
        names += [f"enc{l}.0", f"enc{l}.1"]
    for l in range(levels - 2, -1, -1):
        names += [f"dec{l}.0", f"dec{l}.1"]
    names.append("head")
    out = []
    for n in names:
        out += [n + ".w", n + ".b"]
    return out


_UNET_SIG = False


def _load_unet():
    global _UNET_SIG
    lib = load()
    if not _UNET_SIG:
        P, I, D, F, V, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, None, ctypes.c_longlong
        sig = {
            "pns_unet_create": (I, [ctypes.POINTER(P), I, P, I, I, I, I, I, I, ctypes.c_uint64, P]),
            "pns_unet_destroy": (V, [P]),
            "pns_unet_last_error": (ctypes.c_char_p, [P]),
            "pns_unet_num_params": (LL, [P]),
            "pns_unet_set_params": (I, [P, P]),
            "pns_unet_get_params": (I, [P, P]),
            "pns_unet_get_grads": (I, [P, P]),
            "pns_unet_forward": (I, [P, P, I, I, I, I, P]),
            "pns_unet_backward": (I, [P, P]),
            "pns_unet_mse": (I, [P, P, P, P, I, I, I, I, P, ctypes.POINTER(D)]),
            "pns_unet_adam": (I, [P, F, F, F, F]),
            "pns_unet_train_step": (I, [P, P, P, P, I, I, I, I, F, ctypes.POINTER(D)]),
            "pns_unet_features": (I, [P, P, P, D, I, I, I, P, I, P]),
            "pns_unet_targets": (I, [P, P, P, P, D, D, I, I, I, P, P, I]),
            "pns_unet_proposal": (I, [P, P, I, P, D, D, I, I, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _UNET_SIG = True
    return lib


def _fptr(t, dtype=None):
    import torch
    if t is None:
        return None
    want = dtype or torch.float32
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise TypeError(f"expected a contiguous {want} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class UNet:
    """The 3D U-Net of the learned Newton initial guess (include/pns_unet.h): BF16 tensor-core kernels,
    FP32 master weights, Adam.  Tensors are float32 CUDA tensors of shape (N, C, D, H, W)."""

    def __init__(self, channels=(16, 32, 64, 64), in_ch=6, out_ch=4, batch=1, shape=(64, 64, 64), seed=0,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpns needs a CUDA device")
        self.lib = _load_unet()
        self.channels, self.in_ch, self.out_ch = tuple(channels), in_ch, out_ch
        self.levels = len(channels)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        ch = (ctypes.c_int * self.levels)(*channels)
        h = ctypes.c_void_p()
        nz, ny, nx = shape
        rc = self.lib.pns_unet_create(ctypes.byref(h), self.levels, ctypes.cast(ch, ctypes.c_void_p), in_ch, out_ch,
                                      batch, nz, ny, nx, seed, ctypes.c_void_p(s.cuda_stream))
        if rc != 0:
            raise PnsError(rc, "pns_unet_create failed (bad sizes, or out of device memory)")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.pns_unet_destroy(h)
            self.h = None

    def close(self):
        self.__del__()

    def _check(self, rc, what):
        if rc != 0:
            raise PnsError(rc, f"{what}: {self.lib.pns_unet_last_error(self.h).decode()}")

    def num_params(self):
        return int(self.lib.pns_unet_num_params(self.h))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.num_params():
            raise ValueError("wrong parameter count")
        self._check(self.lib.pns_unet_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "pns_unet_set_params")

    def get_params(self):
        a = np.zeros(self.num_params(), np.float32)
        self._check(self.lib.pns_unet_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "pns_unet_get_params")
        return a

    def get_grads(self):
        a = np.zeros(self.num_params(), np.float32)
        self._check(self.lib.pns_unet_get_grads(self.h, a.ctypes.data_as(ctypes.c_void_p)), "pns_unet_get_grads")
        return a

    def forward(self, x, out=None):
        import torch
        n, c, d, hh, w = x.shape
        out = torch.empty((n, self.out_ch, d, hh, w), dtype=torch.float32, device="cuda") if out is None else out
        self._check(self.lib.pns_unet_forward(self.h, _fptr(x), n, d, hh, w, _fptr(out)), "pns_unet_forward")
        return out

    def backward(self, gout):
        self._check(self.lib.pns_unet_backward(self.h, _fptr(gout)), "pns_unet_backward")

    def mse(self, out, target, weight):
        import torch
        n, c, d, hh, w = out.shape
        g = torch.empty_like(out)
        loss = ctypes.c_double()
        self._check(self.lib.pns_unet_mse(self.h, _fptr(out), _fptr(target), _fptr(weight), n, d, hh, w, _fptr(g),
                                          ctypes.byref(loss)), "pns_unet_mse")
        return loss.value, g

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self._check(self.lib.pns_unet_adam(self.h, lr, b1, b2, eps), "pns_unet_adam")

    def train_step(self, x, target, weight, lr=1e-3):
        n, c, d, hh, w = x.shape
        loss = ctypes.c_double()
        self._check(self.lib.pns_unet_train_step(self.h, _fptr(x), _fptr(target), _fptr(weight), n, d, hh, w, lr,
                                                 ctypes.byref(loss)), "pns_unet_train_step")
        return loss.value

    def features(self, mask_u8, x_stokes, re, x, b=0):
        """Encode one image (device uint8 mask, FP64 full-layout Stokes solution) into batch entry b of x;
        returns the scales (U, P)."""
        import torch
        nz, ny, nx = mask_u8.shape
        sc = (ctypes.c_double * 2)()
        self._check(self.lib.pns_unet_features(self.h, _fptr(mask_u8, torch.uint8), _ptr(x_stokes), float(re), nz, ny,
                                               nx, _fptr(x), b, ctypes.cast(sc, ctypes.c_void_p)), "pns_unet_features")
        return sc[0], sc[1]

    def targets(self, mask_u8, x_ns, x_stokes, scales, t, w=None, b=0):
        import torch
        nz, ny, nx = mask_u8.shape
        self._check(self.lib.pns_unet_targets(self.h, _fptr(mask_u8, torch.uint8), _ptr(x_ns), _ptr(x_stokes),
                                              float(scales[0]), float(scales[1]), nz, ny, nx, _fptr(t),
                                              _fptr(w) if w is not None else None, b), "pns_unet_targets")

    def proposal(self, out, x_stokes, scales, x_out, b=0):
        nz, ny, nx = out.shape[2:]
        self._check(self.lib.pns_unet_proposal(self.h, _fptr(out), b, _ptr(x_stokes), float(scales[0]),
                                               float(scales[1]), nz, ny, nx, _ptr(x_out)), "pns_unet_proposal")
        return x_out
