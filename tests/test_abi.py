"""The C-ABI library loads and exports every entry point that the headers under include/ declare (no GPU
and no compute calls needed)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pns_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pns_setup", "pns_residual", "pns_jacobian_apply", "pns_precond_apply", "pns_newton_solve",
              "pns_build_precond", "pns_stokes_solve", "pns_export_maps", "pns_destroy", "pns_last_error",
              "pns_unet_create", "pns_unet_forward", "pns_unet_backward", "pns_unet_train_step", "pns_unet_proposal"]:
        assert n in names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2510_22077_gb300 import build, pns
    if not os.path.exists(pns.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libpns")
        build.build()
    return pns.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pns_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_with_ctypes(lib_path):
    import ctypes
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n)
    # pure host call: default options
    from paper_2510_22077_gb300 import pns
    pns._lib = None
    o = pns.default_options()
    assert o.restart == 100 and o.periodic[0] == 1 and abs(o.newton_tol - 1e-8) < 1e-20


def test_product_path_fails_loudly_without_a_device(lib_path):
    """No CPU fallback: without a CUDA device the binding refuses to build a solver, and the C ABI's
    pns_setup returns an error code (no context) instead of computing anything on the host."""
    import ctypes

    import numpy as np
    import torch

    from paper_2510_22077_gb300 import pns
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    mask = np.ones((1, 4, 8), np.uint8)
    labels = np.ones((1, 4, 8), np.int32)
    with pytest.raises(RuntimeError):
        pns.Solver(mask, labels, 1.0, 1.0, (1.0, 0.0, 0.0))
    lib = pns.load()
    opt = pns.default_options()
    ctx = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(1.0, 0.0, 0.0)
    rc = lib.pns_setup(ctypes.byref(ctx), 1, 4, 8, mask.ctypes.data_as(ctypes.c_void_p),
                       labels.ctypes.data_as(ctypes.c_void_p), 1.0, 1.0, b, 0.0, ctypes.byref(opt))
    assert rc != 0 and not ctx.value


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of pns_options, pns_stats and pns_info have the C layout of include/pns.h: the same
    size and every field at the same offset (a C program compiled against the header prints them)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2510_22077_gb300 import pns
    structs = {"pns_options": pns.Options, "pns_stats": pns.Stats, "pns_info": pns.Info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pns.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes_sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)
