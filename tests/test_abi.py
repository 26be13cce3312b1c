"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(CPU only: no compute call is made here)."""
import ctypes
import functools
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hodlr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("hodlr_", "gmres_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_5337_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_call_list():
    d = _declared()
    for name in ("hodlr_build", "hodlr_factor", "hodlr_solve", "gmres_solve", "hodlr_ctx_create",
                 "hodlr_destroy", "hodlr_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_1403_5337_gb300 import hodlr as B
    assert sorted(B.SYMBOLS) == _declared()


def test_status_strings(lib):
    lib.hodlr_status_string.restype = ctypes.c_char_p
    assert lib.hodlr_status_string(0) == b"ok"
    assert b"converge" in lib.hodlr_status_string(6)


def test_ctx_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.hodlr_ctx_create.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    code = lib.hodlr_ctx_create(0, None, None, None, ctypes.byref(h))
    assert code in (1, 3)          # INVALID_ARG (no device) or CUDA_ERROR


def test_cuda_sources_target_sm103a_only():
    from paper_1403_5337_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_invalid_arguments_are_rejected_before_any_device_call():
    """Every entry point checks its arguments before it touches the device:
    NULL handles, negative counts and sizes beyond a fixed limit come back as
    status codes with a message (no GPU is needed to see them)."""
    from paper_1403_5337_gb300 import build
    from paper_1403_5337_gb300 import hodlr as B
    build.build()
    L = B.load_library()
    C = ctypes
    INVALID, RANGE = 1, 9

    def msg():
        return L.hodlr_last_error().decode()

    dummy = C.create_string_buffer(64)   # a non-NULL pointer that is never dereferenced
    mat = B._Matrix(C.cast(dummy, C.c_void_p), 64, 64, 1)
    out = C.c_void_p()
    assert L.hodlr_build(None, C.byref(mat), 16, 1e-4, 0, None, None, None, C.byref(out)) == INVALID
    assert "hodlr_build" in msg()
    assert L.hodlr_factor(None, None) == INVALID
    assert L.hodlr_solve(None, 1, None, 64, None) == INVALID
    info = B._Info()
    assert L.gmres_solve(None, C.byref(mat), 1, None, 64, None, 64, None, 1e-12, 10, 0, C.byref(info),
                         None) == INVALID
    assert "gmres_solve" in msg()
    assert L.hodlr_matvec(None, C.byref(mat), 1, None, 64, None, 64, None) == INVALID
    assert L.hodlr_factor_batched(-1, None, None) == INVALID
    assert L.gmres_solve_batched(None, 1, None, None, None, None, None, None, None, 1e-12, 10, 0, None,
                                 None) == INVALID
    outs = (C.c_void_p * 1)()
    assert L.hodlr_build_batched(None, 1, None, None, 1e-4, 0, None, None, outs) == INVALID
    # BDLR needs one graph per front: refused for batches before the context is used
    assert L.hodlr_build_batched(C.cast(dummy, C.c_void_p), 0, None, None, 1e-4, 1, None, None, outs) == INVALID
    assert "BDLR" in msg()
    st = B._Stats()
    assert L.hodlr_stats_get(None, C.byref(st)) == INVALID
    assert L.hodlr_export_level(None, 1, None, None, None, None, None, None, None) == INVALID
    assert L.hodlr_export_core(None, 0, None, None) == INVALID
    val = C.c_double()
    assert L.hodlr_precond_error(None, 4, None, 64, C.byref(val), None) == INVALID
    assert L.hodlr_launch_count(None) == INVALID
    # the allocation-free product's static scratch holds n s <= 2^19 entries
    big = B._Matrix(C.cast(dummy, C.c_void_p), 1 << 16, 1 << 16, 1)
    assert L.hodlr_matvec_noalloc(C.byref(big), 16, C.cast(dummy, C.c_void_p), 1 << 16,
                                  C.cast(dummy, C.c_void_p), 1 << 16, None) == RANGE
    assert "static scratch" in msg()
    # releasing nothing is not an error
    assert L.hodlr_destroy(None) == 0
    assert L.hodlr_ctx_destroy(None) == 0


_C_CHECK = r"""
#include "hodlr.h"
#include <stdio.h>
#include <string.h>
int main(void) {
    hodlr_opts o;
    long long launches = -1;
    hodlr_opts_default(&o);
    if (strcmp(hodlr_status_string(HODLR_OK), "ok") != 0) return 1;
    if (hodlr_launch_count(&launches) != HODLR_OK || launches < 0) return 2;
    if (hodlr_factor(NULL, NULL) != HODLR_INVALID_ARG) return 3;
    if (hodlr_last_error()[0] == '\0') return 4;
    if (hodlr_destroy(NULL) != HODLR_OK) return 5;
    printf("ok\n");
    return 0;
}
"""


def test_boundary_is_plain_c():
    """The boundary is usable from C: a C99 program including include/hodlr.h
    compiles with -Wall -Wextra -Werror, links against libhodlr.so and calls
    the entry points that need no device (status strings, option defaults,
    launch count, argument checks)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1403_5337_gb300 import build
    libpath = build.build()
    d = os.path.join(ROOT, "paper_1403_5337_gb300", "_build", "ctest")
    os.makedirs(d, exist_ok=True)
    src, exe = os.path.join(d, "abi_check.c"), os.path.join(d, "abi_check")
    with open(src, "w") as f:
        f.write(_C_CHECK)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), src,
                    "-o", exe, libpath, "-Wl,-rpath," + os.path.dirname(libpath)], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


_PTXAS_SOURCES = ("ozaki.cu", "gmres.cu", "apply.cu", "factor.cu", "aca_cluster.cu")


@functools.lru_cache(maxsize=None)
def _ptxas_all():
    """ptxas reports of the checked sources, compiled in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(_PTXAS_SOURCES)) as ex:
        return dict(zip(_PTXAS_SOURCES, ex.map(_ptxas_compile, _PTXAS_SOURCES)))


def _ptxas_report(src):
    return _ptxas_all()[src]


def _ptxas_compile(src):
    """(kernel, stack bytes, spill store bytes, spill load bytes, registers) for
    every entry function of one source, from ptxas -v (the library's flags)."""
    import subprocess
    from paper_1403_5337_gb300 import build
    d = os.path.join(ROOT, "paper_1403_5337_gb300", "_build", "ptxas")
    os.makedirs(d, exist_ok=True)
    obj = os.path.join(d, os.path.basename(src) + ".o")
    cmd = [build.nvcc(), "-c", os.path.join(build.CSRC, src), "-o", obj, "-I", build.INCLUDE, "-I", build.CSRC,
           "-Xptxas", "-v"] + build.NVCC_FLAGS + build.ARCH
    out = subprocess.run(cmd, capture_output=True, text=True, check=True).stderr
    rows, name = [], None
    for line in out.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name:
            rows.append([name, int(m.group(1)), int(m.group(2)), int(m.group(3)), None])
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and rows and rows[-1][0] == name and rows[-1][4] is None:
            rows[-1][4] = int(m.group(1))
    return rows


@pytest.mark.parametrize("src,kernels,allowed", [
    ("ozaki.cu", ("oz_tc_gemm_kernel", "oz_split_rows_kernel", "oz_split_cols_kernel", "oz_finalize_kernel"), 0),
    ("gmres.cu", ("arnoldi_tail_kernel", "residual_kernel", "start_cycle_kernel", "backsolve_kernel"), 0),
    # the double-float product at its 64-register cap (four CTAs of 256 threads
    # per SM): the variant for a general FP64 z spills 12 bytes
    ("gmres.cu", ("df_matvec_kernel",), 16),
    # the apply in chunks of 4 and 1 right-hand sides (FP32 factors, every
    # storage type); the chunk-of-2 variants and the FP64 apply spill (at most
    # 48 stores / 80 loads, 24-byte frames) and are bounded below
    ("apply.cu", ("apply_fused_kernelIffLi4", "apply_fused_kernelIf6__halfLi4",
                  "apply_fused_kernelIf13__nv_bfloat16Li4", "apply_fused_kernelIffLi1"), 0),
    ("apply.cu", ("apply_fused_kernel",), 80),
    # register-tiled Gauss-Jordan (one CTA up to 128 rows, a cluster of CTAs up to 256)
    ("factor.cu", ("gj_blocked_kernel", "gemm_batched_kernel", "gj_cluster_kernel", "core_cond_kernel",
                   "core_store_kernel", "gj_inverse_reg_kernel"), 0),
    ("aca_cluster.cu", ("aca_cluster_kernel",), 0),
])
def test_product_and_gmres_kernels_do_not_spill(src, kernels, allowed):
    """The products' and the GMRES kernels keep their state in registers for
    sm_103a: spill stores, spill loads and stack frame within `allowed` bytes."""
    rows = _ptxas_report(src)
    for k in kernels:
        found = [r for r in rows if k in r[0]]
        assert found, (k, [r[0] for r in rows])
        for name, stack, st, ld, regs in found:
            assert max(st, ld, stack) <= allowed, (name, stack, st, ld, regs)
