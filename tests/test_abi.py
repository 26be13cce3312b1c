"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(CPU only: no compute call is made here)."""
import ctypes
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
