"""Thin Python binding of libhodlr (ctypes): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts torch
tensors to pointers, torch streams to cudaStream_t and status codes to
exceptions.  Device memory of the library comes from torch's caching allocator.

Conventions: A is an (n, n) float64 CUDA tensor in tree order (row-major,
contiguous or with a row stride); right-hand sides and solutions are (s, n)
float64 CUDA tensors, i.e. n x s column-major with ld = n (a 1-D (n,) tensor is
one right-hand side).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_PKG, "libhodlr.so")

FP64, FP32, BF16, FP16 = 0, 1, 2, 3
ACA, BDLR = 0, 1
_PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16}
_METHOD = {"aca": ACA, "bdlr": BDLR}
MAX_LEVELS = 16

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA_ERROR", 4: "SINGULAR",
          5: "NOT_FACTORED", 6: "NOT_CONVERGED", 7: "TIMEOUT", 8: "NONFINITE_INPUT", 9: "RANGE"}


class HodlrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class NotConverged(HodlrError):
    pass


class _Matrix(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n", C.c_int64), ("ld", C.c_int64), ("symmetric", C.c_int)]


class _Graph(C.Structure):
    _fields_ = [("rowptr", C.c_void_p), ("colind", C.c_void_p), ("n", C.c_int64)]


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("compress_precision", C.c_int), ("rank_cap", C.c_int),
                ("bdlr_depth", C.c_int), ("core_cond_threshold", C.c_double),
                ("leaf_bounds", C.c_void_p), ("n_leaf_bounds", C.c_int), ("seed", C.c_uint64),
                ("defer_factor", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int), ("leaf_max", C.c_int),
                ("rank_max", C.c_int * MAX_LEVELS), ("rank_pad", C.c_int * MAX_LEVELS),
                ("rank_mean", C.c_double * MAX_LEVELS), ("cap", C.c_int * MAX_LEVELS),
                ("cap_hit", C.c_int), ("bytes_factors", C.c_int64), ("factored", C.c_int),
                ("ms_compress", C.c_double), ("ms_factor", C.c_double),
                ("core_cond_max", C.c_double * MAX_LEVELS), ("cores_promoted", C.c_int * MAX_LEVELS),
                ("core_cond_threshold", C.c_double), ("bdlr_depth_max", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_void_p), ("est_relres", C.c_void_p), ("true_relres", C.c_void_p),
                ("restarts", C.c_int), ("ms_total", C.c_double)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# every exported symbol of include/hodlr.h
SYMBOLS = ["hodlr_ctx_create", "hodlr_ctx_destroy", "hodlr_opts_default", "hodlr_build", "hodlr_factor",
           "hodlr_solve", "gmres_solve", "hodlr_matvec", "hodlr_matvec_noalloc", "hodlr_precond_error",
           "hodlr_stats_get",
           "hodlr_export_level", "hodlr_export_core", "hodlr_export_core_cond", "hodlr_destroy", "hodlr_status_string",
           "hodlr_last_error", "hodlr_launch_count", "hodlr_build_batched", "hodlr_factor_batched",
           "gmres_solve_batched", "hodlr_ctx_set_wait_test", "hodlr_ctx_set_apply_path", "hodlr_profile_enable", "hodlr_profile_read",
           "hodlr_build_diag", "hodlr_dense_lu_solve", "hodlr_save", "hodlr_load"]

_lib = None
# Library calls in progress on this process.  The torch allocator callbacks run
# Python code inside a library call, which may trigger garbage collection; a
# Hodlr collected then must not re-enter the library, so its destruction is
# deferred to the end of the outermost call.
_depth = 0
_deferred = []


class _Call:
    def __enter__(self):
        global _depth
        _depth += 1

    def __exit__(self, *exc):
        global _depth
        _depth -= 1
        if _depth == 0:
            while _deferred:
                _lib.hodlr_destroy(_deferred.pop())
        return False


def load_library(path: str = _LIBPATH):
    """Load libhodlr.so (raises if it was not built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhodlr.so not found at {path}: run paper_1403_5337_gb300.build.build() first")
    lib = C.CDLL(path)
    vp, i64, ci, cd = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.hodlr_ctx_create.argtypes = [ci, _ALLOC, _FREE, vp, C.POINTER(vp)]
    lib.hodlr_ctx_destroy.argtypes = [vp]
    lib.hodlr_opts_default.argtypes = [C.POINTER(_Opts)]
    lib.hodlr_opts_default.restype = None
    lib.hodlr_build.argtypes = [vp, C.POINTER(_Matrix), ci, cd, ci, C.POINTER(_Graph), C.POINTER(_Opts), vp,
                                C.POINTER(vp)]
    lib.hodlr_factor.argtypes = [vp, vp]
    lib.hodlr_build_diag.argtypes = [vp, C.POINTER(_Matrix), vp, C.POINTER(vp)]
    lib.hodlr_save.argtypes = [vp, vp, C.c_size_t, C.POINTER(C.c_size_t), vp]
    lib.hodlr_load.argtypes = [vp, C.POINTER(_Matrix), vp, C.c_size_t, vp, C.POINTER(vp)]
    lib.hodlr_dense_lu_solve.argtypes = [vp, C.POINTER(_Matrix), ci, vp, i64, vp, i64, vp]
    lib.hodlr_solve.argtypes = [vp, ci, vp, i64, vp]
    lib.gmres_solve.argtypes = [vp, C.POINTER(_Matrix), ci, vp, i64, vp, i64, vp, cd, ci, ci, C.POINTER(_Info), vp]
    lib.hodlr_matvec.argtypes = [vp, C.POINTER(_Matrix), ci, vp, i64, vp, i64, vp]
    lib.hodlr_matvec_noalloc.argtypes = [C.POINTER(_Matrix), ci, vp, i64, vp, i64, vp]
    lib.hodlr_precond_error.argtypes = [vp, ci, vp, i64, C.POINTER(cd), vp]
    lib.hodlr_stats_get.argtypes = [vp, C.POINTER(_Stats)]
    lib.hodlr_export_level.argtypes = [vp, ci, vp, vp, vp, vp, vp, vp, vp]
    lib.hodlr_export_core.argtypes = [vp, ci, vp, vp]
    lib.hodlr_export_core_cond.argtypes = [vp, ci, vp, vp, vp]
    lib.hodlr_destroy.argtypes = [vp]
    lib.hodlr_launch_count.argtypes = [C.POINTER(C.c_longlong)]
    lib.hodlr_ctx_set_wait_test.argtypes = [vp, C.c_ulonglong, ci]
    lib.hodlr_ctx_set_apply_path.argtypes = [vp, ci]
    lib.hodlr_profile_enable.argtypes = [ci]
    lib.hodlr_profile_read.argtypes = [C.c_char_p, C.POINTER(cd), C.POINTER(C.c_longlong)]
    lib.hodlr_build_batched.argtypes = [vp, ci, C.POINTER(_Matrix), C.POINTER(ci), cd, ci, C.POINTER(_Opts), vp,
                                        C.POINTER(vp)]
    lib.hodlr_factor_batched.argtypes = [ci, C.POINTER(vp), vp]
    lib.gmres_solve_batched.argtypes = [vp, ci, C.POINTER(_Matrix), C.POINTER(ci), C.POINTER(vp), C.POINTER(i64),
                                        C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), cd, ci, ci, C.POINTER(_Info),
                                        vp]
    lib.hodlr_status_string.argtypes = [ci]
    lib.hodlr_status_string.restype = C.c_char_p
    lib.hodlr_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        fn = getattr(lib, name)
        if name not in ("hodlr_opts_default", "hodlr_status_string", "hodlr_last_error"):
            fn.restype = ci
    _lib = _GuardedLib(lib)
    return _lib


class _GuardedLib:
    """The loaded library with every call bracketed by _Call (see above)."""

    def __init__(self, lib):
        self._raw = lib
        for name in SYMBOLS:
            fn = getattr(lib, name)
            setattr(self, name, self._guard(fn))

    @staticmethod
    def _guard(fn):
        def call(*args):
            with _Call():
                return fn(*args)
        return call


def _check(code):
    if code != 0:
        msg = _lib.hodlr_last_error().decode(errors="replace")
        if code == 6:
            raise NotConverged(code, msg)
        raise HodlrError(code, msg)


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream):
    if stream is None:
        if _raw_stream is not None:   # the current stream's handle without a Stream object
            return C.c_void_p(_raw_stream(torch.cuda.current_device()))
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


_default_opts = None


def _opts() -> "_Opts":
    """A fresh copy of the library's default options (read from it once)."""
    global _default_opts
    if _default_opts is None:
        o = _Opts()
        load_library().hodlr_opts_default(C.byref(o))
        _default_opts = bytes(o)
    return _Opts.from_buffer_copy(_default_opts)


def _mat(A: torch.Tensor, symmetric: bool) -> _Matrix:
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square float64 CUDA tensor")
    if A.stride(1) != 1:
        raise ValueError("A must be row-major (stride(1) == 1)")
    return _Matrix(A.data_ptr(), A.shape[0], A.stride(0), 1 if symmetric else 0)


def _rhs(X: torch.Tensor, n: int):
    """(s, n) or (n,) float64 CUDA tensor -> (pointer, s, ld)."""
    if X.dtype != torch.float64 or not X.is_cuda:
        raise ValueError("right-hand sides must be float64 CUDA tensors")
    if X.dim() == 1:
        if X.shape[0] != n or X.stride(0) != 1:
            raise ValueError("vector length / stride mismatch")
        return X.data_ptr(), 1, n
    if X.shape[1] != n or (X.stride(1) != 1 and n > 1):
        raise ValueError("right-hand sides must be an (s, n) tensor with unit stride along n")
    # the stride of a size-1 dimension is arbitrary: use n
    ld = X.stride(0) if X.shape[0] > 1 else n
    if X.shape[0] > 1 and ld < n:
        raise ValueError("right-hand sides overlap (row stride < n)")
    return X.data_ptr(), X.shape[0], ld


class Context:
    """A libhodlr context on one CUDA device; library memory comes from torch."""

    def __init__(self, device: int = 0, torch_allocator: bool = True):
        lib = load_library()
        self.device = device
        self._keep = []
        if torch_allocator:
            def _a(nbytes, user, stream):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
                except Exception:
                    return None

            def _f(ptr, nbytes, user, stream):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = _ALLOC(_a)
            self._free = _FREE(_f)
        else:
            self._alloc = _ALLOC()
            self._free = _FREE()
        h = C.c_void_p()
        _check(lib.hodlr_ctx_create(device, self._alloc, self._free, None, C.byref(h)))
        self.handle = h

    def set_wait_test(self, spin_limit: int = 0, unreachable: bool = False):
        """Test hook of the bounded device waits (see include/hodlr.h)."""
        _check(_lib.hodlr_ctx_set_wait_test(self.handle, int(spin_limit), 1 if unreachable else 0))

    def set_apply_path(self, path: int = 0):
        """0: automatic, 1: one cooperative launch, 2: one launch per phase
        (include/hodlr.h, hodlr_ctx_set_apply_path)."""
        _check(_lib.hodlr_ctx_set_apply_path(self.handle, int(path)))

    def close(self):
        if self.handle:
            _lib.hodlr_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class GmresInfo:
    iters: np.ndarray
    est_relres: np.ndarray
    true_relres: np.ndarray
    restarts: int
    ms_total: float
    converged: bool


class Hodlr:
    """A compressed (and, after hodlr_factor, factored) HODLR matrix."""

    def __init__(self, ctx: Context, handle, A: torch.Tensor, keep):
        self.ctx = ctx
        self.handle = handle
        self.A = A          # the library keeps a pointer to A: keep it alive
        self._keep = keep
        self.n = int(A.shape[0]) if A is not None else self.stats()["n"]

    def stats(self) -> dict:
        st = _Stats()
        _check(_lib.hodlr_stats_get(self.handle, C.byref(st)))
        L = st.levels
        return dict(n=st.n, levels=L, leaf_max=st.leaf_max, rank_max=list(st.rank_max[:L]),
                    rank_pad=list(st.rank_pad[:L]), rank_mean=list(st.rank_mean[:L]), cap=list(st.cap[:L]),
                    cap_hit=bool(st.cap_hit), bytes_factors=st.bytes_factors, factored=bool(st.factored),
                    ms_compress=st.ms_compress, ms_factor=st.ms_factor,
                    core_cond_max=list(st.core_cond_max[:L]), cores_promoted=list(st.cores_promoted[:L]),
                    core_cond_threshold=st.core_cond_threshold, bdlr_depth_max=st.bdlr_depth_max)

    def export_level(self, level: int, stream=None):
        """(U, V, ranks, piv_rows, piv_cols) of level `level` as numpy arrays."""
        s = self.stats()
        n, rp, cap = s["n"], s["rank_pad"][level - 1], s["cap"][level - 1]
        U = np.zeros((rp, n))
        V = np.zeros((rp, n))
        ranks = np.zeros(1 << level, dtype=np.int32)
        pr = np.zeros((1 << level, cap), dtype=np.int32)
        pc = np.zeros((1 << level, cap), dtype=np.int32)
        _check(_lib.hodlr_export_level(self.handle, level, U.ctypes.data, None, V.ctypes.data, ranks.ctypes.data,
                                       pr.ctypes.data, pc.ctypes.data, _stream(stream)))
        return U.T.copy(), V.T.copy(), ranks, pr, pc

    def export_d(self, level: int, stream=None):
        """d = K_node^-1 U_node of level `level` (n x rank_pad), after the factorisation."""
        s = self.stats()
        n, rp = s["n"], s["rank_pad"][level - 1]
        d = np.zeros((rp, n))
        _check(_lib.hodlr_export_level(self.handle, level, None, d.ctypes.data, None, None, None, None,
                                       _stream(stream)))
        return d.T.copy()

    def export_core(self, level: int, stream=None):
        s = self.stats()
        rp = s["rank_pad"][level]
        out = np.zeros(((1 << level), 2 * rp, 2 * rp))
        _check(_lib.hodlr_export_core(self.handle, level, out.ctypes.data, _stream(stream)))
        return np.transpose(out, (0, 2, 1)).copy()   # column-major blocks -> [i][row][col]

    def export_core_cond(self, level: int, stream=None):
        """(kappa_1 of each core of level `level`, re-inverted-in-FP64 flags)."""
        cond = np.zeros(1 << level)
        flag = np.zeros(1 << level, dtype=np.int32)
        _check(_lib.hodlr_export_core_cond(self.handle, level, cond.ctypes.data, flag.ctypes.data,
                                           _stream(stream)))
        return cond, flag.astype(bool)

    def close(self):
        if self.handle and self.ctx is not None and not self.ctx.handle:
            # the context is gone, and the device memory with it: nothing to release
            self.handle = None
            return
        if self.handle:
            if _depth > 0:
                _deferred.append(self.handle)
            else:
                with _Call():
                    _lib.hodlr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hodlr_build(ctx: Context, A: torch.Tensor, leaf: int, tol: float, method: str = "aca", graph=None,
                precision: str = "fp32", compress_precision: str | None = None, rank_cap: int = 0,
                bdlr_depth: int = -1, leaf_bounds=None, symmetric: bool = True, stream=None,
                defer_factor: bool = False, core_cond_threshold: float = 0.0) -> Hodlr:
    """Compress A into HODLR form (Sec. 4.3 step 1, Sec. 5) and, unless
    defer_factor, factor it level by level meanwhile: see include/hodlr.h."""
    lib = load_library()
    mat = _mat(A, symmetric)
    o = _opts()
    o.precision = _PREC[precision]
    o.compress_precision = -1 if compress_precision is None else _PREC[compress_precision]
    o.rank_cap = rank_cap
    o.bdlr_depth = bdlr_depth
    o.defer_factor = 1 if defer_factor else 0
    o.core_cond_threshold = float(core_cond_threshold)
    keep = []
    if leaf_bounds is not None:
        lb = np.ascontiguousarray(np.asarray(leaf_bounds, dtype=np.int64))
        keep.append(lb)
        o.leaf_bounds = lb.ctypes.data
        o.n_leaf_bounds = lb.shape[0]
    gp = None
    if graph is not None and method == "bdlr":   # only BDLR reads the graph
        rp = np.ascontiguousarray(np.asarray(graph[0], dtype=np.int32))
        ci = np.ascontiguousarray(np.asarray(graph[1], dtype=np.int32))
        keep += [rp, ci]
        gp = C.byref(_Graph(rp.ctypes.data, ci.ctypes.data, A.shape[0]))
    h = C.c_void_p()
    _check(lib.hodlr_build(ctx.handle, C.byref(mat), int(leaf), float(tol), _METHOD[method], gp, C.byref(o),
                           _stream(stream), C.byref(h)))
    return Hodlr(ctx, h, A, keep)


def hodlr_build_diag(ctx: Context, A: torch.Tensor, symmetric: bool = True, stream=None) -> Hodlr:
    """The diagonal (Jacobi) preconditioner of the paper's comparison (Fig. 8):
    a handle that gmres_solve and hodlr_solve take like a HODLR matrix."""
    lib = load_library()
    mat = _mat(A, symmetric)
    h = C.c_void_p()
    _check(lib.hodlr_build_diag(ctx.handle, C.byref(mat), _stream(stream), C.byref(h)))
    return Hodlr(ctx, h, A, [])


def hodlr_dense_lu_solve(ctx: Context, A: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """The paper's dense LU comparator (Table 3): X = A^-1 B by partial-pivoting
    LU on the GPU; B is (s, n) or (n,)."""
    lib = load_library()
    mat = _mat(A, False)
    bptr, s, ldb = _rhs(B, A.shape[0])
    X = torch.empty_like(B, memory_format=torch.contiguous_format)
    xptr, _, ldx = _rhs(X, A.shape[0])
    _check(lib.hodlr_dense_lu_solve(ctx.handle, C.byref(mat), s, C.c_void_p(bptr), ldb, C.c_void_p(xptr), ldx,
                                    _stream(stream)))
    return X


def hodlr_save(h: Hodlr, stream=None) -> bytes:
    """The checkpoint image of a factored HODLR matrix (host bytes)."""
    need = C.c_size_t(0)
    _check(_lib.hodlr_save(h.handle, None, 0, C.byref(need), _stream(stream)))
    buf = (C.c_char * need.value)()
    _check(_lib.hodlr_save(h.handle, buf, need.value, C.byref(need), _stream(stream)))
    return bytes(buf)


def hodlr_load(ctx: Context, image: bytes, A: torch.Tensor | None = None, symmetric: bool = True,
               stream=None) -> Hodlr:
    """Restore a HODLR matrix from hodlr_save's image (A optional: only
    hodlr_precond_error needs it)."""
    lib = load_library()
    mat = C.byref(_mat(A, symmetric)) if A is not None else None
    h = C.c_void_p()
    _check(lib.hodlr_load(ctx.handle, mat, image, len(image), _stream(stream), C.byref(h)))
    return Hodlr(ctx, h, A, [])


def hodlr_factor(h: Hodlr, stream=None) -> None:
    """Recursive Woodbury factorisation (Sec. 4.3 steps 2-5)."""
    _check(_lib.hodlr_factor(h.handle, _stream(stream)))


def hodlr_solve(h: Hodlr, X: torch.Tensor, stream=None) -> torch.Tensor:
    """X <- K~^-1 X in place (Sec. 4.3 Solve); X is (s, n) or (n,)."""
    ptr, s, ld = _rhs(X, h.n)
    _check(_lib.hodlr_solve(h.handle, s, C.c_void_p(ptr), ld, _stream(stream)))
    return X


def hodlr_matvec(ctx: Context, A: torch.Tensor, Z: torch.Tensor, symmetric: bool = True, stream=None):
    """W = A Z, FP64-accurate; Z is (s, n) or (n,).  Fewer than 16 right-hand
    sides (or n < 256): the double-float product on the FP32 pipes; otherwise the
    exact digit-slice product on the BF16 tensor cores."""
    mat = _mat(A, symmetric)
    ptr, s, ld = _rhs(Z, A.shape[0])
    W = torch.empty_like(Z, memory_format=torch.contiguous_format)
    _check(_lib.hodlr_matvec(ctx.handle, C.byref(mat), s, C.c_void_p(ptr), ld, C.c_void_p(W.data_ptr()),
                             A.shape[0], _stream(stream)))
    return W


def hodlr_matvec_noalloc(A: torch.Tensor, Z: torch.Tensor, W: torch.Tensor, symmetric: bool = True,
                         stream=None) -> torch.Tensor:
    """W = A Z into a caller-provided W, allocating nothing on the device (the
    library's fixed scratch holds n * s <= 524288 entries); Z, W are (s, n)."""
    lib = load_library()
    mat = _mat(A, symmetric)
    ptr, s, ld = _rhs(Z, A.shape[0])
    wptr, s2, ldw = _rhs(W, A.shape[0])
    if s2 != s:
        raise ValueError("W and Z differ in the number of columns")
    _check(lib.hodlr_matvec_noalloc(C.byref(mat), s, C.c_void_p(ptr), ld, C.c_void_p(wptr), ldw,
                                    _stream(stream)))
    return W


def gmres_solve(ctx: Context, A: torch.Tensor, B: torch.Tensor, P: Hodlr | None = None, tol: float = 1e-12,
                max_iter: int = 1000, restart: int = 0, X: torch.Tensor | None = None, symmetric: bool = True,
                stream=None, raise_on_fail: bool = False):
    """GMRES with right preconditioner P^-1 (Sec. 3).  Returns (X, GmresInfo)."""
    mat = _mat(A, symmetric)
    n = A.shape[0]
    bptr, s, ldb = _rhs(B, n)
    if X is None:
        X = torch.empty_like(B, memory_format=torch.contiguous_format)
    xptr, s2, ldx = _rhs(X, n)
    if s2 != s:
        raise ValueError("X and B differ in the number of right-hand sides")
    it = np.zeros(s, dtype=np.int32)
    est = np.zeros(s)
    tr = np.zeros(s)
    info = _Info(it.ctypes.data, est.ctypes.data, tr.ctypes.data, 0, 0.0)
    code = _lib.gmres_solve(ctx.handle, C.byref(mat), s, C.c_void_p(bptr), ldb, C.c_void_p(xptr), ldx,
                            P.handle if P is not None else None, float(tol), int(max_iter), int(restart),
                            C.byref(info), _stream(stream))
    if code not in (0, 6) or (code == 6 and raise_on_fail):
        _check(code)
    return X, GmresInfo(it, est, tr, info.restarts, info.ms_total, code == 0)


def hodlr_build_batched(ctx: Context, As, leaves, tol: float, method: str = "aca", precision: str = "fp32",
                        rank_cap: int = 0, symmetric: bool = True, stream=None, core_cond_threshold: float = 0.0):
    """Compress every front of a batch (list of (n_f, n_f) FP64 device tensors):
    one HODLR matrix per front, same tol and options (include/hodlr.h)."""
    lib = load_library()
    nf = len(As)
    mats = (_Matrix * max(nf, 1))(*[_mat(A, symmetric) for A in As])
    lv = (C.c_int * max(nf, 1))(*[int(x) for x in leaves])
    o = _opts()
    o.precision = _PREC[precision]
    o.rank_cap = rank_cap
    o.core_cond_threshold = float(core_cond_threshold)
    out = (C.c_void_p * max(nf, 1))()
    _check(lib.hodlr_build_batched(ctx.handle, nf, mats, lv, float(tol), _METHOD[method], C.byref(o),
                                   _stream(stream), out))
    return [Hodlr(ctx, C.c_void_p(out[f]), As[f], []) for f in range(nf)]


def hodlr_factor_batched(hs, stream=None) -> None:
    """hodlr_factor of every HODLR matrix in the list."""
    nf = len(hs)
    arr = (C.c_void_p * max(nf, 1))(*[h.handle.value if isinstance(h.handle, C.c_void_p) else h.handle
                                     for h in hs])
    _check(_lib.hodlr_factor_batched(nf, arr, _stream(stream)))


def gmres_solve_batched(ctx: Context, As, Bs, Ps=None, tol: float = 1e-12, max_iter: int = 1000,
                        restart: int = 0, symmetric: bool = True, stream=None):
    """GMRES for every front f: A_f X_f = B_f (B_f is (s_f, n_f) or (n_f,)).
    Returns a list of (X_f, GmresInfo)."""
    nf = len(As)
    mats = (_Matrix * max(nf, 1))(*[_mat(A, symmetric) for A in As])
    Xs, infos, keep = [], [], []
    sv = (C.c_int * max(nf, 1))()
    bp = (C.c_void_p * max(nf, 1))()
    xp = (C.c_void_p * max(nf, 1))()
    lb = (C.c_int64 * max(nf, 1))()
    lx = (C.c_int64 * max(nf, 1))()
    pp = (C.c_void_p * max(nf, 1))()
    inf = (_Info * max(nf, 1))()
    for f in range(nf):
        n = As[f].shape[0]
        bptr, s, ldb = _rhs(Bs[f], n)
        X = torch.empty_like(Bs[f], memory_format=torch.contiguous_format)
        xptr, _, ldx = _rhs(X, n)
        it, est, tr = np.zeros(s, dtype=np.int32), np.zeros(s), np.zeros(s)
        keep.append((it, est, tr))
        sv[f], bp[f], xp[f], lb[f], lx[f] = s, bptr, xptr, ldb, ldx
        pp[f] = Ps[f].handle if Ps is not None and Ps[f] is not None else None
        inf[f] = _Info(it.ctypes.data, est.ctypes.data, tr.ctypes.data, 0, 0.0)
        Xs.append(X)
    code = _lib.gmres_solve_batched(ctx.handle, nf, mats, sv, bp, lb, xp, lx, pp if Ps is not None else None,
                                    float(tol), int(max_iter), int(restart), inf, _stream(stream))
    if code not in (0, 6):
        _check(code)
    out = []
    for f in range(nf):
        it, est, tr = keep[f]
        out.append((Xs[f], GmresInfo(it, est, tr, inf[f].restarts, inf[f].ms_total,
                                     bool(np.all(tr <= tol)))))
    return out


def hodlr_launch_count() -> int:
    """Kernels launched by libhodlr in this process so far (see include/hodlr.h)."""
    lib = load_library()
    out = C.c_longlong(0)
    _check(lib.hodlr_launch_count(C.byref(out)))
    return int(out.value)


def hodlr_precond_error(h: Hodlr, Omega: torch.Tensor, stream=None) -> float:
    """||(I - P^-1 A) Omega||_F / ||Omega||_F for a (k, n) probe block Omega."""
    ptr, k, ld = _rhs(Omega, h.n)
    out = C.c_double()
    _check(_lib.hodlr_precond_error(h.handle, k, C.c_void_p(ptr), ld, C.byref(out), _stream(stream)))
    return out.value


def hodlr_profile_enable(on: bool = True) -> None:
    """Switch the library's per-kernel event timing on or off (clears it)."""
    _check(load_library().hodlr_profile_enable(1 if on else 0))


def hodlr_profile_read(kernel: str):
    """(total ms, launches) recorded for `kernel` since profiling was enabled."""
    ms = C.c_double()
    cnt = C.c_longlong()
    _check(load_library().hodlr_profile_read(kernel.encode(), C.byref(ms), C.byref(cnt)))
    return ms.value, int(cnt.value)
