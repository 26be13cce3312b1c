"""HODLR-preconditioned GMRES for dense frontal matrices on GB300 (sm_103a).

The solver of Aminfar, Ambikasaran and Darve (arXiv:1403.5337): HODLR compression
by ACA or BDLR, the recursive Woodbury factorisation and its solve, and GMRES
with the HODLR solve as preconditioner -- all in the CUDA library libhodlr.so,
reached through the ctypes binding in `hodlr`.
"""
from .hodlr import (ACA, BDLR, BF16, FP16, FP32, FP64, Context, GmresInfo, Hodlr, HodlrError,  # noqa: F401
                    NotConverged, gmres_solve, hodlr_build, hodlr_factor, hodlr_matvec,
                    hodlr_launch_count, hodlr_matvec_noalloc, hodlr_precond_error, hodlr_solve,
                    hodlr_build_batched, hodlr_factor_batched, gmres_solve_batched, load_library,
                    hodlr_profile_enable, hodlr_profile_read, hodlr_build_diag, hodlr_dense_lu_solve,
                    hodlr_save, hodlr_load)
