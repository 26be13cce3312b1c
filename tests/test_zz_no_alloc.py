"""hodlr_matvec_noalloc: the matvec for callers that may not allocate device
memory (its scratch is a fixed array inside the library).

Its results must match the FP64 product computed by NumPy and hodlr_matvec,
the allocating entry point, on consecutive calls -- the fixed scratch keeps
whatever the previous call left in it, so the larger call runs first and the
smaller one after it reads a scratch array still holding the larger call's
values beyond its own size.  The calls must not change the device's free
memory.  One case passes A with an odd leading dimension (a 577-column view),
which takes the library's scalar (non-vectorised) loads.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import frontgen as fg  # noqa: E402

# the matvec tolerance of the other GPU tests: 16 * 2^-48 relative to |A| |z|
TOL = 16 * 2.0 ** -48


@pytest.fixture(scope="module")
def H():
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    return H


def _check_close(W, ref, A, Z):
    scale = (np.abs(A) @ np.abs(Z.T)).T.max(axis=1, keepdims=True)
    err = np.abs(W - ref)
    assert np.all(err <= TOL * scale), float((err / scale).max())


@pytest.mark.parametrize("odd_ld", [False, True])
def test_noalloc_matvec_matches_fp64_and_allocating_one_twice(H, odd_ld):
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    n = F.n
    if odd_ld:
        buf = torch.zeros((n, n + 1), dtype=torch.float64, device="cuda")
        buf[:, :n] = torch.as_tensor(F.A, device="cuda")
        A = buf[:, :n]                                   # ld = n + 1
        assert A.stride(0) == n + 1
    else:
        A = torch.as_tensor(F.A, device="cuda")
    ctx = H.Context(0)
    rng = np.random.default_rng(11)
    shapes = (7, 2)           # larger first: the second call reads a dirty scratch
    Zs = [torch.as_tensor(rng.standard_normal((s, n)), device="cuda") for s in shapes]
    Ws = [torch.full((s, n), np.nan, dtype=torch.float64, device="cuda") for s in shapes]
    refs = [H.hodlr_matvec(ctx, A, Z).cpu().numpy() for Z in Zs]
    # the first call on a device looks up the scratch address (and the driver
    # may load the library's device code): make it before measuring
    warm = torch.empty((1, n), dtype=torch.float64, device="cuda")
    H.hodlr_matvec_noalloc(A, Zs[1][:1].contiguous(), warm)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for Z, W in zip(Zs, Ws):  # two calls in a row
        H.hodlr_matvec_noalloc(A, Z, W)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for Z, W, ref in zip(Zs, Ws, refs):
        z = Z.cpu().numpy()
        w = W.cpu().numpy()
        _check_close(w, (F.A @ z.T).T, F.A, z)   # the FP64 product
        _check_close(w, ref, F.A, z)             # the allocating entry point
    ctx.close()


def test_noalloc_matvec_refuses_oversize(H):
    n = 1024
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    Z = torch.zeros((600, n), dtype=torch.float64, device="cuda")     # 614400 > 524288
    W = torch.zeros_like(Z)
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_matvec_noalloc(A, Z, W)
    assert e.value.code == 9
