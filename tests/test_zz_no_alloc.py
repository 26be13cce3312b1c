"""hodlr_matvec_noalloc: the matvec for callers that may not allocate device
memory (its scratch is a fixed array inside the library).  Its results must
match hodlr_matvec, the allocating entry point, on consecutive calls -- the
fixed scratch keeps whatever the previous call left in it.

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
    assert np.all(np.abs(W - ref) <= TOL * scale)


def test_noalloc_matvec_matches_allocating_one_twice(H):
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    A = torch.as_tensor(F.A, device="cuda")
    ctx = H.Context(0)
    rng = np.random.default_rng(11)
    for s in (3, 5):          # two calls in a row, different shapes and data
        Z = torch.as_tensor(rng.standard_normal((s, F.n)), device="cuda")
        W = torch.full((s, F.n), np.nan, dtype=torch.float64, device="cuda")
        H.hodlr_matvec_noalloc(A, Z, W)
        ref = H.hodlr_matvec(ctx, A, Z)
        torch.cuda.synchronize()
        _check_close(W.cpu().numpy(), ref.cpu().numpy(), F.A, Z.cpu().numpy())
    ctx.close()


def test_noalloc_matvec_refuses_oversize(H):
    n = 1024
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    Z = torch.zeros((600, n), dtype=torch.float64, device="cuda")     # 614400 > 524288
    W = torch.zeros_like(Z)
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_matvec_noalloc(A, Z, W)
    assert e.value.code == 9
