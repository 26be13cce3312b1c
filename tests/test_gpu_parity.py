"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic):
* FP64 compression forms every residual with the same round-to-nearest
  multiply/subtract sequence as the oracle, so pivots, ranks and U, V agree
  exactly up to the norm recurrence's summation order: 1e-12 relative.
* FP64 factor / solve: different (blocked, level-synchronous) order of the same
  algebra, explicit inverses instead of LU solves: 1e-10 relative (cond(K~) of the
  test fronts is below 1e3, FP64 unit roundoff 1.1e-16, with a margin).
* FP32 factor / solve: 2e-4 relative (FP32 unit roundoff 6e-8 times cond ~1e3).
* GMRES: the true FP64 relative residual <= 1e-12 on both sides; iterates agree
  to cond * 1e-12 (1e-9 here); iteration counts within 1 (FP64) or 2 (FP32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import frontgen as fg  # noqa: E402
from oracle import hodlr_oracle as O  # noqa: E402


@pytest.fixture(scope="module")
def H():
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    return H


@pytest.fixture(scope="module")
def ctx(H):
    c = H.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def front576():
    return fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)


@pytest.fixture(scope="module")
def front4096():
    F = fg.make_front(64, 64, 32, 32, "lognormal", 0.5, leaf=128, seed=0, device="cuda", cache=True)
    F.A = F.A.cpu().numpy()
    return F


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _oracle_block(blocks, l, i):
    """(U, V, rows, cols) of node i of level l's block A(node, sibling)."""
    b = blocks[(l - 1, i // 2)]
    if i % 2 == 0:
        return b.Ua, b.Vab, b.info_ab
    return b.Ub, b.Vba, b.info_ba


def _compare_compression(h, F, blocks, tree, rtol, exact_pivots=True):
    for l in range(1, tree.L + 1):
        U, V, ranks, pr, pc = h.export_level(l)
        for i in range(1 << l):
            Uo, Vo, info = _oracle_block(blocks, l, i)
            k = Uo.shape[1]
            assert ranks[i] == k, (l, i, ranks[i], k)
            r0, r1 = tree.range(l, i)
            c0, c1 = tree.range(l, i ^ 1)
            if exact_pivots:
                if isinstance(info, O.ACAResult):
                    rows, cols = list(info.rows), list(info.cols)
                else:
                    rows, cols = [v - r0 for v in info.Ir], [v - c0 for v in info.Jr]
                assert pr[i, :k].tolist() == rows, (l, i)
                assert pc[i, :k].tolist() == cols, (l, i)
            Ug = U[r0:r1, :k]
            Vg = V[c0:c1, :k]
            scale_u = max(np.abs(Uo).max(), 1e-300) if k else 1.0
            scale_v = max(np.abs(Vo).max(), 1e-300) if k else 1.0
            assert np.abs(Ug - Uo).max() <= rtol * scale_u, (l, i)
            assert np.abs(Vg - Vo).max() <= rtol * scale_v, (l, i)
            # padding columns are zero
            assert not np.any(U[r0:r1, k:]) and not np.any(V[c0:c1, k:])


@pytest.mark.parametrize("cprec,dtype,rtol", [("fp64", np.float64, 1e-12), ("fp32", np.float32, 2e-6)])
def test_aca_matches_oracle(H, ctx, front576, cprec, dtype, rtol):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks = O.build(F.A, tree, "aca", 1e-6, symmetric=True, dtype=dtype)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp64", compress_precision=cprec)
    _compare_compression(h, F, blocks, tree, rtol)
    h.close()


@pytest.mark.parametrize("cprec,dtype,rtol", [("fp64", np.float64, 1e-10), ("fp32", np.float32, 1e-3)])
def test_bdlr_matches_oracle(H, ctx, front576, cprec, dtype, rtol):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    g = (F.rowptr, F.colind)
    blocks = O.build(F.A, tree, "bdlr", 1e-4, graph=g, depth=4, dtype=dtype)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-4, "bdlr", graph=g, precision="fp64", compress_precision=cprec,
                      bdlr_depth=4)
    _compare_compression(h, F, blocks, tree, rtol)
    h.close()


@pytest.mark.parametrize("cprec,dtype,rtol", [("fp64", np.float64, 1e-10), ("fp32", np.float32, 1e-3)])
@pytest.mark.parametrize("tol", [1e-3, 1e-6])
def test_adaptive_bdlr_matches_oracle(H, ctx, front576, cprec, dtype, rtol, tol):
    """The adaptive pseudo-skeleton (Sec. 5.3, bdlr_depth = -2): every block
    grows its depth until the held-out error meets tol; the selected pivots and
    ranks of every block equal the oracle's, and so does the largest depth."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    g = (F.rowptr, F.colind)
    blocks = O.build(F.A, tree, "bdlr", tol, graph=g, depth=-2, dtype=dtype)
    dmax = 0
    for (l, i) in blocks:
        a, b = range(*tree.range(l + 1, 2 * i)), range(*tree.range(l + 1, 2 * i + 1))
        for rows, cols in ((a, b), (b, a)):
            _, d, _ = O.bdlr_adaptive(F.A, g[0], g[1], rows, cols, tol, 1, 1 << 30, dtype)
            dmax = max(dmax, d)
    h = H.hodlr_build(ctx, _dev(F.A), 64, tol, "bdlr", graph=g, precision="fp64", compress_precision=cprec,
                      bdlr_depth=-2)
    _compare_compression(h, F, blocks, tree, rtol)
    assert h.stats()["bdlr_depth_max"] == dmax
    h.close()


def test_aca_nonsymmetric_column_reads(H, ctx, front576):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    rng = np.random.default_rng(0)
    A = F.A + 0.01 * np.triu(rng.standard_normal(F.A.shape), 1)   # not symmetric
    blocks = O.build(A, tree, "aca", 1e-6)
    h = H.hodlr_build(ctx, _dev(A), 64, 1e-6, "aca", precision="fp64", symmetric=False)
    _compare_compression(h, F, blocks, tree, 1e-12)
    h.close()


def test_factor_and_solve_fp64(H, ctx, front576):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks = O.build(F.A, tree, "aca", 1e-6)
    Fac = O.factor(F.A, tree, blocks)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp64")
    H.hodlr_factor(h)
    st = h.stats()
    for l in range(1, tree.L + 1):
        D = h.export_d(l)
        for i in range(1 << l):
            r0, r1 = tree.range(l, i)
            ref = Fac.d[(l, i)]
            got = D[r0:r1, :ref.shape[1]]
            assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (l, i)
    for l in range(tree.L):
        S = h.export_core(l)
        rp = st["rank_pad"][l]
        for i in range(1 << l):
            blk = blocks[(l, i)]
            ra, rb = blk.Ua.shape[1], blk.Ub.shape[1]
            idx = np.concatenate([np.arange(rb), rp + np.arange(ra)])
            ref = np.linalg.inv(Fac.S[(l, i)])
            got = S[i][np.ix_(idx, idx)]
            assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (l, i)
    b = fg.rhs(F.n, 3, seed=1)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b)
    got = X.cpu().numpy().T
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    h.close()


def test_deferred_factor_matches_pipelined(H, ctx, front576):
    """A build with defer_factor leaves the matrix compressed only (solve is
    refused); hodlr_factor then gives the solve of the build that factored each
    level as soon as it was compressed, and a second hodlr_factor is a no-op."""
    F = front576
    A = _dev(F.A)
    b = fg.rhs(F.n, 2, seed=4)
    hp = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision="fp32")
    assert hp.stats()["factored"] == 1
    Xp = _dev(b.T)
    H.hodlr_solve(hp, Xp)
    ref = Xp.cpu().numpy()
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision="fp32", defer_factor=True)
    assert h.stats()["factored"] == 0
    with pytest.raises(H.HodlrError):
        H.hodlr_solve(h, _dev(b.T))
    with pytest.raises(H.HodlrError):
        h.export_d(1)
    c0 = H.hodlr_launch_count()
    H.hodlr_factor(h)
    c1 = H.hodlr_launch_count()
    H.hodlr_factor(h)
    assert c1 > c0 and H.hodlr_launch_count() == c1   # the second call launches nothing
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    # split-K products and node sums add with atomics: equal up to FP32 rounding
    assert np.linalg.norm(X.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    assert info.converged and np.all(info.iters <= 6)
    h.close()
    hp.close()


def test_launch_count_covers_replayed_iterations(H, ctx, front576):
    """hodlr_launch_count includes the kernels a recorded Arnoldi iteration runs
    on every device-side replay, not only the host-side launches."""
    F = front576
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision="fp32")
    H.hodlr_factor(h)
    b = fg.rhs(F.n, 1, seed=5)
    c0 = H.hodlr_launch_count()
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    c1 = H.hodlr_launch_count()
    it = int(info.iters.max())
    assert info.converged and it >= 2
    # per replayed iteration: the apply (which also splits z for the product),
    # the product, the fused Arnoldi step; per cycle at least the start, the
    # back substitution, the true-residual product and the residual
    assert c1 - c0 >= 3 * it + 4
    h.close()


def test_solve_fp32(H, ctx, front576):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks = O.build(F.A, tree, "aca", 1e-6, dtype=np.float32)
    Fac = O.factor(F.A, tree, blocks)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp32")
    H.hodlr_factor(h)
    b = fg.rhs(F.n, 2, seed=1)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b)
    got = X.cpu().numpy().T
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-4
    h.close()


@pytest.mark.parametrize("prec,rtol", [("bf16", 4e-2), ("fp16", 5e-3)])
def test_solve_16bit_storage(H, ctx, front576, prec, rtol):
    """FP32 factorisation, V and d stored in BF16 (unit roundoff 2^-8) or FP16 with
    a power-of-two scale per node column (2^-11) for the apply: the apply agrees
    with the oracle's FP64 solve to a few units of that roundoff times the growth
    through ~5 levels, and GMRES still reaches the FP64 target."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks = O.build(F.A, tree, "aca", 1e-6, dtype=np.float32)
    Fac = O.factor(F.A, tree, blocks)
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision=prec)
    H.hodlr_factor(h)
    b = fg.rhs(F.n, 2, seed=1)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b)
    err = np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref)
    assert err < rtol, err
    Xg, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    assert info.converged and np.all(info.true_relres <= 1e-12)
    h.close()


def test_matvec_is_fp64_accurate(H, ctx, front576):
    F = front576
    rng = np.random.default_rng(3)
    z = rng.standard_normal((5, F.n))
    W = H.hodlr_matvec(ctx, _dev(F.A), _dev(z)).cpu().numpy()
    ref = (F.A @ z.T).T
    # per term: a and z represented to 2^-48, cross terms and the float-pair
    # compensation rounded at 2^-48 each; 32 terms per pair, then FP64
    err = np.abs(W - ref).max(axis=1) / (np.abs(F.A) @ np.abs(z.T)).T.max(axis=1)
    assert err.max() < 16 * 2.0 ** -48
    # an FP64 dot product of this length is accurate to about sqrt(n) 2^-53 ~ 3e-15
    assert np.median(np.abs(W - ref) / (np.abs(F.A) @ np.abs(z.T)).T) < 2.0 ** -48


def _row_exponents(M):
    """Least e with max |M(i, :)| < 2^e per row (np.frexp's exponent)."""
    return np.frexp(np.abs(M).max(axis=1))[1].astype(np.float64)


@pytest.mark.parametrize("n,s", [(576, 32), (300, 20), (576, 45)])
def test_tensor_core_product_fp64_accurate(H, ctx, front576, n, s):
    """hodlr_matvec with 16 or more right-hand sides takes the digit-slice
    product on the tensor cores: seven base-256 digits per entry relative to a
    power of two per row of A and per column of Z (the last one rounded), slice
    pairs up to level 6 kept.  Per entry of A Z the digit and dropped-pair
    errors are at most n (2^-57 + 2^-57 + 6 * 256^2 2^-72) 2^(e_i + f_j)
    < 8 n 2^(e_i + f_j - 56); the float-pair and FP32 sums add at most about
    n 2^-51 of (|A||Z|)(i, j), the FP64 reference n 2^-53.  Statistically the
    error is far below the double-float product's 2^-48 per term.  Ragged sizes (n = 300: 384 padded rows, 320
    padded k; s = 20, 45: padded columns), a zero column and a column spanning
    30 orders of magnitude are included."""
    rng = np.random.default_rng(11)
    if n == 576:
        A = front576.A
    else:
        A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-8, 8, (n, n)))
    Z = rng.standard_normal((s, n))
    Z[1] = 0.0
    Z[2] *= np.exp(rng.uniform(-35, 35, n))
    W = H.hodlr_matvec(ctx, _dev(A), _dev(Z)).cpu().numpy()
    ref = (A @ Z.T).T
    scale = np.ldexp(1.0, (_row_exponents(Z)[:, None] + _row_exponents(A)[None, :]).astype(int))
    scale[1] = 0.0
    absz = (np.abs(A) @ np.abs(Z.T)).T
    err = np.abs(W - ref)
    assert np.all(err <= 8 * n * 2.0 ** -56 * scale + n * 2.0 ** -50 * absz)
    assert np.all(W[1] == 0.0)
    nz = absz > 0
    assert np.median(err[nz] / absz[nz]) < 2.0 ** -48


def test_tensor_core_product_digit_edges(H, ctx):
    """Rows whose largest entry lies just below a power of two (the top digit
    at its largest), rows of +-(2 - 2^-52), a row of one value, rows with
    subnormal and zero entries, a row of tiny entries at the padded edge and a
    row at 2^41: each entry of A Z within the digit-rounding bound of the
    other test, and a zero row of A gives exact zeros."""
    rng = np.random.default_rng(5)
    n, s = 300, 17
    A = rng.standard_normal((n, n))
    A[0, :] = (2.0 - 2.0 ** -52) * np.sign(rng.standard_normal(n))
    A[1, :] = rng.uniform(-1.0, 1.0, n)
    A[1, 7] = 1.9990234375
    A[1, 8] = -1.9990234375
    A[2, :] = 1.9921875 * rng.uniform(-1.0, 1.0, n)
    A[2, 3] = -1.9921875
    A[3, :] = 0.75
    A[4, :] = 5e-324 * rng.integers(-3, 4, n)    # subnormal: below the digits' reach
    A[4, 0] = 1.0
    A[5, :] = 0.0
    A[6, :] = np.ldexp(rng.uniform(1.99, 2.0, n), 40) * np.sign(rng.standard_normal(n))
    A[n - 1, :] = rng.standard_normal(n) * 1e-300
    Z = rng.standard_normal((s, n))
    W = H.hodlr_matvec(ctx, _dev(A), _dev(Z)).cpu().numpy()
    ref = (A @ Z.T).T
    scale = np.ldexp(1.0, (_row_exponents(Z)[:, None] + _row_exponents(A)[None, :]).astype(int))
    absz = (np.abs(A) @ np.abs(Z.T)).T
    err = np.abs(W - ref)
    assert np.all(err <= 8 * n * 2.0 ** -56 * scale + n * 2.0 ** -50 * absz)
    assert np.all(W[:, 5] == 0.0)
    # the constant row: 0.75 sum_k Z(j, k) to FP64 accuracy
    np.testing.assert_allclose(W[:, 3], 0.75 * Z.sum(axis=1), rtol=0, atol=1e-13 * np.abs(Z).sum(axis=1).max())


def test_gmres_many_rhs_tensor_core_product(H, ctx, front576):
    """GMRES with 20 right-hand sides (products on the tensor cores) gives the
    same solutions as two solves of 10 (double-float products), each to a true
    relative residual below 1e-12."""
    F = front576
    A = _dev(F.A)
    b = fg.rhs(F.n, 20, seed=12)
    h = H.hodlr_build(ctx, A, 64, 1e-4, "aca", precision="fp32")
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    assert info.converged and np.all(info.true_relres <= 1e-12)
    x = X.cpu().numpy()
    true = np.linalg.norm(b - F.A @ x.T, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(true <= 1.5e-12)
    for r0 in (0, 10):
        X2, i2 = H.gmres_solve(ctx, A, _dev(b[:, r0:r0 + 10].T), h, tol=1e-12)
        assert i2.converged
        assert np.abs(info.iters[r0:r0 + 10] - i2.iters).max() <= 1
        x2 = X2.cpu().numpy()
        assert np.linalg.norm(x[r0:r0 + 10] - x2) / np.linalg.norm(x2) < 1e-10
    ref = np.linalg.solve(F.A, b)
    assert np.linalg.norm(x.T - ref) / np.linalg.norm(ref) < 1e-9
    h.close()


@pytest.mark.parametrize("prec,itol", [("fp64", 1), ("fp32", 2)])
def test_gmres_matches_oracle(H, ctx, front576, prec, itol):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    dtype = np.float64 if prec == "fp64" else np.float32
    _, _, P = O.hodlr_precond(F.A, tree, "aca", 1e-6, dtype=dtype)
    b = fg.rhs(F.n, 2, seed=1)
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision=prec)
    H.hodlr_factor(h)
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    x = X.cpu().numpy()
    for r in range(2):
        ref = O.gmres(F.A, b[:, r], prec=P, tol=1e-12)
        assert info.true_relres[r] <= 1e-12
        true = np.linalg.norm(b[:, r] - F.A @ x[r]) / np.linalg.norm(b[:, r])
        assert true <= 1.5e-12
        assert abs(int(info.iters[r]) - ref.iters) <= itol
        assert np.linalg.norm(x[r] - ref.x) / np.linalg.norm(ref.x) < 1e-9
    h.close()


def test_gmres_multi_rhs_on_dirty_memory(H, ctx, front576):
    """Library buffers come from torch's caching allocator: fill its cache with
    garbage first, so that any read of a not-yet-written buffer shows."""
    F = front576
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision="fp32")
    H.hodlr_factor(h)
    b = fg.rhs(F.n, 6, seed=3)
    B = _dev(b.T)
    iters = None
    for trial in range(6):
        junk = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
        junk.fill_(0x7F if trial % 2 else 0xFF)
        del junk
        X, info = H.gmres_solve(ctx, A, B, h, tol=1e-12, max_iter=100)
        assert info.converged and np.all(info.true_relres <= 1e-12), (trial, info.iters)
        if iters is None:
            iters = info.iters.copy()
        assert np.abs(info.iters - iters).max() <= 1
    h.close()


def test_gmres_restarts_six_rhs(H, ctx, front576):
    """Restarted GMRES (several cycles: the per-cycle report, the stored split
    of A kept across cycles) with six right-hand sides (two launches per
    product): same solution as the unrestarted solve."""
    F = front576
    A = _dev(F.A)
    b = fg.rhs(F.n, 6, seed=8)
    h = H.hodlr_build(ctx, A, 64, 1e-3, "aca", precision="fp32")
    X1, i1 = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    X2, i2 = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12, restart=2)
    assert i1.converged and i2.converged
    assert i2.restarts >= 1 and np.all(i2.true_relres <= 1e-12)
    ref = np.linalg.solve(F.A, b)
    for X in (X1, X2):
        assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-9
    h.close()


def test_batched_shared_preconditioner_restarts(H, ctx, front576):
    """Batched GMRES with one preconditioner shared by three fronts of 1, 2 and
    3 right-hand sides (a window ends where the preconditioner repeats) and
    restarted cycles: every solution is exact and converged."""
    F = front576
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-3, "aca", precision="fp32")
    bs = [fg.rhs(F.n, k + 1, seed=20 + k) for k in range(3)]
    res = H.gmres_solve_batched(ctx, [A] * 3, [_dev(b.T) for b in bs], [h] * 3, tol=1e-12, restart=2)
    for b, (X, info) in zip(bs, res):
        assert info.converged and info.restarts >= 1 and np.all(info.true_relres <= 1e-12)
        ref = np.linalg.solve(F.A, b)
        assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-9
    h.close()


def test_streams_and_block_reuse(H, ctx, front576):
    """Build, solve and destroy on alternating streams: released blocks are
    reused across streams (ordered by their events); every solve is exact."""
    F = front576
    A = _dev(F.A)
    b = fg.rhs(F.n, 2, seed=9)
    ref = np.linalg.solve(F.A, b)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for st in (s1, s2, s1, s2):
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision="fp32")
            X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
            h.close()
        st.synchronize()
        assert info.converged
        assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-9


def test_gmres_unpreconditioned_and_nonconvergence(H, ctx, front576):
    F = front576
    b = fg.rhs(F.n, 1, seed=1)
    A = _dev(F.A)
    ref = O.gmres(F.A, b[:, 0], tol=1e-8, max_iter=400)
    X, info = H.gmres_solve(ctx, A, _dev(b.T), None, tol=1e-8, max_iter=400)
    assert info.converged and abs(int(info.iters[0]) - ref.iters) <= 2
    X, info = H.gmres_solve(ctx, A, _dev(b.T), None, tol=1e-14, max_iter=3)
    assert not info.converged and info.iters[0] == 3
    with pytest.raises(H.NotConverged):
        H.gmres_solve(ctx, A, _dev(b.T), None, tol=1e-14, max_iter=3, raise_on_fail=True)


def test_ragged_tree_and_zero_rhs(H, ctx):
    # n = 1000 with leaf 60: 16 leaves of 62/63 rows, odd node sizes at every level
    F = fg.make_front(25, 40, 5, 5, "lognormal", 0.5, leaf=60, seed=4)
    A = F.A
    n = F.n
    tree = O.make_tree(n, 60)
    blocks, Fac, P = O.hodlr_precond(A, tree, "aca", 1e-5)
    h = H.hodlr_build(ctx, _dev(A), 60, 1e-5, "aca", precision="fp64")
    H.hodlr_factor(h)
    st = h.stats()
    assert st["levels"] == tree.L and st["leaf_max"] == int(np.diff(tree.bounds).max())
    b = fg.rhs(n, 3, seed=1)
    b[:, 1] = 0.0
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b)
    assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-10
    Xg, info = H.gmres_solve(ctx, _dev(A), _dev(b.T), h, tol=1e-12)
    assert info.converged and info.iters[1] == 0 and np.all(Xg.cpu().numpy()[1] == 0)
    h.close()


def test_custom_leaf_bounds_and_single_leaf(H, ctx, front576):
    F = front576
    A = _dev(F.A)
    bounds = [0, 100, 288, 400, 576]
    tree = O.make_tree(F.n, 0, bounds)
    blocks, Fac, P = O.hodlr_precond(F.A, tree, "aca", 1e-6)
    h = H.hodlr_build(ctx, A, 0, 1e-6, "aca", precision="fp64", leaf_bounds=bounds)
    H.hodlr_factor(h)
    b = fg.rhs(F.n, 1, seed=2)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    assert np.linalg.norm(X.cpu().numpy().T - O.solve(Fac, b)) / np.linalg.norm(b) < 1e-10
    h.close()
    # leaf >= n: one dense leaf, the solve is a dense inverse
    h = H.hodlr_build(ctx, A, 1000, 1e-6, "aca", precision="fp64")
    H.hodlr_factor(h)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = np.linalg.solve(F.A, b)
    assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-12
    h.close()


def test_rank_zero_blocks(H, ctx):
    # block-diagonal matrix: every off-diagonal block is zero, every rank 0
    rng = np.random.default_rng(5)
    n = 256
    A = np.zeros((n, n))
    for s in range(0, n, 32):
        M = rng.standard_normal((32, 32))
        A[s:s + 32, s:s + 32] = M @ M.T + 32 * np.eye(32)
    h = H.hodlr_build(ctx, _dev(A), 32, 1e-6, "aca", precision="fp64")
    H.hodlr_factor(h)
    assert all(r == 0 for r in h.stats()["rank_max"])
    b = rng.standard_normal((1, n))
    X = _dev(b)
    H.hodlr_solve(h, X)
    assert np.linalg.norm(X.cpu().numpy()[0] - np.linalg.solve(A, b[0])) / np.linalg.norm(b) < 1e-12
    h.close()


@pytest.mark.parametrize("prec,tol,rtol", [("fp64", 1e-8, 1e-10), ("fp32", 1e-5, 2e-4)])
def test_large_leaves_cluster_inverse(H, ctx, prec, tol, rtol):
    """Leaves of 193 to 256 rows (ragged: 230, 250, 220, 256) are inverted by a
    cluster of CTAs sharing the columns; d = K_leaf^-1 U of the deepest level
    and the solve agree with the oracle's LU-based recursion."""
    rng = np.random.default_rng(8)
    n = 956
    bounds = np.array([0, 230, 480, 700, 956])
    # a Gaussian kernel (numerically low-rank off the diagonal) plus a random
    # SPD block on every leaf
    x = np.linspace(0, 1, n)
    A = np.exp(-((x[:, None] - x[None, :]) / 0.3) ** 2) + 0.5 * np.eye(n)
    for i in range(4):
        r0, r1 = bounds[i], bounds[i + 1]
        M = rng.standard_normal((r1 - r0, r1 - r0))
        A[r0:r1, r0:r1] += M @ M.T / (r1 - r0)
    tree = O.make_tree(n, 256, bounds)
    dtype = np.float64 if prec == "fp64" else np.float32
    blocks = O.build(A, tree, "aca", tol, dtype=dtype)
    Fac = O.factor(A, tree, blocks)
    h = H.hodlr_build(ctx, _dev(A), 256, tol, "aca", precision=prec, leaf_bounds=bounds)
    D = h.export_d(2)
    for i in range(4):
        r0, r1 = tree.range(2, i)
        ref = Fac.d[(2, i)]
        got = D[r0:r1, :ref.shape[1]]
        assert np.abs(got - ref).max() <= rtol * np.abs(ref).max(), (i, np.abs(got - ref).max())
    b = rng.standard_normal((3, n))
    X = _dev(b)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b.T).T
    assert np.linalg.norm(X.cpu().numpy() - ref) / np.linalg.norm(ref) < rtol
    h.close()


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("leaf", [32, 64, 96, 128, 160, 192, 256])
@pytest.mark.parametrize("scale", [1e6, 1e-6])
def test_leaf_inverse_is_scale_invariant(H, ctx, prec, rtol, leaf, scale):
    """Every Gauss-Jordan size class (registers, blocked panels, clusters of
    CTAs) on a matrix scaled by 1e6 or 1e-6: a uniform scale leaves the
    condition unchanged, so d = K_leaf^-1 U of the deepest level must agree
    with the FP64 solve of the leaf to the arithmetic's unit roundoff times
    the leaf's condition (below 10 here), whatever the size of the pivots."""
    rng = np.random.default_rng(leaf)
    n = 4 * leaf
    x = np.linspace(0, 1, n)
    K = np.exp(-((x[:, None] - x[None, :]) / 0.3) ** 2) + 0.5 * np.eye(n)
    for i in range(4):
        M = rng.standard_normal((leaf, leaf))
        K[i * leaf:(i + 1) * leaf, i * leaf:(i + 1) * leaf] += M @ M.T / leaf
    A = scale * K
    tol = 1e-8 if prec == "fp64" else 1e-5
    h = H.hodlr_build(ctx, _dev(A), leaf, tol, "aca", precision=prec)
    st = h.stats()
    L = st["levels"]
    assert L == 2 and st["leaf_max"] == leaf
    U, _, _, _, _ = h.export_level(L)
    D = h.export_d(L)
    for i in range(4):
        r0, r1 = i * leaf, (i + 1) * leaf
        ref = np.linalg.solve(A[r0:r1, r0:r1], U[r0:r1])
        err = np.abs(D[r0:r1] - ref).max() / np.abs(ref).max()
        assert err <= rtol, (leaf, scale, i, err)
    h.close()


def test_nonfinite_input_is_reported(H, ctx, front576):
    A = front576.A.copy()
    A[0, 300] = np.nan                   # row 0 of the top block is always read
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_build(ctx, _dev(A), 64, 1e-6, "aca", precision="fp64", symmetric=False)
    assert e.value.code == 8


def test_invalid_arguments(H, ctx, front576):
    A = _dev(front576.A)
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_build(ctx, A, 64, 2.0, "aca")
    assert e.value.code == 1
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_build(ctx, A, 64, 1e-3, "bdlr")          # BDLR without a graph
    assert e.value.code == 1
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_build(ctx, A, 64, 1e-3, "aca", rank_cap=5000)
    assert e.value.code == 9


def test_singular_leaf_is_reported(H, ctx):
    n = 128
    A = np.eye(n)
    A[:32, :32] = 0.0                     # first leaf singular
    # the leaf inverses are computed while the matrix is built: the zero pivot is
    # reported by hodlr_build (or, at the latest, by the next synchronising call)
    with pytest.raises(H.HodlrError) as e:
        h = H.hodlr_build(ctx, _dev(A), 32, 1e-6, "aca", precision="fp64")
        H.hodlr_factor(h)
        H.gmres_solve(ctx, _dev(A), _dev(np.ones((1, n))), h, tol=1e-12, max_iter=5)
    assert e.value.code == 4


# ---------------------------------------------------------------- the 4096 front
def test_cores_fp32_vs_fp64_front4096(H, ctx, front4096):
    """The FP32 factorisation (blocked Gauss-Jordan for the cores wider than
    64) against the FP64 one on the same FP32 compression: every inverted core
    agrees to FP32 accuracy."""
    F = front4096
    A = _dev(F.A)
    g = (F.rowptr, F.colind)
    h32 = H.hodlr_build(ctx, A, 128, 1e-4, "aca", graph=g, precision="fp32", compress_precision="fp32")
    h64 = H.hodlr_build(ctx, A, 128, 1e-4, "aca", graph=g, precision="fp64", compress_precision="fp32")
    s32, s64 = h32.stats(), h64.stats()
    assert s32["rank_max"] == s64["rank_max"]
    assert max(s32["rank_pad"]) > 128   # cores of several widths above 64
    for l in range(s32["levels"]):
        S32, S64 = h32.export_core(l), h64.export_core(l)
        for i in range(len(S64)):
            err = np.abs(S32[i] - S64[i]).max() / np.abs(S64[i]).max()
            assert err < 1e-4, (l, i, err)
    h32.close()
    h64.close()


@pytest.mark.parametrize("method,tol,prec", [("aca", 1e-4, "fp32"), ("aca", 1e-4, "fp64"),
                                             ("bdlr", 1e-4, "fp32"), ("aca", 1e-8, "fp32"),
                                             ("bdlr", 1e-8, "fp64")])
def test_front4096_gmres(H, ctx, front4096, method, tol, prec):
    F = front4096
    g = (F.rowptr, F.colind)
    tree = O.make_tree(F.n, 128, F.bounds)
    dtype = np.float64 if prec == "fp64" else np.float32
    blocks, Fac, P = O.hodlr_precond(F.A, tree, method, tol, graph=g, dtype=dtype)
    b = fg.rhs(F.n, 4, seed=1)
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 128, tol, method, graph=g, precision=prec)
    st = h.stats()
    for l in range(1, tree.L + 1):
        ro = max(max(blocks[(l - 1, i // 2)].Ua.shape[1] if i % 2 == 0 else blocks[(l - 1, i // 2)].Ub.shape[1]
                      for i in range(1 << l)), 0)
        assert st["rank_max"][l - 1] == ro
    H.hodlr_factor(h)
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    x = X.cpu().numpy()
    assert info.converged and np.all(info.true_relres <= 1e-12)
    for r in range(4):
        ref = O.gmres(F.A, b[:, r], prec=P, tol=1e-12)
        assert abs(int(info.iters[r]) - ref.iters) <= 2, (r, info.iters, ref.iters)
        assert np.linalg.norm(x[r] - ref.x) / np.linalg.norm(ref.x) < 1e-9
    h.close()


def test_reduced_plane32768_fp16_32_rhs(H, ctx):
    """The n = 32768 workload's construction scaled down: a 32 x 64 x 9 grid (4
    planes per side, lognormal sigma 0.5, n = 2048), leaf 256 (3 levels), ACA
    tol 1e-3, FP16 storage with per-(node, column) power-of-two scales, 32
    right-hand sides (the tensor-core product).  The apply agrees element by
    element with the oracle's solve on the FP32-compressed blocks to the FP16
    storage's rounding (2^-11 per entry, grown through 3 levels: 5e-3 relative
    per column); GMRES reaches 1e-12 on all 32; sampled columns agree with the
    oracle's GMRES iterates to 1e-9 and its iteration counts within 3."""
    F = fg.make_front(32, 64, 4, 4, "lognormal", 0.5, leaf=256, seed=0)
    n = F.n
    assert n == 2048 and F.levels == 3
    tree = O.make_tree(n, 256, F.bounds)
    blocks, Fac, P = O.hodlr_precond(F.A, tree, "aca", 1e-3, symmetric=True, dtype=np.float32)
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 256, 1e-3, "aca", precision="fp16", leaf_bounds=F.bounds)
    st = h.stats()
    for l in range(1, tree.L + 1):
        ro = max(blocks[(l - 1, i // 2)].Ua.shape[1] if i % 2 == 0 else blocks[(l - 1, i // 2)].Ub.shape[1]
                 for i in range(1 << l))
        assert st["rank_max"][l - 1] == ro
    b = fg.rhs(n, 32, seed=1)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    ref = O.solve(Fac, b)
    got = X.cpu().numpy().T
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() < 5e-3, err.max()
    Xg, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    assert info.converged and np.all(info.true_relres <= 1e-12)
    x = Xg.cpu().numpy()
    for r in (0, 13, 31):
        o = O.gmres(F.A, b[:, r], prec=P, tol=1e-12)
        assert abs(int(info.iters[r]) - o.iters) <= 3, (r, info.iters[r], o.iters)
        assert np.linalg.norm(x[r] - o.x) / np.linalg.norm(o.x) < 1e-9
    h.close()


@pytest.mark.parametrize("method,prec", [("aca", "fp64"), ("aca", "fp32"), ("bdlr", "fp64")])
def test_elastic_front_gmres(H, ctx, method, prec):
    """The 3-dof elasticity front (Navier-Cauchy, lognormal shear modulus,
    Poisson ratio 0.3) of a 24 x 24 x 9 box, n = 1728, leaves of 36 nodes:
    ranks per level equal the oracle's, GMRES reaches 1e-12, iterates agree with
    the oracle's to 1e-9 and iteration counts within 2."""
    E = fg.make_elastic_front(24, 24, 4, 4, leaf_nodes=64)
    tree = O.make_tree(E.n, 108, E.bounds)
    g = (E.rowptr, E.colind)
    tol = 1e-6 if method == "aca" else 1e-4
    dtype = np.float64 if prec == "fp64" else np.float32
    blocks, Fac, P = O.hodlr_precond(E.A, tree, method, tol, graph=g, symmetric=True, dtype=dtype)
    A = _dev(E.A)
    h = H.hodlr_build(ctx, A, 108, tol, method, graph=g, precision=prec, leaf_bounds=E.bounds)
    st = h.stats()
    for l in range(1, tree.L + 1):
        ro = max(blocks[(l - 1, i // 2)].Ua.shape[1] if i % 2 == 0 else blocks[(l - 1, i // 2)].Ub.shape[1]
                 for i in range(1 << l))
        assert st["rank_max"][l - 1] == ro
    b = fg.rhs(E.n, 2, seed=1)
    X, info = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    assert info.converged and np.all(info.true_relres <= 1e-12)
    x = X.cpu().numpy()
    for r in range(2):
        ref = O.gmres(E.A, b[:, r], prec=P, tol=1e-12)
        assert abs(int(info.iters[r]) - ref.iters) <= 2, (info.iters[r], ref.iters)
        assert np.linalg.norm(x[r] - ref.x) / np.linalg.norm(ref.x) < 1e-9
    h.close()


@pytest.fixture(scope="module")
def front16384():
    return fg.make_front(**fg.WORKLOADS["checker16384"], device="cuda", cache=True)


def test_front16384_bf16_high_contrast(H, ctx, front16384):
    """The high-contrast n = 16384 front (checkerboard 1/1e6), BF16 storage of the
    factors, ACA tol 1e-3, leaf 256, one right-hand side.  Checked at full size:
    the ACA pivots and rank of the top-level block A(0:8192, 8192:16384) against
    the oracle (FP32 decisions); FP64 GMRES reaches max(1e-12, 10 rho_LU), rho_LU
    the dense FP64 LU solve's own residual (the contrast of 1e6 puts that floor
    above 1e-12); and the BF16 preconditioner is
    compared with the FP64 HODLR one, ||(P_bf16^-1 - P_fp64^-1) A Omega|| / ||Omega||."""
    F = front16384
    n = F.n
    A = F.A if torch.is_tensor(F.A) else _dev(F.A)
    h = H.hodlr_build(ctx, A, 256, 1e-3, "aca", precision="bf16", leaf_bounds=F.bounds)
    # top-level block against the oracle, in FP32 decisions
    Ah = A.cpu().numpy()
    half = int(F.bounds[len(F.bounds) // 2])
    blk = Ah[:half, half:]
    ref = O.aca(lambda i: blk[i, :], lambda j: blk[:, j], blk.shape[0], blk.shape[1], 1e-3, 1 << 30, np.float32)
    U, V, ranks, pr, pc = h.export_level(1)
    k = ref.U.shape[1]
    assert ranks[0] == k
    assert list(pr[0][:k]) == list(ref.rows) and list(pc[0][:k]) == list(ref.cols)
    H.hodlr_factor(h)
    b = fg.rhs(n, 1, seed=1)
    Bd = _dev(b.T)
    # the attainable residual: FP64 dense LU's own, times 10 (and at most 1e-12)
    xl = torch.linalg.solve(A, Bd.T)
    rho = float(torch.linalg.norm(Bd.T - A @ xl) / torch.linalg.norm(Bd))
    target = max(1e-12, 10 * rho)
    del xl
    X, info = H.gmres_solve(ctx, A, Bd, h, tol=target)
    assert info.converged and info.true_relres[0] <= target, (info.iters, info.true_relres, rho)
    # preconditioner error of the BF16 factors against the FP64 HODLR
    h64 = H.hodlr_build(ctx, A, 256, 1e-3, "aca", precision="fp64", leaf_bounds=F.bounds)
    H.hodlr_factor(h64)
    g = torch.Generator(device="cpu").manual_seed(2)
    Om = torch.randn(16, n, generator=g, dtype=torch.float64).cuda()
    AOm = (A @ Om.T).T.contiguous()
    Y1 = AOm.clone()
    Y2 = AOm.clone()
    H.hodlr_solve(h, Y1)
    H.hodlr_solve(h64, Y2)
    perr = float(torch.linalg.norm(Y1 - Y2) / torch.linalg.norm(Om))
    print(f"checker16384 bf16: target {target:.2e} iters {info.iters.tolist()} true {info.true_relres.tolist()} rho_LU {rho:.2e} "
          f"rank1 {k} precond-diff {perr:.3e}")
    assert np.isfinite(perr) and perr < 1.0
    h64.close()
    # the Woodbury-core condition guard on this front: with a threshold below
    # the root core's kappa_1 that core (and any above it) is re-inverted in FP64
    # from the stored factors; its exported inverse is the FP64 inverse of the
    # core formed from them, and the solve still reaches the target
    st = h.stats()
    thr = 0.5 * st["core_cond_max"][0]
    hg = H.hodlr_build(ctx, A, 256, 1e-3, "aca", precision="bf16", leaf_bounds=F.bounds, core_cond_threshold=thr)
    stg = hg.stats()
    assert stg["cores_promoted"][0] == 1 and sum(stg["cores_promoted"]) >= 1
    _, Vx, _, _, _ = hg.export_level(1)
    Dx = hg.export_d(1)
    rp = stg["rank_pad"][0]
    S = np.eye(2 * rp)
    S[:rp, rp:] = Vx[:half].T @ Dx[:half]
    S[rp:, :rp] = Vx[half:].T @ Dx[half:]
    ref = np.linalg.inv(S)
    got = hg.export_core(0)[0]
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    cond, flag = hg.export_core_cond(0)
    kap = np.linalg.norm(S, 1) * np.linalg.norm(ref, 1)
    assert flag[0] and abs(cond[0] - kap) <= 1e-3 * kap
    X2, info2 = H.gmres_solve(ctx, A, Bd, hg, tol=target)
    assert info2.converged and info2.true_relres[0] <= target
    print(f"checker16384 guard: kappa_max per level {st['core_cond_max']} promoted at thr {thr:.3g}: "
          f"{stg['cores_promoted']} iters {info2.iters.tolist()}")
    hg.close()
    h.close()


def test_batched_octree_fronts(H, ctx):
    """A batch of octree fronts of uneven sizes (1024, 256 and 64: leaf 128, 64, 64
    -> 3, 2 and 0 levels) through the batched calls: every front converges to
    1e-12, the fronts agree with the oracle (iterations within 2, iterates within
    1e-9) and with the single-front calls."""
    boxes = fg.octree_boxes(64, 8)
    pick = boxes[1:3] + boxes[9:12] + boxes[73:77]
    fronts, leaves = [], []
    for s_, org in pick:
        leaf = 128 if s_ * s_ >= 1024 else 64
        F = fg.make_octree_front(s_, org, leaf, sigma=1.0, seed=0, device="cuda")
        fronts.append(F)
        leaves.append(leaf)
    As = [F.A if torch.is_tensor(F.A) else _dev(F.A) for F in fronts]
    Bs = [_dev(fg.rhs(F.n, 1, seed=1 + f).T) for f, F in enumerate(fronts)]
    hs = H.hodlr_build_batched(ctx, As, leaves, 1e-6, "aca", precision="fp32")
    H.hodlr_factor_batched(hs)
    res = H.gmres_solve_batched(ctx, As, Bs, hs, tol=1e-12)
    for f, (X, info) in enumerate(res):
        assert info.converged and np.all(info.true_relres <= 1e-12), (f, info.iters, info.true_relres)
    # the single-front calls give the same solutions
    for f in (0, 3, 6):
        h1 = H.hodlr_build(ctx, As[f], leaves[f], 1e-6, "aca", precision="fp32", leaf_bounds=fronts[f].bounds)
        H.hodlr_factor(h1)
        X1, info1 = H.gmres_solve(ctx, As[f], Bs[f], h1, tol=1e-12)
        x, x1 = res[f][0].cpu().numpy(), X1.cpu().numpy()
        assert np.linalg.norm(x - x1) / np.linalg.norm(x1) < 1e-10
        h1.close()
    # against the oracle
    for f in (0, 4, 8):
        F = fronts[f]
        An = As[f].cpu().numpy()
        tree = O.make_tree(F.n, leaves[f], F.bounds)
        _, _, P = O.hodlr_precond(An, tree, "aca", 1e-6, dtype=np.float32)
        b = Bs[f].cpu().numpy().reshape(-1)
        ref = O.gmres(An, b, prec=P, tol=1e-12)
        X, info = res[f]
        assert abs(int(info.iters[0]) - ref.iters) <= 2, (f, info.iters, ref.iters)
        x = X.cpu().numpy().reshape(-1)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-9
    for h in hs:
        h.close()


@pytest.mark.parametrize("precision,nrhs", [("fp32", 4), ("fp16", 32), ("fp64", 3)])
def test_apply_paths_agree(H, ctx, front4096, precision, nrhs):
    """The apply launched once for all levels (per-node waits) and launched
    once per phase (one CTA per row tile) compute the same K~^-1 X up to the
    rounding order of the node sums, and GMRES on the per-phase path converges
    to 1e-12 in the iterations of the single launch (+-1)."""
    F = front4096
    A = _dev(F.A)
    B = fg.rhs(F.n, nrhs, seed=21)
    h = H.hodlr_build(ctx, A, 128, 1e-4, "aca", precision=precision)
    out = {}
    try:
        for path in (1, 2):
            ctx.set_apply_path(path)
            X = _dev(B.T)
            H.hodlr_solve(h, X)
            torch.cuda.synchronize()
            Xg, info = H.gmres_solve(ctx, A, _dev(B.T), h, tol=1e-12)
            out[path] = (X.cpu().numpy(), info)
    finally:
        ctx.set_apply_path(0)
    x1, i1 = out[1]
    x2, i2 = out[2]
    assert np.all(np.isfinite(x2))
    # FP32 (FP16-stored) arithmetic: node sums in another order differ by a few
    # units of 2^-24 of the terms; FP64: of 2^-53
    rtol = 1e-13 if precision == "fp64" else 2e-5
    assert np.linalg.norm(x2 - x1) <= rtol * np.linalg.norm(x1)
    assert i2.converged and np.all(i2.true_relres <= 1e-12)
    assert np.abs(i1.iters - i2.iters).max() <= 1
    h.close()


@pytest.mark.parametrize("precision,nrhs", [("fp32", 5), ("fp16", 40), ("bf16", 33)])
def test_per_phase_apply_ragged_tiles(H, ctx, front576, precision, nrhs):
    """FP32-arithmetic per-phase apply on leaves of 72 rows (row tiles of 32, 32
    and 8) and, past 32 right-hand sides, in two passes: the same K~^-1 X as
    the single launch up to the rounding order of the sums, and the same as the
    oracle's solve with the FP64 factors to the storage's rounding."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    Fac = O.factor(F.A, tree, O.build(F.A, tree, "aca", 1e-6))
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision=precision)
    b = fg.rhs(F.n, nrhs, seed=7)
    out = {}
    try:
        for path in (1, 2):
            ctx.set_apply_path(path)
            X = _dev(b.T)
            H.hodlr_solve(h, X)
            torch.cuda.synchronize()
            out[path] = X.cpu().numpy().T
    finally:
        ctx.set_apply_path(0)
    x1, x2 = out[1], out[2]
    assert np.all(np.isfinite(x2))
    assert np.linalg.norm(x2 - x1) <= 2e-5 * np.linalg.norm(x1)
    ref = O.solve(Fac, b)
    tol = {"fp32": 1e-4, "fp16": 1e-2, "bf16": 5e-2}[precision]
    assert np.linalg.norm(x2 - ref) <= tol * np.linalg.norm(ref)
    h.close()


def test_per_phase_apply_matches_oracle(H, ctx, front576):
    """The per-phase apply against the oracle's recursive solve (FP64 factors,
    ACA 1e-6), to the factor-and-solve tolerance."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks = O.build(F.A, tree, "aca", 1e-6)
    Fac = O.factor(F.A, tree, blocks)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp64")
    b = fg.rhs(F.n, 5, seed=2)
    X = _dev(b.T)
    try:
        ctx.set_apply_path(2)
        H.hodlr_solve(h, X)
        torch.cuda.synchronize()
    finally:
        ctx.set_apply_path(0)
    ref = O.solve(Fac, b)
    assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-10
    h.close()
