"""GPU tests of the Woodbury-core condition guard, the preconditioner-error
report against the oracle, the device status word and the bounded waits.

Tolerances:
* kappa_1(S) is computed by the library from the FP32 P, Q and S^-1 it formed;
  the reference forms S from the exported FP32 factors with FP64 products.
  The two differ by FP32 rounding amplified by kappa (below 1e3 here): 1e-3.
* A core re-inverted in FP64 is, by construction, the FP64 inverse of S formed
  from the stored FP32 d and V with FP64 products: its export agrees with
  numpy's inverse of that S to kappa * n * 2^-53 (below 1e-10 here).
* ||(I - P^-1 A) Omega||_F / ||Omega||_F: the FP64 library path against the
  oracle on the same Omega, 1e-6 relative (both are FP64 evaluations of the same
  HODLR inverse, whose own error is about tol).
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


def _cores_from_factors(h, l, tree):
    """The cores S of level l (parents of level l + 1) formed in FP64 from the
    exported d and V of level l + 1: S = [[I, V_ba^T d_a], [V_ab^T d_b, I]]
    (padded to 2 rank_pad, rows of node a in V hold V_ba)."""
    _, V, _, _, _ = h.export_level(l + 1)
    D = h.export_d(l + 1)
    rp = h.stats()["rank_pad"][l]
    out = []
    for i in range(1 << l):
        a0, a1 = tree.range(l + 1, 2 * i)
        b0, b1 = tree.range(l + 1, 2 * i + 1)
        S = np.eye(2 * rp)
        S[:rp, rp:] = V[a0:a1].T @ D[a0:a1]
        S[rp:, :rp] = V[b0:b1].T @ D[b0:b1]
        out.append(S)
    return out


def _kappa1(S):
    return np.linalg.norm(S, 1) * np.linalg.norm(np.linalg.inv(S), 1)


def test_core_condition_guard_front4096(H, ctx, front4096):
    """kappa_1 of every Woodbury core, and the FP64 re-inversion of the cores
    above the threshold (FP32 factor arithmetic, ACA tol 1e-4, leaf 128)."""
    F = front4096
    A = _dev(F.A)
    tree = O.make_tree(F.n, 128, F.bounds)
    # default threshold tol / 2^-24 = 1678: these cores (kappa ~ 1e2) stay FP32
    h = H.hodlr_build(ctx, A, 128, 1e-4, "aca", precision="fp32")
    st = h.stats()
    assert st["core_cond_threshold"] == pytest.approx(1e-4 / 2.0 ** -24)
    assert sum(st["cores_promoted"]) == 0
    kap = {}
    for l in range(tree.L):
        cond, flag = h.export_core_cond(l)
        assert not flag.any()
        ref = np.array([_kappa1(S) for S in _cores_from_factors(h, l, tree)])
        assert np.all(np.abs(cond - ref) <= 1e-3 * ref), (l, cond, ref)
        assert st["core_cond_max"][l] == pytest.approx(cond.max())
        kap[l] = ref
    # a threshold inside the observed range: exactly the cores above it are
    # re-inverted in FP64, and their exported inverse is the FP64 inverse of
    # the core formed from the stored factors
    allk = np.concatenate(list(kap.values()))
    thr = float(np.median(allk))
    h2 = H.hodlr_build(ctx, A, 128, 1e-4, "aca", precision="fp32", core_cond_threshold=thr)
    st2 = h2.stats()
    assert st2["core_cond_threshold"] == pytest.approx(thr)
    n_prom = 0
    for l in range(tree.L):
        cond, flag = h2.export_core_cond(l)
        np.testing.assert_array_equal(flag, cond > thr)
        n_prom += int(flag.sum())
        Sg = h2.export_core(l)
        for i, S in enumerate(_cores_from_factors(h2, l, tree)):
            ref = np.linalg.inv(S)
            err = np.abs(Sg[i] - ref).max() / np.abs(ref).max()
            if flag[i]:
                assert err <= 1e-10, (l, i, err)
            else:
                assert err <= 1e-4, (l, i, err)
    assert n_prom == sum(st2["cores_promoted"]) and n_prom > 0
    # the solves of both builds reach the FP64 target in the same iterations
    b = fg.rhs(F.n, 4, seed=1)
    X1, i1 = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    X2, i2 = H.gmres_solve(ctx, A, _dev(b.T), h2, tol=1e-12)
    assert i1.converged and i2.converged
    assert np.abs(i1.iters - i2.iters).max() <= 1
    x1, x2 = X1.cpu().numpy(), X2.cpu().numpy()
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-10
    # threshold 0 < kappa: every core; negative: the guard is off
    h3 = H.hodlr_build(ctx, A, 128, 1e-4, "aca", precision="fp32", core_cond_threshold=1e-300)
    assert sum(h3.stats()["cores_promoted"]) == sum(1 << l for l in range(tree.L))
    h4 = H.hodlr_build(ctx, A, 128, 1e-4, "aca", precision="fp32", core_cond_threshold=-1.0)
    assert h4.stats()["core_cond_threshold"] == -1.0
    with pytest.raises(H.HodlrError):
        h4.export_core_cond(0)
    for x in (h, h2, h3, h4):
        x.close()


def test_core_condition_fp64_arithmetic_never_promotes(H, ctx, front576):
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp64", core_cond_threshold=1e-300)
    st = h.stats()
    assert sum(st["cores_promoted"]) == 0 and st["core_cond_threshold"] == float("inf")
    blocks = O.build(F.A, tree, "aca", 1e-6)
    Fac = O.factor(F.A, tree, blocks)
    for l in range(tree.L):
        cond, _ = h.export_core_cond(l)
        for i in range(1 << l):
            ref = _kappa1(Fac.S[(l, i)])
            assert abs(cond[i] - ref) <= 1e-8 * ref, (l, i, cond[i], ref)
    h.close()


@pytest.mark.parametrize("prec,tol,rtol", [("fp64", 1e-6, 1e-6), ("fp64", 1e-3, 1e-6), ("fp32", 1e-4, 5e-2)])
def test_precond_error_matches_oracle_576(H, ctx, front576, prec, tol, rtol):
    """O10 (i): ||(I - P^-1 A) Omega||_F / ||Omega||_F with the same seeded
    Omega (n x 16 N(0,1), stream 2) in the library and the oracle.  The FP32
    case compares with the oracle's FP64 factorisation of the FP32-compressed
    blocks (the difference is the FP32 factorisation's own rounding)."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    dtype = np.float64 if prec == "fp64" else np.float32
    _, _, P = O.hodlr_precond(F.A, tree, "aca", tol, symmetric=True, dtype=dtype)
    Om = fg.rhs(F.n, 16, seed=2)
    ref = O.precond_error(F.A, P, Om)
    h = H.hodlr_build(ctx, _dev(F.A), 64, tol, "aca", precision=prec)
    got = H.hodlr_precond_error(h, _dev(Om.T))
    assert abs(got - ref) <= rtol * ref, (got, ref)
    h.close()


def test_precond_error_matches_oracle_4096(H, ctx, front4096):
    F = front4096
    tree = O.make_tree(F.n, 128, F.bounds)
    _, _, P = O.hodlr_precond(F.A, tree, "aca", 1e-4, symmetric=True)
    Om = fg.rhs(F.n, 16, seed=2)
    ref = O.precond_error(F.A, P, Om)
    h = H.hodlr_build(ctx, _dev(F.A), 128, 1e-4, "aca", precision="fp64")
    got = H.hodlr_precond_error(h, _dev(Om.T))
    assert abs(got - ref) <= 1e-6 * ref, (got, ref)
    h.close()


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-8), ("fp32", 5e-2)])
def test_precond_error_two_norm_576(H, ctx, front576, prec, rtol):
    """O10 (ii): the exact ||I - P^-1 A||_2 of the oracle (dense SVD) against the
    same norm of the library's own P^-1 applied to every column of A."""
    F = front576
    tree = O.make_tree(F.n, 64, F.bounds)
    dtype = np.float64 if prec == "fp64" else np.float32
    _, _, P = O.hodlr_precond(F.A, tree, "aca", 1e-4, symmetric=True, dtype=dtype)
    ref = O.precond_error_2norm(F.A, P)
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-4, "aca", precision=prec)
    X = _dev(F.A.T)          # the columns of A, one right-hand side each
    H.hodlr_solve(h, X)
    E = np.eye(F.n) - X.cpu().numpy().T
    got = float(np.linalg.svd(E, compute_uv=False)[0])
    assert abs(got - ref) <= rtol * ref, (got, ref)
    h.close()


def test_matvec_reports_nonfinite_and_clears_status(H, ctx, front576):
    """A NaN in A makes hodlr_matvec return NONFINITE_INPUT (both product
    paths), and the flag does not leak into the next call on the context."""
    F = front576
    A = F.A.copy()
    A[5, 17] = np.nan
    Ad = _dev(A)
    for s in (3, 20):                     # double-float product; tensor-core product
        Z = _dev(np.ones((s, F.n)))
        with pytest.raises(H.HodlrError) as e:
            H.hodlr_matvec(ctx, Ad, Z)
        assert e.value.code == 8
    h = H.hodlr_build(ctx, _dev(F.A), 64, 1e-6, "aca", precision="fp32")
    X, info = H.gmres_solve(ctx, _dev(F.A), _dev(fg.rhs(F.n, 1, seed=1).T), h, tol=1e-12)
    assert info.converged
    h.close()


def test_apply_wait_budget_runs_out(H, front576):
    """The apply's per-node waits are bounded: with an arrival target that can
    never be met (a test setting) every wait gives up after its budget, the
    kernel returns, and the next synchronising call reports TIMEOUT.  After the
    setting is reset the same context solves correctly again."""
    F = front576
    c = H.Context(0)
    A = _dev(F.A)
    h = H.hodlr_build(c, A, 64, 1e-6, "aca", precision="fp32")
    b = fg.rhs(F.n, 2, seed=3)
    X0 = _dev(b.T)
    H.hodlr_solve(h, X0)
    torch.cuda.synchronize()
    c.set_wait_test(spin_limit=1000, unreachable=True)
    X = _dev(b.T)
    H.hodlr_solve(h, X)                   # stream-ordered: no status read yet
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_matvec(c, A, _dev(np.ones((1, F.n))))
    assert e.value.code == 7
    c.set_wait_test(0, False)
    X = _dev(b.T)
    H.hodlr_solve(h, X)
    H.hodlr_matvec(c, A, _dev(np.ones((1, F.n))))   # status clean again
    assert torch.equal(X, X0) or float(torch.linalg.norm(X - X0) / torch.linalg.norm(X0)) < 1e-6
    h.close()
    c.close()


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-13), ("fp32", 1e-5), ("fp16", 1e-5)])
def test_save_load_round_trip(H, ctx, front576, prec, rtol):
    """A factored HODLR matrix written to host memory and restored (after the
    original is destroyed) holds the same factors bit for bit (saving the
    restored object gives the same image); its solves agree with the
    original's to the apply's own run-to-run rounding (its node sums are
    atomic), and GMRES with it takes the same iterations to the same solution."""
    F = front576
    A = _dev(F.A)
    h = H.hodlr_build(ctx, A, 64, 1e-6, "aca", precision=prec)
    b = fg.rhs(F.n, 3, seed=6)
    X0 = _dev(b.T)
    H.hodlr_solve(h, X0)
    Xg0, i0 = H.gmres_solve(ctx, A, _dev(b.T), h, tol=1e-12)
    st0 = h.stats()
    img = H.hodlr_save(h)
    h.close()
    h2 = H.hodlr_load(ctx, img, A)
    assert H.hodlr_save(h2) == img
    st2 = h2.stats()
    assert st2["rank_max"] == st0["rank_max"] and st2["factored"]
    X1 = _dev(b.T)
    H.hodlr_solve(h2, X1)
    assert float(torch.linalg.norm(X1 - X0) / torch.linalg.norm(X0)) <= rtol
    Xg1, i1 = H.gmres_solve(ctx, A, _dev(b.T), h2, tol=1e-12)
    assert np.abs(i0.iters - i1.iters).max() <= 1
    assert float(torch.linalg.norm(Xg1 - Xg0) / torch.linalg.norm(Xg0)) <= 1e-10
    assert H.hodlr_precond_error(h2, _dev(fg.rhs(F.n, 4, seed=2).T)) > 0
    h2.close()
    # an image that is not one is refused
    with pytest.raises(H.HodlrError) as e:
        H.hodlr_load(ctx, b"not an image" * 4)
    assert e.value.code == 1
