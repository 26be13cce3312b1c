"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
hand-derived worked examples, closed forms, identities, brute force on tiny inputs.
CPU only."""
import math
import os

import numpy as np
import pytest

import frontgen as fg
from oracle import hodlr_oracle as O


# --------------------------------------------------------------------------- inputs
def _dense_3d_operator(a):
    """Assemble the 7-point operator of the whole box as a dense matrix, straight
    from its stencil definition (x-fastest natural order)."""
    nz, ny, nx = a.shape
    fx, fy, fz = fg.face_coefficients(a)
    N = nx * ny * nz
    M = np.zeros((N, N))
    idx = lambda i, j, k: i + nx * (j + ny * k)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                faces = [(fx[k, j, i], (i - 1, j, k)), (fx[k, j, i + 1], (i + 1, j, k)),
                         (fy[k, j, i], (i, j - 1, k)), (fy[k, j + 1, i], (i, j + 1, k)),
                         (fz[k, j, i], (i, j, k - 1)), (fz[k + 1, j, i], (i, j, k + 1))]
                for c, (ii, jj, kk) in faces:
                    M[p, p] += c
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        M[p, idx(ii, jj, kk)] -= c
    return M


@pytest.mark.parametrize("field", ["lognormal", "checkerboard"])
def test_front_is_brute_force_schur_complement(field):
    nx, ny, nz, below = 4, 4, 5, 2
    a = (fg.coefficient_lognormal(nx, ny, nz, 0.7, seed=3) if field == "lognormal"
         else fg.coefficient_checkerboard(nx, ny, nz, cell=2, contrast=1e3))
    M = _dense_3d_operator(a)
    s = np.arange(nx * ny) + nx * ny * below
    i = np.setdiff1d(np.arange(M.shape[0]), s)
    S = M[np.ix_(s, s)] - M[np.ix_(s, i)] @ np.linalg.solve(M[np.ix_(i, i)], M[np.ix_(i, s)])
    F = fg.plane_front(a, below)
    assert np.allclose(F, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())


@pytest.mark.parametrize("field", ["lognormal", "checkerboard"])
@pytest.mark.parametrize("shape", [(4, 5, 2, 2), (5, 4, 3, 1), (3, 4, 1, 0)])
def test_line_elimination_is_brute_force_schur_complement(field, shape):
    """The elimination across the lines of the slabs (the one the thin n = 32768
    front takes) against the dense Schur complement, both line directions."""
    nx, ny, below, above = shape
    nz = below + 1 + above
    a = (fg.coefficient_lognormal(nx, ny, nz, 0.7, seed=5) if field == "lognormal"
         else fg.coefficient_checkerboard(nx, ny, nz, cell=2, contrast=1e3))
    M = _dense_3d_operator(a)
    s = np.arange(nx * ny) + nx * ny * below
    i = np.setdiff1d(np.arange(M.shape[0]), s)
    S = M[np.ix_(s, s)] - M[np.ix_(s, i)] @ np.linalg.solve(M[np.ix_(i, i)], M[np.ix_(i, s)])
    F = fg.plane_front(a, below, method="rows")
    assert np.allclose(F, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())


def test_line_and_plane_eliminations_agree():
    a = fg.coefficient_lognormal(12, 20, 9, 0.5, seed=0)
    F1 = fg.plane_front(a, 4, method="planes")
    F2 = fg.plane_front(a, 4, method="rows")
    assert np.abs(F1 - F2).max() <= 1e-13 * np.abs(F1).max()


def test_elastic_operator_spd_and_consistent():
    """The 3-dof elasticity operator: symmetric positive definite, and with a
    constant shear modulus it annihilates every linear displacement field
    u(x) = M x + c on the nodes whose stencil stays inside the box (the
    discrete Laplacian of a linear field and the gradient of a constant
    divergence both vanish)."""
    nz, ny, nx = 6, 6, 6
    K = fg.elastic_operator(np.ones((nz, ny, nx)), nu=0.3).toarray()
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0
    rng = np.random.default_rng(3)
    M = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(float)    # x-fastest node order
    u = (X @ M.T + c).reshape(-1)                                            # 3 dofs per node
    r = (K @ u).reshape(-1, 3)
    inner = ((X > 1) & (X < np.array([nx, ny, nz]) - 2)).all(axis=1)
    assert inner.sum() > 0
    assert np.abs(r[inner]).max() <= 1e-12 * np.abs(K).max() * np.abs(u).max()
    assert np.abs(r[~inner]).max() > 1e-3   # the Dirichlet boundary does act


def test_elastic_front_is_brute_force_schur_complement():
    mu = fg.coefficient_lognormal(4, 3, 5, 0.7, seed=2)
    K = fg.elastic_operator(mu).toarray()
    m = 3 * 4 * 3
    s = np.arange(m) + 2 * m
    i = np.setdiff1d(np.arange(K.shape[0]), s)
    S = K[np.ix_(s, s)] - K[np.ix_(s, i)] @ np.linalg.solve(K[np.ix_(i, i)], K[np.ix_(i, s)])
    F = fg.elastic_front(mu, 2)
    assert np.allclose(F, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    E = fg.make_elastic_front(8, 8, 2, 2, leaf_nodes=16)
    np.linalg.cholesky(E.A)
    assert E.n == 192 and E.bounds[-1] == 192 and np.all(np.diff(E.bounds) % 3 == 0)


def test_front_invariants():
    F = fg.make_front(8, 6, 3, 2, "lognormal", 0.5, leaf=8, seed=0)
    A = F.A
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)                                   # SPD
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0.0                                 # M-matrix signs
    assert A.sum(axis=1).min() >= -1e-12 * np.abs(A).max()  # row sums >= 0
    # tree order: every leaf is a rectangle of the plane, sizes add up to n
    assert F.bounds[-1] == F.n and np.all(np.diff(F.bounds) > 0)
    assert sorted(F.perm.tolist()) == list(range(F.n))


def test_constant_coefficient_stencil_is_translation_invariant():
    a = np.ones((7, 10, 10))
    F = fg.plane_front(a, 3)                                # natural order, 10x10 plane
    idx = lambda x, y: x + 10 * y
    # interior couplings depend only on the offset (away from the Dirichlet edges)
    ref = F[idx(4, 4), idx(5, 6)]
    assert math.isclose(F[idx(5, 5), idx(6, 7)], ref, rel_tol=1e-2)


def test_rng_is_counter_based_and_normal():
    z = fg.normal(7, np.arange(200000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert np.array_equal(fg.normal(7, np.arange(10, 20)), z[10:20])
    # SplitMix64 reference value for input 0 (published test vector of the mixer)
    assert int(fg.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF


def test_bisection_tree_geometry():
    perm, bounds, L, rects = fg.bisection_order(24, 24, 64)
    assert L == 4 and np.all(np.diff(bounds) == 36)
    perm, bounds, L, rects = fg.bisection_order(64, 64, 128)
    assert L == 5 and np.all(np.diff(bounds) == 128)
    perm, bounds, L, rects = fg.bisection_order(256, 128, 256)
    assert L == 7 and np.all(np.diff(bounds) == 256)
    perm, bounds, L, rects = fg.bisection_order(64, 64, 128)
    # the first split of a 64x64 plane is x < 32 | x >= 32
    x = perm % 64
    assert x[:2048].max() == 31 and x[2048:].min() == 32 and len(perm) == 4096


def test_octree_count():
    boxes = fg.octree_boxes(64, 8)
    assert len(boxes) == 585
    assert sorted({s for s, _ in boxes}) == [8, 16, 32, 64]


# --------------------------------------------------------------------------- dense LU
def test_lu_partial_textbook_example():
    # Hand elimination of [[1,2,3],[4,5,6],[7,8,10]]: pivot 7 (row 3), then 6/7
    # (original row 1) -> perm [2,0,1], L = [[1],[1/7,1],[4/7,1/2,1]],
    # U = [[7,8,10],[0,6/7,11/7],[0,0,-1/2]].
    A = np.array([[1.0, 2, 3], [4, 5, 6], [7, 8, 10]])
    LU, perm = O.lu_partial(A)
    assert perm.tolist() == [2, 0, 1]
    L = np.tril(LU, -1) + np.eye(3)
    U = np.triu(LU)
    assert np.allclose(L, [[1, 0, 0], [1 / 7, 1, 0], [4 / 7, 0.5, 1]], atol=1e-15)
    assert np.allclose(U, [[7, 8, 10], [0, 6 / 7, 11 / 7], [0, 0, -0.5]], atol=1e-15)
    x = O.lu_solve(LU, perm, np.array([6.0, 15, 25]))
    assert np.allclose(x, [1, 1, 1], atol=1e-14)


def test_lu_partial_matches_lapack_pivots_and_residual():
    import scipy.linalg as sla
    rng = np.random.default_rng(0)
    A = rng.standard_normal((60, 60))
    LU, perm = O.lu_partial(A)
    P, L, U = sla.lu(A)                    # A = P L U
    assert np.array_equal(np.argmax(P, axis=0), perm)
    assert np.allclose(np.tril(LU, -1) + np.eye(60), L, atol=1e-12)
    b = rng.standard_normal(60)
    x = O.lu_solve(LU, perm, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-14 * np.linalg.cond(A)


def test_lu_partial_zero_pivot_raises():
    with pytest.raises(np.linalg.LinAlgError):
        O.lu_partial(np.array([[0.0, 1.0], [0.0, 2.0]]))


# --------------------------------------------------------------------------- ACA
def _aca_matrix(M, tol, cap=1 << 30):
    return O.aca(lambda i: M[i], lambda j: M[:, j], M.shape[0], M.shape[1], tol, cap)


def test_aca_hand_example():
    # Hand run of partial-pivoting ACA on [[1,3,2],[2,1,0],[0,0,5]]:
    # row 0 -> |3| at col 1, v1 = [1/3,1,2/3], u1 = [3,1,0]; next row = 1 (|u1|);
    # residual row 1 = [5/3,0,-2/3] -> col 0, v2 = [1,0,-2/5], u2 = [0,5/3,0];
    # row 2 residual [0,0,5] -> col 2, v3 = [0,0,1], u3 = [0,0,5].
    M = np.array([[1.0, 3, 2], [2, 1, 0], [0, 0, 5]])
    r = _aca_matrix(M, 1e-15)
    assert r.rows == [0, 1, 2] and r.cols == [1, 0, 2]
    assert np.allclose(r.V[:, 0], [1 / 3, 1, 2 / 3], atol=1e-15)
    assert np.allclose(r.U[:, 1], [0, 5 / 3, 0], atol=1e-15)
    assert np.allclose(r.V[:, 1], [1, 0, -0.4], atol=1e-15)
    assert np.allclose(r.U @ r.V.T, M, atol=1e-14)


def test_aca_tie_break_and_zero_row():
    # equal magnitudes in the first row -> lowest column; a zero first row is
    # skipped (marked used) and the lowest unused row is tried next.
    M = np.array([[2.0, -2.0, 1.0], [1.0, 1.0, 1.0]])
    r = _aca_matrix(M, 1e-15)
    assert r.cols[0] == 0
    Z = np.array([[0.0, 0.0, 0.0], [0.0, 4.0, 1.0], [0.0, 2.0, 3.0]])
    r = _aca_matrix(Z, 1e-15)
    assert r.rows[0] == 1 and r.cols[0] == 1
    assert np.allclose(r.U @ r.V.T, Z, atol=1e-14)


@pytest.mark.parametrize("k", [1, 4, 9])
def test_aca_recovers_exact_rank_k(k):
    rng = np.random.default_rng(k)
    M = rng.standard_normal((70, k)) @ rng.standard_normal((k, 55))
    r = _aca_matrix(M, 1e-10)
    assert r.U.shape[1] in (k, k + 1)
    assert np.linalg.norm(M - r.U @ r.V.T) / np.linalg.norm(M) < 1e-13


def test_aca_norm_recurrence_is_frobenius_norm():
    rng = np.random.default_rng(5)
    x = np.linspace(0, 1, 80)
    M = 1.0 / (1.0 + np.abs(x[:, None] - (x[None, :] + 1.5)))   # smooth kernel
    r = _aca_matrix(M, 1e-9)
    exact = np.linalg.norm(r.U @ r.V.T) ** 2
    assert math.isclose(r.norm2, exact, rel_tol=1e-12)
    assert np.linalg.norm(M - r.U @ r.V.T) / np.linalg.norm(M) < 1e-7


def test_aca_rank_cap():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((30, 30))
    r = _aca_matrix(M, 1e-12, cap=5)
    assert r.U.shape[1] == 5 and r.cap_hit


def test_aca_zero_block():
    r = _aca_matrix(np.zeros((4, 6)), 1e-6)
    assert r.U.shape == (4, 0) and r.V.shape == (6, 0)


# ------------------------------------------------- ACA and LU in FP32 arithmetic
# The single-precision compression mode rounds the block entries to FP32 and
# forms every residual entry term by term, one FP32 multiply and one FP32
# subtract per term, every pivot scaling and LU update in FP32.  The values
# below are worked out by hand from IEEE round-to-nearest-even:
#   fl32(1/3) = 11184811 * 2^-25, fl32(2/3) = 11184811 * 2^-24,
#   fl32(3 * fl32(1/3)) = fl32(1 + 2^-25) = 1, fl32(3 * fl32(2/3)) = fl32(2 + 2^-24) = 2,
#   fl32(1 - fl32(1/3)) = fl32(11184810.5 * 2^-24) = 11184810 * 2^-24 (tie to even).
THIRD32 = 11184811 * 2.0 ** -25


def _aca_dense(A, tol, dtype, cap=100):
    m, n = A.shape
    return O.aca(lambda i: A[i, :], lambda j: A[:, j], m, n, tol, cap, dtype)


def test_aca_fp32_rounds_entries_first():
    # 1 and 1 + 2^-30 are the same FP32 number: a tie, so the lowest column wins;
    # in FP64 the larger entry wins.
    A = np.array([[1.0, 1.0 + 2.0 ** -30, 0.5], [0.25, 0.5, 2.0], [0.5, 0.125, 1.0]])
    assert _aca_dense(A, 1e-12, np.float32).cols[0] == 0
    assert _aca_dense(A, 1e-12, np.float64).cols[0] == 1


def test_aca_fp32_hand_run_rounding_points():
    """Step 1 pivots on the 3 of row 0, v_1 = [1, fl32(1/3), fl32(2/3)], u_1 = [3, 3, 1].
    Step 2 takes row 1: per-term FP32 gives r = [0, 2^-22, -2^-22], a tie, so j_2 = 1
    and v_2 = [0, 1, -1], u_2 = [0, 2^-22, -fl32(1/3)].  Forming the products
    u_1[1] v_1 exactly and rounding the residual once would give
    r = [0, 7 * 2^-25, -10 * 2^-25] and j_2 = 2 instead."""
    A = np.array([[3.0, 1.0, 2.0],
                  [3.0, 1.0 + 2.0 ** -22, 2.0 - 2.0 ** -22],
                  [1.0, 0.0, 0.0]])
    r = _aca_dense(A, 1e-12, np.float32)
    assert r.rows[:2] == [0, 1] and r.cols[:2] == [0, 1]
    assert r.V[:, 0].tolist() == [1.0, THIRD32, 2 * THIRD32]
    assert r.U[:, 0].tolist() == [3.0, 3.0, 1.0]
    assert r.V[:, 1].tolist() == [0.0, 1.0, -1.0]
    assert r.U[:, 1].tolist() == [0.0, 2.0 ** -22, -THIRD32]
    # the wrong rounding point changes the decision (the reading is not vacuous)
    rr = np.float32(A[1, 1]) - np.float32(np.float64(3.0) * THIRD32)
    r_once = np.float32(A[1, 1] - 3.0 * THIRD32), np.float32(A[1, 2] - 3.0 * 2 * THIRD32)
    assert float(rr) == 2.0 ** -22 and abs(r_once[1]) > abs(r_once[0])


def test_aca_fp32_equals_fp64_on_dyadic_block():
    """Two rank-one blocks on disjoint rows/columns with power-of-two pivots: every
    FP32 operation is exact, so both modes take the same steps and values."""
    A = np.zeros((6, 5))
    A[np.ix_([0, 3], [1, 4])] = [[8.0, 4.0], [4.0, 2.0]]
    A[np.ix_([1, 5], [0, 2])] = [[16.0, 2.0], [4.0, 0.5]]
    A[2, 3] = 0.25
    r32, r64 = _aca_dense(A, 1e-12, np.float32), _aca_dense(A, 1e-12, np.float64)
    assert r32.rows == r64.rows and r32.cols == r64.cols and len(r32.rows) == 3
    assert np.array_equal(r32.U, r64.U) and np.array_equal(r32.V, r64.V)
    assert np.array_equal(r32.U @ r32.V.T, A)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_aca_fp32_recovers_rank_k_to_single_precision(k):
    rng = np.random.default_rng(k)
    X = rng.standard_normal((48, k)).astype(np.float32).astype(np.float64)
    Y = rng.standard_normal((40, k)).astype(np.float32).astype(np.float64)
    A = X @ Y.T
    r = _aca_dense(A, 1e-5, np.float32)
    assert len(r.rows) in (k, k + 1)
    assert np.linalg.norm(A - r.U @ r.V.T) <= 2e-5 * np.linalg.norm(A)


def test_full_pivot_lu_fp32_hand_example():
    # [[3,1],[1,1]]: pivot 3, multiplier fl32(1/3), second pivot fl32(1 - fl32(1/3))
    LU, prow, pcol, r = O.full_pivot_lu(np.array([[3.0, 1.0], [1.0, 1.0]]), 1e-12, dtype=np.float32)
    assert r == 2 and LU.dtype == np.float32
    assert float(LU[0, 0]) == 3.0 and float(LU[1, 0]) == THIRD32
    assert float(LU[1, 1]) == 11184810 * 2.0 ** -24
    LU64, _, _, _ = O.full_pivot_lu(np.array([[3.0, 1.0], [1.0, 1.0]]), 1e-12)
    assert float(LU64[1, 1]) != float(LU[1, 1])


def test_bdlr_fp32_skeleton_hand_example():
    # path graph 0-1-2-3, rows {0,1}, columns {2,3}: boundary rows I = [1, 0],
    # columns J = [2, 3] (distance 0, then 1); A(I,J) = [[3,1],[1,1]]
    A = np.array([[5.0, 2.0, 1.0, 1.0], [2.0, 5.0, 3.0, 1.0], [1.0, 3.0, 5.0, 2.0], [1.0, 1.0, 2.0, 5.0]])
    rowptr = np.array([0, 1, 3, 5, 6], dtype=np.int32)
    colind = np.array([1, 0, 2, 1, 3, 2], dtype=np.int32)
    r = O.bdlr(A, rowptr, colind, range(0, 2), range(2, 4), 1e-12, depth=1, dtype=np.float32)
    assert r.I == [1, 0] and r.J == [2, 3] and r.Ir == [1, 0] and r.Jr == [2, 3]
    assert r.pivots.tolist() == [3.0, 11184810 * 2.0 ** -24]
    # rank 2 of a 2 x 2 block: the skeleton reproduces it to FP32 rounding
    assert np.allclose(r.U @ r.V.T, A[:2, 2:], rtol=0, atol=1e-6)


# --------------------------------------------------------------------------- BDLR
def test_boundary_distance_on_grid():
    # 4x4 plane, natural order; rows = left half (x in {0,1}) is not contiguous in
    # natural order, so use the tree order of bisection_order(4,4,8): first half x<2.
    perm, bounds, L, _ = fg.bisection_order(4, 4, 8)
    rowptr, colind = fg.plane_graph(4, 4, perm)
    sel, dist = O.boundary_distance(rowptr, colind, range(0, 8), range(8, 16), depth=5)
    xs = perm[:8] % 4
    assert np.array_equal(dist, np.where(xs == 1, 0, 1))       # x=1 column is d=0
    assert [int(perm[v] % 4) for v in sel[:4]] == [1, 1, 1, 1]
    sel0, _ = O.boundary_distance(rowptr, colind, range(0, 8), range(8, 16), depth=0)
    assert len(sel0) == 4


def test_full_pivot_lu_hand_example():
    # [[1,4],[2,3]]: largest |4| at (0,1) -> swap columns; l = 3/4; 2 - 3/4 = 5/4.
    LU, prow, pcol, r = O.full_pivot_lu(np.array([[1.0, 4.0], [2.0, 3.0]]), 0.0)
    assert r == 2 and prow.tolist() == [0, 1] and pcol.tolist() == [1, 0]
    assert np.allclose(np.diag(LU), [4.0, 1.25])
    # truncation: keep while |p_k| >= eps |p_1|
    _, _, _, r = O.full_pivot_lu(np.array([[1.0, 4.0], [2.0, 3.0]]), 0.5)
    assert r == 1


def test_full_pivot_lu_reconstructs():
    rng = np.random.default_rng(2)
    Ah = rng.standard_normal((12, 9))
    LU, prow, pcol, r = O.full_pivot_lu(Ah, 0.0)
    assert r == 9
    L = np.tril(LU, -1)[:, :9] + np.eye(12, 9)
    U = np.triu(LU[:9, :9])
    assert np.allclose(Ah[prow][:, pcol], L @ U, atol=1e-13)


def _front_small(leaf=16):
    return fg.make_front(12, 12, 4, 4, "lognormal", 0.5, leaf=leaf, seed=0)


def test_bdlr_closed_form_skeleton():
    F = _front_small()
    A = F.A
    tree = O.make_tree(F.n, 16, F.bounds)
    a0, a1 = tree.range(1, 0)
    b0, b1 = tree.range(1, 1)
    res = O.bdlr(A, F.rowptr, F.colind, range(a0, a1), range(b0, b1), 1e-6, 3)
    r = len(res.Ir)
    assert r > 0 and len(set(res.Ir)) == r and set(res.Ir) <= set(res.I)
    C = A[a0:a1][:, res.Jr]
    R = A[res.Ir][:, b0:b1]
    closed = C @ np.linalg.solve(A[np.ix_(res.Ir, res.Jr)], R)
    assert np.allclose(res.U @ res.V.T, closed, rtol=1e-10, atol=1e-12 * np.abs(closed).max())


def test_bdlr_exact_when_skeleton_has_full_rank():
    rng = np.random.default_rng(9)
    n = 32
    k = 3
    A = np.eye(n) * 10
    A[:16, 16:] = rng.standard_normal((16, k)) @ rng.standard_normal((k, 16))
    A[16:, :16] = A[:16, 16:].T
    # chain graph 0-1-...-31: the boundary of [0,16) is vertex 15
    rows = [[1]] + [[i - 1, i + 1] for i in range(1, n - 1)] + [[n - 2]]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.asarray([c for r in rows for c in r], dtype=np.int32)
    res = O.bdlr(A, rowptr, colind, range(0, 16), range(16, 32), 1e-10, 6)
    assert len(res.Ir) == k
    blk = A[:16, 16:]
    assert np.linalg.norm(res.U @ res.V.T - blk) / np.linalg.norm(blk) < 1e-12


def _top_block(F, leaf=64):
    tree = O.make_tree(F.n, leaf, F.bounds)
    a0, a1 = tree.range(1, 0)
    b0, b1 = tree.range(1, 1)
    return range(a0, a1), range(b0, b1)


def test_bdlr_error_never_beats_svd():
    """Figs. 4-6 diagnostics: by Eckart-Young, no rank-r approximation beats the
    truncated SVD in the Frobenius norm, so the BDLR error at every rank is at
    least the SVD's; and the largest pivots sit on the boundary (distance 0)."""
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    R, C = _top_block(F)
    D = O.bdlr_diagnostics(F.A, F.rowptr, F.colind, R, C, 1e-8, 6)
    assert len(D["bdlr_err"]) >= 20
    assert np.all(D["bdlr_err"] >= D["svd_err"] * (1 - 1e-9))
    assert np.all(np.diff(D["singular_values"]) <= 0)
    assert D["row_dist"][0] == 0 and D["col_dist"][0] == 0
    assert np.mean(D["row_dist"][:8]) <= np.mean(D["row_dist"])


def test_heldout_error_closed_forms():
    rng = np.random.default_rng(1)
    X, Y = rng.standard_normal((30, 3)), rng.standard_normal((20, 3))
    A = np.zeros((50, 50))
    A[:30, 30:] = X @ Y.T
    R, C = range(0, 30), range(30, 50)
    # exact factors: no residual
    assert O.heldout_error(A, R, C, X, Y, [1, 5], [33], [0], [30]) <= 1e-15
    # no factors: the held-out rows' and columns' share of the examined mass
    Z, W = np.zeros((30, 3)), np.zeros((20, 3))
    Hr, Hc, I, J = [2, 7], [35], [0, 1], [30, 31]
    num = sum(np.sum(A[h, 30:] ** 2) for h in Hr) + np.sum(A[:30, 35] ** 2)
    den = sum(np.sum(A[h, 30:] ** 2) for h in Hr + I) + sum(np.sum(A[:30, h] ** 2) for h in Hc + J)
    assert O.heldout_error(A, R, C, Z, W, Hr, Hc, I, J) == pytest.approx(np.sqrt(num / den), rel=1e-14)
    assert O.heldout_error(A, R, C, Z, W, [], [], I, J) == 0.0


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_adaptive_bdlr_takes_the_least_sufficient_depth(eps):
    """Section 5.3's adaptive pseudo-skeleton: the returned depth meets eps on
    its held-out rows and columns and the depth below it does not."""
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    R, C = _top_block(F)
    res, d, err = O.bdlr_adaptive(F.A, F.rowptr, F.colind, R, C, eps)
    assert err <= eps
    if d > 1:
        prev = O.bdlr(F.A, F.rowptr, F.colind, R, C, eps, d - 1)
        _, dr = O.boundary_distance(F.rowptr, F.colind, R, C, d)
        _, dc = O.boundary_distance(F.rowptr, F.colind, C, R, d)
        Hr = [R.start + i for i in np.flatnonzero(dr == d)]
        Hc = [C.start + j for j in np.flatnonzero(dc == d)]
        assert O.heldout_error(F.A, R, C, prev.U, prev.V, Hr, Hc, prev.I, prev.J) > eps
    blk = F.A[R.start:R.stop, C.start:C.stop]
    assert np.linalg.norm(blk - res.U @ res.V.T) / np.linalg.norm(blk) < 20 * eps


# --------------------------------------------------------------------------- HODLR
def test_make_tree_halving():
    t = O.make_tree(576, 64)
    assert t.L == 4 and t.range(4, 0) == (0, 36) and t.range(0, 0) == (0, 576)
    t = O.make_tree(100, 30)
    assert t.L == 2 and t.bounds.tolist() == [0, 25, 50, 75, 100]


def test_assemble_exact_hodlr_matrix():
    # A matrix that is exactly HODLR (rank-2 off-diagonal blocks) is reproduced.
    rng = np.random.default_rng(4)
    n = 64
    tree = O.make_tree(n, 16)
    A = np.diag(rng.uniform(5, 6, n))
    for l in range(tree.L):
        for i in range(1 << l):
            a0, a1 = tree.range(l + 1, 2 * i)
            b0, b1 = tree.range(l + 1, 2 * i + 1)
            A[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, 2)) @ rng.standard_normal((2, b1 - b0)) * 0.1
            A[b0:b1, a0:a1] = rng.standard_normal((b1 - b0, 2)) @ rng.standard_normal((2, a1 - a0)) * 0.1
    for l in range(tree.L + 1):          # leaf blocks random
        pass
    blocks = O.build(A, tree, "aca", 1e-12)
    K = O.assemble(A, tree, blocks)
    assert np.linalg.norm(K - A) / np.linalg.norm(A) < 1e-13


def test_one_level_woodbury_by_hand():
    # One level: K~ = diag(K1,K2) + [[0, U1 V12^T],[U2 V21^T, 0]] = D + U C V^T with
    # U = blkdiag(U1,U2), V^T = [[0, V12^T],[V21^T, 0]]; Woodbury:
    # K~^-1 = D^-1 - D^-1 U (I + V^T D^-1 U)^-1 V^T D^-1.
    rng = np.random.default_rng(8)
    F = fg.make_front(8, 8, 3, 3, "lognormal", 0.5, leaf=32, seed=1)
    A = F.A
    tree = O.make_tree(F.n, 32, F.bounds)
    assert tree.L == 1
    blocks = O.build(A, tree, "aca", 1e-3)
    blk = blocks[(0, 0)]
    K = O.assemble(A, tree, blocks)
    D = np.zeros_like(A)
    D[:32, :32] = A[:32, :32]
    D[32:, 32:] = A[32:, 32:]
    ra, rb = blk.Ua.shape[1], blk.Ub.shape[1]
    Ublk = np.zeros((64, ra + rb))
    Ublk[:32, :ra] = blk.Ua
    Ublk[32:, ra:] = blk.Ub
    Vt = np.zeros((ra + rb, 64))
    Vt[:ra, 32:] = blk.Vab.T
    Vt[ra:, :32] = blk.Vba.T
    assert np.allclose(D + Ublk @ Vt, K, atol=1e-13)
    Dinv = np.linalg.inv(D)
    Kinv = Dinv - Dinv @ Ublk @ np.linalg.solve(np.eye(ra + rb) + Vt @ Dinv @ Ublk, Vt @ Dinv)
    Fac = O.factor(A, tree, blocks)
    b = rng.standard_normal((64, 3))
    assert np.allclose(O.solve(Fac, b), Kinv @ b, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("method", ["aca", "bdlr"])
def test_solve_equals_dense_inverse_of_assembled(method):
    F = fg.make_front(16, 16, 4, 4, "lognormal", 0.5, leaf=16, seed=0)
    A = F.A
    tree = O.make_tree(F.n, 16, F.bounds)
    blocks = O.build(A, tree, method, 1e-4, graph=(F.rowptr, F.colind), depth=4)
    K = O.assemble(A, tree, blocks)
    Fac = O.factor(A, tree, blocks)
    b = fg.rhs(F.n, 3, seed=1)
    x = O.solve(Fac, b)
    ref = np.linalg.solve(K, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-12 * np.linalg.cond(K)
    # the approximation error of K~ is small at this tolerance
    assert np.linalg.norm(K - A) / np.linalg.norm(A) < 1e-3


def test_factor_d_is_inverse_times_u():
    F = _front_small()
    A = F.A
    tree = O.make_tree(F.n, 16, F.bounds)
    blocks = O.build(A, tree, "aca", 1e-6)
    K = O.assemble(A, tree, blocks)
    Fac = O.factor(A, tree, blocks)
    # d_i^(l) = (K~ restricted to node (l,i))^-1 U_i^(l)
    for (l, i), d in Fac.d.items():
        s, e = tree.range(l, i)
        par = blocks[(l - 1, i // 2)]
        U = par.Ua if i % 2 == 0 else par.Ub
        ref = np.linalg.solve(K[s:e, s:e], U)
        assert np.allclose(d, ref, rtol=1e-10, atol=1e-12 * max(1.0, np.abs(ref).max()))


# --------------------------------------------------------------------------- GMRES
def test_gmres_diagonal_distinct_eigenvalues():
    vals = np.repeat([1.0, 2.0, 5.0, 7.0], 10)
    A = np.diag(vals)
    b = np.random.default_rng(0).standard_normal(40)
    r = O.gmres(A, b, tol=1e-12, max_iter=50)
    assert r.iters <= 4 and r.true_relres <= 1e-12


def test_gmres_exact_preconditioner_one_step():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 30)) + 30 * np.eye(30)
    b = rng.standard_normal(30)
    r = O.gmres(A, b, prec=lambda v: np.linalg.solve(A, v), tol=1e-12)
    assert r.iters == 1 and r.true_relres < 1e-13


def test_gmres_iterate_is_krylov_least_squares():
    rng = np.random.default_rng(2)
    n = 24
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    M = np.diag(rng.uniform(0.5, 2.0, n))               # right preconditioner M^-1
    b = rng.standard_normal(n)
    for k in (1, 3, 6):
        r = O.gmres(A, b, prec=lambda v: M @ v, tol=1e-30, max_iter=k)
        # brute force: x in M K_k(A M, b), minimise ||b - A x||
        Kry = [b]
        for _ in range(k - 1):
            Kry.append(A @ (M @ Kry[-1]))
        Kmat = M @ np.stack(Kry, axis=1)
        c, *_ = np.linalg.lstsq(A @ Kmat, b, rcond=None)
        assert np.allclose(r.x, Kmat @ c, rtol=1e-8, atol=1e-10)
        assert math.isclose(r.est_relres, np.linalg.norm(b - A @ (Kmat @ c)) / np.linalg.norm(b),
                            rel_tol=1e-6)


def test_gmres_restart_one_is_minimal_residual_iteration():
    """GMRES(1) (restart = 1) is the minimal residual iteration:
    x_{k+1} = x_k + a_k M r_k, a_k = (r_k . A M r_k) / ||A M r_k||^2."""
    rng = np.random.default_rng(4)
    n = 20
    A = rng.standard_normal((n, n)) + 8 * np.eye(n)
    M = np.diag(rng.uniform(0.5, 2.0, n))
    b = rng.standard_normal(n)
    x = np.zeros(n)
    for k in range(1, 6):
        r = b - A @ x
        q = A @ (M @ r)
        x = x + (r @ q) / (q @ q) * (M @ r)
        res = O.gmres(A, b, prec=lambda v: M @ v, tol=1e-30, max_iter=k, restart=1)
        assert res.iters == k and not res.converged
        assert np.allclose(res.x, x, rtol=1e-10, atol=1e-12)


def test_gmres_two_restart_cycles_are_two_least_squares_solves():
    """GMRES(m) over two cycles: each cycle minimises ||b - A x|| over
    x_prev + M K_m(A M, r_prev), r_prev the true residual of the previous iterate."""
    rng = np.random.default_rng(5)
    n, m = 30, 4
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    M = np.diag(rng.uniform(0.5, 2.0, n))
    b = rng.standard_normal(n)
    x = np.zeros(n)
    for _ in range(2):
        r = b - A @ x
        Kry = [r]
        for _ in range(m - 1):
            Kry.append(A @ (M @ Kry[-1]))
        Kmat = M @ np.stack(Kry, axis=1)
        c, *_ = np.linalg.lstsq(A @ Kmat, r, rcond=None)
        x = x + Kmat @ c
    res = O.gmres(A, b, prec=lambda v: M @ v, tol=1e-30, max_iter=2 * m, restart=m)
    assert res.iters == 2 * m
    assert np.allclose(res.x, x, rtol=1e-8, atol=1e-10)


def test_gmres_zero_rhs_and_max_iter():
    A = np.eye(5) * 2
    r = O.gmres(A, np.zeros(5))
    assert r.iters == 0 and r.converged
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40)) + 2 * np.eye(40)
    r = O.gmres(A, rng.standard_normal(40), tol=1e-14, max_iter=3)
    assert r.iters == 3 and not r.converged


def test_hodlr_preconditioned_gmres_on_front():
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    A = F.A
    tree = O.make_tree(F.n, 64, F.bounds)
    blocks, Fac, P = O.hodlr_precond(A, tree, "aca", 1e-6)
    b = fg.rhs(F.n, 1, seed=1)[:, 0]
    r = O.gmres(A, b, prec=P, tol=1e-12)
    assert r.converged and r.true_relres <= 1e-12
    plain = O.gmres(A, b, tol=1e-12)
    assert r.iters < plain.iters
    assert O.dense_floor(A, b) < 1e-14


def test_precond_error_limits():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 20)) + 20 * np.eye(20)
    Om = rng.standard_normal((20, 4))
    assert O.precond_error(A, lambda v: np.linalg.solve(A, v), Om) < 1e-14
    e = O.precond_error(A, lambda v: v, Om)
    assert math.isclose(e, np.linalg.norm(Om - A @ Om) / np.linalg.norm(Om))


def _golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows.append(line)
    return rows


def test_precond_error_2norm_closed_forms():
    """P = A (exact inverse): 0.  P = I (no preconditioner) on an SPD A:
    max |1 - lambda_i|, from the eigenvalues.  P = 2A: 1/2 exactly."""
    rng = np.random.default_rng(4)
    M = rng.standard_normal((40, 40))
    A = M @ M.T / 40 + 0.5 * np.eye(40)
    assert O.precond_error_2norm(A, lambda X: np.linalg.solve(A, X)) < 1e-12
    lam = np.linalg.eigvalsh(A)
    assert O.precond_error_2norm(A, lambda X: X) == pytest.approx(np.abs(1 - lam).max(), rel=1e-12)
    assert O.precond_error_2norm(A, lambda X: np.linalg.solve(2 * A, X)) == pytest.approx(0.5, rel=1e-12)


def test_default_bdlr_depth_follows_table3():
    """Without an explicit depth the oracle's BDLR build takes the depth the
    paper pairs with the tolerance (Table 3 caption, tests/golden): the blocks
    and the candidate row / column sets equal those of the explicit depth, and
    the candidate sets differ from those of the next depth."""
    F = fg.make_front(16, 16, 4, 4, "lognormal", 0.5, leaf=16, seed=0)
    tree = O.make_tree(F.n, 16, F.bounds)
    graph = (F.rowptr, F.colind)
    rows = _golden("bdlr_depth_per_tolerance.txt")
    assert [(float(t), int(d)) for t, d in rows] == [(1e-1, 1), (1e-3, 3), (1e-5, 5)]
    for t, d in rows:
        tol, depth = float(t), int(d)
        auto = O.build(F.A, tree, "bdlr", tol, graph=graph)
        expl = O.build(F.A, tree, "bdlr", tol, graph=graph, depth=depth)
        other = O.build(F.A, tree, "bdlr", tol, graph=graph, depth=depth + 1)
        assert auto.keys() == expl.keys()
        for key in auto:
            assert np.array_equal(O.assemble(F.A, tree, {key: auto[key]}), O.assemble(F.A, tree, {key: expl[key]}))
            assert auto[key].info_ab.I == expl[key].info_ab.I and auto[key].info_ba.J == expl[key].info_ba.J
        assert any(auto[k].info_ab.I != other[k].info_ab.I for k in auto)


@pytest.mark.parametrize("method", ["aca", "bdlr"])
def test_iterations_fall_as_the_tolerance_tightens(method):
    """The preconditioner improves with the compression tolerance: GMRES
    iterations to 1e-10 (the paper's target) fall from 1e-1 to 1e-3 to 1e-5 on
    the 576 front, the trend of the paper's Table 3 (ACA: e.g. 223, 72, 15
    iterations on its 23K cube front), and every solve converges."""
    F = fg.make_front(24, 24, 8, 8, "lognormal", 0.5, leaf=64, seed=0)
    tree = O.make_tree(F.n, 64, F.bounds)
    b = fg.rhs(F.n, 1, seed=1)[:, 0]
    its = []
    for tol in (1e-1, 1e-3, 1e-5):
        _, _, P = O.hodlr_precond(F.A, tree, method, tol, graph=(F.rowptr, F.colind))
        r = O.gmres(F.A, b, prec=P, tol=1e-10)
        assert r.converged
        its.append(r.iters)
    assert its[0] > its[1] > its[2], its

