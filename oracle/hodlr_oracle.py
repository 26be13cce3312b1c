"""FP64 CPU oracle of the HODLR-preconditioned GMRES frontal solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or runs this
module; only the tests, the smoke check and the benchmark's CPU-baseline leg do.
It shares no code with the CUDA path: every step below is written from the paper
(Aminfar, Ambikasaran, Darve, "A Fast Block Low-Rank Dense Solver with
Applications to Finite-Element Matrices", arXiv:1403.5337) in plain NumPy FP64,
single-threaded by intent, in the paper's order and notation.  A library call is
used only as one whole step (a matrix product, or LAPACK's partial-pivoting LU
for the dense comparator), never to block or reorder the method.

Contents and the passage each follows
-------------------------------------
* Tree                 -- the HODLR partition of Section 4.1 (eq. HODLR2).
* lu_partial/lu_solve  -- dense LU with row partial pivoting (leaves, Woodbury
                          cores; the "conventional LU" comparator of Section 7).
* aca                  -- partial-pivoting ACA (Section 5.1, Rjasanow's scheme).
* bdlr                 -- boundary-distance row/column selection plus the
                          full-pivoting-LU pseudo-skeleton of Section 5.3.
* bdlr_adaptive        -- the same with the depth grown until the relative
                          Frobenius error on held-out rows and columns meets
                          the tolerance (Section 5.3).
* bdlr_diagnostics     -- pivot size vs boundary distance, singular values,
                          BDLR vs SVD error per rank (Figs. 4-6).
* build / assemble     -- the HODLR approximation K~ of the front.
* factor / solve       -- the recursive Woodbury factorisation and solve of
                          Section 4.3 (Factorize steps 1-5, Solve steps 1-3).
* gmres                -- GMRES (Section 3) with the HODLR solve as a right
                          preconditioner.
* precond_error        -- the randomised estimate ||(I - P^-1 A) Omega||_F/||Omega||_F.
* precond_error_2norm  -- the exact ||I - P^-1 A||_2 by dense SVD (small n).
* dense_floor          -- FP64 partial-pivoting dense LU residual floor.

Readings of points the paper leaves open (each is also tested):
* ACA start row 0; ties in every argmax go to the lowest index; an exactly zero
  residual row is marked used and the lowest unused row is tried next; stop after
  the term k with ||u_k|| ||v_k|| <= tol ||S_k||_F, or at min(m, n), or the rank cap;
  no recompression.  The residual entries are formed term by term in the order
  l = 0..k-1 with a separate multiply and subtract (two roundings), so that a
  decision taken on them is reproducible in any FP64 implementation that forms
  them the same way.
* BDLR distance is the BFS distance inside the subgraph induced on the row set
  (column set) from its boundary vertices; rows/columns with d <= depth, sorted by
  (d, index); full-pivot LU with ties to the lowest local row then column; keep
  pivots while |p_k| >= eps |p_1|.  The paper calls U(1:r,1:r)^-1 a lower
  triangular solve; it is an upper triangular one.
* "Z_1^0 = 0" is the empty n x 0 matrix; the leaves use partial-pivoting LU.
* GMRES: right preconditioning, x0 = 0, modified Gram-Schmidt, Givens rotations,
  2-norm relative to ||b||; restart from the current x only if the true residual
  misses the tolerance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------- tree
@dataclass
class Tree:
    """Complete binary HODLR tree (Section 4.1): level 0 is the whole index range,
    level L holds the leaves; node (l, i) covers the contiguous range spanned by
    leaves i*2^(L-l) .. (i+1)*2^(L-l) - 1.  Its children are (l+1, 2i), (l+1, 2i+1)."""
    n: int
    L: int
    bounds: np.ndarray

    def range(self, l: int, i: int):
        w = 1 << (self.L - l)
        return int(self.bounds[i * w]), int(self.bounds[(i + 1) * w])

    def size(self, l, i):
        a, b = self.range(l, i)
        return b - a


def make_tree(n: int, leaf: int, bounds=None) -> Tree:
    """Halve every node (lower half floor(size/2)) until all leaves are <= leaf,
    unless explicit leaf boundaries (2^L + 1 offsets) are supplied."""
    if bounds is not None:
        b = np.asarray(bounds, dtype=np.int64)
        L = int(round(math.log2(len(b) - 1)))
        assert (1 << L) + 1 == len(b) and b[0] == 0 and b[-1] == n
        return Tree(n, L, b)
    ranges = [(0, n)]
    while max(e - s for s, e in ranges) > leaf:
        ranges = [r for s, e in ranges for r in ((s, s + (e - s) // 2), (s + (e - s) // 2, e))]
    b = np.asarray([s for s, _ in ranges] + [n], dtype=np.int64)
    return Tree(n, int(round(math.log2(len(ranges)))), b)


# --------------------------------------------------------------------------- dense LU
def lu_partial(A: np.ndarray):
    """Gaussian elimination with row partial pivoting: P A = L U.

    Column k: pivot row = argmax_{i>=k} |a_ik| (lowest index on ties), swap, divide
    the column below the pivot by it, subtract the rank-1 product from the trailing
    block.  Returns (LU packed, perm) with A[perm] = L U.  Raises on a zero pivot."""
    a = np.array(A, dtype=np.float64, copy=True)
    m = a.shape[0]
    perm = np.arange(m)
    for k in range(m):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        if a[p, k] == 0.0:
            raise np.linalg.LinAlgError("zero pivot")
        if p != k:
            a[[k, p]] = a[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        a[k + 1:, k] /= a[k, k]
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    return a, perm


def lu_solve(LU: np.ndarray, perm: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B from lu_partial's factors: forward (unit L) then back (U)."""
    x = np.array(B, dtype=np.float64, copy=True)[perm]
    m = LU.shape[0]
    for i in range(m):
        x[i] -= LU[i, :i] @ x[:i]
    for i in range(m - 1, -1, -1):
        x[i] = (x[i] - LU[i, i + 1:] @ x[i + 1:]) / LU[i, i]
    return x


def dense_lu_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The paper's comparator (Section 7): a dense partial-pivoting LU solve.  Uses
    LAPACK getrf/getrs as one library step (same pivot rule as lu_partial)."""
    import scipy.linalg as sla
    return sla.lu_solve(sla.lu_factor(A), B)


# --------------------------------------------------------------------------- ACA
@dataclass
class ACAResult:
    U: np.ndarray                 # m x k
    V: np.ndarray                 # n x k  (block ~ U V^T)
    rows: list = field(default_factory=list)   # pivot rows i_1..i_k
    cols: list = field(default_factory=list)   # pivot columns j_1..j_k
    norm2: float = 0.0            # ||S_k||_F^2 by the recurrence
    cap_hit: bool = False


def aca(row, col, m: int, n: int, tol: float, rank_cap: int, dtype=np.float64) -> ACAResult:
    """Partial-pivoting adaptive cross approximation (Section 5.1).

    `row(i)` returns block row i (length n), `col(j)` block column j (length m).
    Step k: residual row r = row(i_k) - sum_l U[i_k,l] V[:,l]; j_k = argmax |r|;
    v_k = r / r[j_k]; u_k = col(j_k) - sum_l V[j_k,l] U[:,l]; next row =
    argmax over unused rows of |u_k|.  ||S_k||_F^2 is updated by
    ||S_{k-1}||^2 + 2 sum_{l<k} (u_k.u_l)(v_k.v_l) + ||u_k||^2 ||v_k||^2.

    `dtype` is the precision the residual rows/columns, their pivots and the
    scaled vectors are formed and decided in (float64, or float32 for the
    single-precision compression: block entries are rounded to float32 first).
    The dot products are formed in that precision too; the norm recurrence and
    the stopping test are evaluated in float64, the test in its squared form
    ||u_k||^2 ||v_k||^2 <= tol^2 ||S_k||_F^2."""
    dt = np.dtype(dtype)
    kmax = min(m, n, rank_cap)
    us, vs = [], []
    rows, cols = [], []
    used = np.zeros(m, dtype=bool)
    norm2 = 0.0
    i = 0
    res = ACAResult(np.zeros((m, 0)), np.zeros((n, 0)))
    while len(us) < kmax:
        r = np.array(row(i), dtype=np.float64).astype(dt)
        for l in range(len(us)):
            r = r - us[l][i] * vs[l]
        used[i] = True
        j = int(np.argmax(np.abs(r)))
        if r[j] == 0.0:
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = r / r[j]
        u = np.array(col(j), dtype=np.float64).astype(dt)
        for l in range(len(us)):
            u = u - vs[l][j] * us[l]
        cross = 0.0
        for l in range(len(us)):
            cross += float(u @ us[l]) * float(v @ vs[l])
        uu, vv = float(u @ u), float(v @ v)
        norm2 = norm2 + 2.0 * cross + uu * vv
        us.append(u)
        vs.append(v)
        rows.append(i)
        cols.append(j)
        # ||u_k|| ||v_k|| <= tol ||S_k||_F, tested squared (no square roots)
        if uu * vv <= tol * tol * max(norm2, 0.0):
            break
        if len(us) >= min(m, n):
            break
        cand = np.where(used, -1.0, np.abs(u))
        if cand.max() < 0:
            break
        i = int(np.argmax(cand))
    k = len(us)
    res.U = np.stack(us, axis=1).astype(np.float64) if k else np.zeros((m, 0))
    res.V = np.stack(vs, axis=1).astype(np.float64) if k else np.zeros((n, 0))
    res.rows, res.cols, res.norm2 = rows, cols, norm2
    res.cap_hit = (k == rank_cap and k < min(m, n))
    return res


# --------------------------------------------------------------------------- BDLR
def boundary_distance(rowptr, colind, own: range, other: range, depth: int):
    """Distances d of the vertices of `own` (a contiguous index range) from its
    boundary set, the vertices with an edge into `other` (Section 5.3, Fig. 1).
    Breadth-first search inside the subgraph induced on `own`.  Returns the list of
    vertices with d <= depth sorted by (d, index), and the full distance array
    (-1 = farther than depth or unreachable)."""
    o0, o1 = own.start, own.stop
    t0, t1 = other.start, other.stop
    dist = -np.ones(o1 - o0, dtype=np.int64)
    frontier = []
    for v in range(o0, o1):
        nb = colind[rowptr[v]:rowptr[v + 1]]
        if np.any((nb >= t0) & (nb < t1)):
            dist[v - o0] = 0
            frontier.append(v)
    d = 0
    while frontier and d < depth:
        nxt = []
        for v in frontier:
            for w in colind[rowptr[v]:rowptr[v + 1]]:
                if o0 <= w < o1 and dist[w - o0] < 0:
                    dist[w - o0] = d + 1
                    nxt.append(int(w))
        frontier = nxt
        d += 1
    sel = [(int(dist[v - o0]), v) for v in range(o0, o1) if dist[v - o0] >= 0]
    sel.sort()
    return [v for _, v in sel], dist


def full_pivot_lu(Ahat: np.ndarray, eps: float, kmax: int = 1 << 30, dtype=np.float64):
    """Full-pivoting LU of A^ (eq. Ahat): at step k take the largest |entry| of the
    trailing block (lowest local row, then column, on ties), swap it to (k,k),
    divide the column below by it and subtract the rank-1 product.  Stop before the
    first pivot with |p_k| < eps |p_1| (or a zero pivot, or exhaustion).
    At most kmax pivots are taken (the rank cap).  The arithmetic (division and
    the rank-1 update, a separate multiply and subtract) runs in `dtype`.
    Returns (LU packed, row order, column order, r)."""
    a = np.array(Ahat, dtype=np.float64).astype(dtype)
    mi, nj = a.shape
    prow = np.arange(mi)
    pcol = np.arange(nj)
    p1 = None
    r = 0
    for k in range(min(mi, nj, kmax)):
        blk = np.abs(a[k:, k:])
        flat = int(np.argmax(blk))            # row-major: lowest row, then column
        pi, pj = divmod(flat, blk.shape[1])
        pi += k
        pj += k
        piv = a[pi, pj]
        if p1 is None:
            p1 = float(abs(piv))
        if piv == 0.0 or float(abs(piv)) < eps * p1:
            break
        a[[k, pi]] = a[[pi, k]]
        prow[[k, pi]] = prow[[pi, k]]
        a[:, [k, pj]] = a[:, [pj, k]]
        pcol[[k, pj]] = pcol[[pj, k]]
        a[k + 1:, k] /= a[k, k]
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
        r = k + 1
    return a, prow, pcol, r


@dataclass
class BDLRResult:
    U: np.ndarray
    V: np.ndarray
    I: list        # selected rows (global), sorted by (d, index)
    J: list
    Ir: list       # kept pivot rows (global), pivot order
    Jr: list
    pivots: np.ndarray


def bdlr(A: np.ndarray, rowptr, colind, rows: range, cols: range, eps: float,
         depth: int, rank_cap: int = 1 << 30, dtype=np.float64) -> BDLRResult:
    """Boundary-distance low-rank approximation of the block A[rows, cols]
    (Section 5.3): R = A(I,:), C = A(:,J), A^ = A(I,J) = P^-1 L U Q^-1 truncated at
    eps, then C~ = (CQ)(:,1:r) U11^-1 and R~ = L11^-1 (PR)(1:r,:), block ~ C~ R~.
    Returns U = C~ (m x r) and V = R~^T (n x r).  The LU (and so the choice of
    I_r, J_r) runs in `dtype` on A^ rounded to it; the triangular solves are
    formed in float64 from the same rounded values."""
    I, _ = boundary_distance(rowptr, colind, rows, cols, depth)
    J, _ = boundary_distance(rowptr, colind, cols, rows, depth)
    m, n = len(rows), len(cols)
    if not I or not J:
        return BDLRResult(np.zeros((m, 0)), np.zeros((n, 0)), I, J, [], [], np.zeros(0))
    Ahat = A[np.ix_(I, J)]
    LU, prow, pcol, r = full_pivot_lu(Ahat, eps, rank_cap, dtype)
    LU = LU.astype(np.float64)
    Ir = [I[p] for p in prow[:r]]
    Jr = [J[p] for p in pcol[:r]]
    Cr = A[rows.start:rows.stop][:, Jr].astype(dtype).astype(np.float64)   # (CQ)(:,1:r)
    Rr = A[Ir][:, cols.start:cols.stop].astype(dtype).astype(np.float64)   # (PR)(1:r,:)
    U11 = np.triu(LU[:r, :r])
    L11 = np.tril(LU[:r, :r], -1) + np.eye(r)
    # C~ : solve X U11 = Cr column by column (upper triangular, from the left column).
    X = np.zeros((m, r))
    for j in range(r):
        X[:, j] = (Cr[:, j] - X[:, :j] @ U11[:j, j]) / U11[j, j]
    # R~ : solve L11 Y = Rr row by row (unit lower triangular).
    Y = np.zeros((r, n))
    for i in range(r):
        Y[i] = Rr[i] - L11[i, :i] @ Y[:i]
    return BDLRResult(X, Y.T.copy(), I, J, Ir, Jr, np.diag(LU)[:r].copy())


def heldout_error(A, rows: range, cols: range, U, V, Hr, Hc, I=(), J=()) -> float:
    """Relative Frobenius error of the approximation A(rows, cols) ~ U V^T
    measured on held-out rows Hr (global indices in rows) and columns Hc (in
    cols): the squared residuals of those rows and columns over the squared
    entries of every row and column examined, the selected I, J and the held
    out ones (the block's magnitude as seen by the sample); 0 when nothing is
    held out."""
    num = den = 0.0
    for h in Hr:
        a = A[h, cols.start:cols.stop]
        r = a - U[h - rows.start] @ V.T
        num += float(r @ r)
    for h in Hc:
        a = A[rows.start:rows.stop, h]
        r = a - U @ V[h - cols.start]
        num += float(r @ r)
    for h in list(Hr) + list(I):
        a = A[h, cols.start:cols.stop]
        den += float(a @ a)
    for h in list(Hc) + list(J):
        a = A[rows.start:rows.stop, h]
        den += float(a @ a)
    return math.sqrt(num / den) if den > 0 and (Hr or Hc) else 0.0


def bdlr_adaptive(A, rowptr, colind, rows: range, cols: range, eps: float, depth0: int = 1,
                  rank_cap: int = 1 << 30, dtype=np.float64):
    """The adaptive pseudo-skeleton of Section 5.3: BDLR at depth d, then the
    relative Frobenius error on the rows and columns held out of it -- those at
    distance exactly d + 1 from the boundary -- relative to every row and
    column examined (heldout_error), and, while that error exceeds eps and
    such rows or columns exist, the same with depth d + 1.  Returns
    (the BDLRResult of the final depth, that depth, its held-out error)."""
    d = depth0
    while True:
        res = bdlr(A, rowptr, colind, rows, cols, eps, d, rank_cap, dtype)
        _, dr = boundary_distance(rowptr, colind, rows, cols, d + 1)
        _, dc = boundary_distance(rowptr, colind, cols, rows, d + 1)
        Hr = [rows.start + i for i in np.flatnonzero(dr == d + 1)]
        Hc = [cols.start + j for j in np.flatnonzero(dc == d + 1)]
        err = heldout_error(A, rows, cols, res.U, res.V, Hr, Hc, res.I, res.J)
        if err <= eps or (not Hr and not Hc):
            return res, d, err
        d += 1


def bdlr_diagnostics(A, rowptr, colind, rows: range, cols: range, eps: float, depth: int):
    """The data of the paper's Figs. 4-6 for one off-diagonal block: the
    magnitude of every pivot of the full-pivoting LU of A^ with the boundary
    distances of its row and column (Fig. 4), the singular values of the block
    (Fig. 5), and for every rank r the relative Frobenius error of the
    BDLR approximation truncated to r pivots next to that of the rank-r SVD
    (Fig. 6)."""
    B = A[rows.start:rows.stop, cols.start:cols.stop]
    I, dI = boundary_distance(rowptr, colind, rows, cols, depth)
    J, dJ = boundary_distance(rowptr, colind, cols, rows, depth)
    LU, prow, pcol, r = full_pivot_lu(A[np.ix_(I, J)], eps)
    piv = np.abs(np.diag(LU)[:r])
    row_d = [int(dI[I[p] - rows.start]) for p in prow[:r]]
    col_d = [int(dJ[J[p] - cols.start]) for p in pcol[:r]]
    sv = np.linalg.svd(B, compute_uv=False)
    nB = np.linalg.norm(B)
    bdlr_err, svd_err = [], []
    for k in range(1, r + 1):
        Ir = [I[p] for p in prow[:k]]
        Jr = [J[p] for p in pcol[:k]]
        C = A[rows.start:rows.stop][:, Jr]
        R = A[Ir][:, cols.start:cols.stop]
        approx = C @ np.linalg.solve(A[np.ix_(Ir, Jr)], R)
        bdlr_err.append(float(np.linalg.norm(B - approx) / nB))
        svd_err.append(float(math.sqrt(max(float(np.sum(sv[k:] ** 2)), 0.0)) / nB))
    return dict(pivots=piv, row_dist=row_d, col_dist=col_d, singular_values=sv,
                bdlr_err=np.array(bdlr_err), svd_err=np.array(svd_err))


# --------------------------------------------------------------------------- HODLR# --------------------------------------------------------------------------- HODLR
@dataclass
class Blocks:
    """Off-diagonal factors per internal node (l, i), children a=(l+1,2i), b=(l+1,2i+1):
    A(a,b) ~ Ua Vab^T and A(b,a) ~ Ub Vba^T (eq. HODLR2)."""
    Ua: np.ndarray
    Vab: np.ndarray
    Ub: np.ndarray
    Vba: np.ndarray
    info_ab: object = None
    info_ba: object = None


def build(A: np.ndarray, tree: Tree, method: str = "aca", tol: float = 1e-6,
          rank_cap: int = 1 << 30, graph=None, depth: int = -1, symmetric=False,
          dtype=np.float64):
    """Compress every off-diagonal block of every level with ACA or BDLR (Section 4.3,
    Factorize step 1).  `symmetric` only changes how a column is fetched (as the
    equal row), never a value.  BDLR depth: >= 0 fixed, -1 round(-log10 tol),
    -2 adaptive per block (bdlr_adaptive)."""
    blocks = {}
    for l in range(tree.L):
        for i in range(1 << l):
            a0, a1 = tree.range(l + 1, 2 * i)
            b0, b1 = tree.range(l + 1, 2 * i + 1)
            pair = []
            for (r0, r1, c0, c1) in ((a0, a1, b0, b1), (b0, b1, a0, a1)):
                if method == "aca":
                    res = aca(lambda k: A[r0 + k, c0:c1],
                              (lambda k: A[c0 + k, r0:r1]) if symmetric else
                              (lambda k: A[r0:r1, c0 + k]),
                              r1 - r0, c1 - c0, tol, rank_cap, dtype)
                elif method == "bdlr" and depth == -2:
                    # the adaptive depth of Section 5.3
                    res, _, _ = bdlr_adaptive(A, graph[0], graph[1], range(r0, r1), range(c0, c1), tol,
                                              1, rank_cap, dtype)
                elif method == "bdlr":
                    d = depth if depth >= 0 else int(round(-math.log10(tol)))
                    res = bdlr(A, graph[0], graph[1], range(r0, r1), range(c0, c1), tol, d,
                               rank_cap, dtype)
                else:
                    raise ValueError(method)
                pair.append(res)
            blocks[(l, i)] = Blocks(pair[0].U, pair[0].V, pair[1].U, pair[1].V, pair[0], pair[1])
    return blocks


def assemble(A: np.ndarray, tree: Tree, blocks) -> np.ndarray:
    """The dense HODLR matrix K~: exact leaf blocks, U V^T off the diagonal."""
    K = np.zeros_like(A)
    for i in range(1 << tree.L):
        s, e = tree.range(tree.L, i)
        K[s:e, s:e] = A[s:e, s:e]
    for (l, i), blk in blocks.items():
        a0, a1 = tree.range(l + 1, 2 * i)
        b0, b1 = tree.range(l + 1, 2 * i + 1)
        K[a0:a1, b0:b1] = blk.Ua @ blk.Vab.T
        K[b0:b1, a0:a1] = blk.Ub @ blk.Vba.T
    return K


@dataclass
class Factors:
    tree: Tree
    leaf_lu: dict            # i -> (LU, perm) of K_i^(L)
    d: dict                  # (l, i) -> d_i^(l) = (K_i^(l))^-1 U_i^(l), l >= 1
    S: dict                  # (l, i) -> S_i^(l) (dense, for inspection)
    S_lu: dict               # (l, i) -> (LU, perm)
    blocks: dict


def factor(A: np.ndarray, tree: Tree, blocks) -> Factors:
    """Recursive Woodbury factorisation (Section 4.3, Factorize).

    Z_1^(0) is the empty matrix; a child's right-hand side is
    [U_child | rows of Z_parent]; a leaf solves it with its LU; a parent forms
    S_i^(p) = [[I, V_{2i,2i-1}^T d_{2i-1}], [V_{2i-1,2i}^T d_{2i}, I]] and, for p >= 1,
    [d_i c_i] = (I - [[0, d_{2i-1}], [d_{2i}, 0]] S^-1 diag(V_{2i,2i-1}^T,
    V_{2i-1,2i}^T)) [c_{2i-1}; c_{2i}]."""
    F = Factors(tree, {}, {}, {}, {}, blocks)

    def rec(l, i, Z):
        s, e = tree.range(l, i)
        if l == tree.L:
            lu = lu_partial(A[s:e, s:e])
            F.leaf_lu[i] = lu
            return lu_solve(*lu, Z) if Z.shape[1] else np.zeros((e - s, 0))
        blk = blocks[(l, i)]
        a0, a1 = tree.range(l + 1, 2 * i)
        ra, rb = blk.Ua.shape[1], blk.Ub.shape[1]
        Za = np.concatenate([blk.Ua, Z[: a1 - a0]], axis=1)
        Zb = np.concatenate([blk.Ub, Z[a1 - a0:]], axis=1)
        Da = rec(l + 1, 2 * i, Za)
        Db = rec(l + 1, 2 * i + 1, Zb)
        da, ca = Da[:, :ra], Da[:, ra:]
        db, cb = Db[:, :rb], Db[:, rb:]
        F.d[(l + 1, 2 * i)] = da
        F.d[(l + 1, 2 * i + 1)] = db
        # S = [[I_rb, Vba^T da], [Vab^T db, I_ra]]; y1 = Vba^T x_a (size rb), y2 = Vab^T x_b.
        S = np.eye(rb + ra)
        S[:rb, rb:] = blk.Vba.T @ da
        S[rb:, :rb] = blk.Vab.T @ db
        F.S[(l, i)] = S
        F.S_lu[(l, i)] = lu_partial(S) if S.shape[0] else (S, np.zeros(0, dtype=int))
        if l == 0 or ca.shape[1] == 0:
            return np.concatenate([ca, cb], axis=0)
        w = np.concatenate([blk.Vba.T @ ca, blk.Vab.T @ cb], axis=0)
        y = lu_solve(*F.S_lu[(l, i)], w)
        y1, y2 = y[:rb], y[rb:]
        return np.concatenate([ca - da @ y2, cb - db @ y1], axis=0)

    rec(0, 0, np.zeros((tree.n, 0)))
    return F


def solve(F: Factors, B: np.ndarray) -> np.ndarray:
    """Recursive HODLR solve (Section 4.3, Solve): split the right-hand side down the
    tree, solve the leaves, then x_i^(p) = (I - [[0,d_{2i-1}],[d_{2i},0]] S^-1
    diag(V_{2i,2i-1}^T, V_{2i-1,2i}^T)) [x_{2i-1}; x_{2i}] upward."""
    tree = F.tree
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    Z = B[:, None] if vec else B

    def rec(l, i, z):
        if l == tree.L:
            return lu_solve(*F.leaf_lu[i], z)
        blk = F.blocks[(l, i)]
        a0, a1 = tree.range(l + 1, 2 * i)
        xa = rec(l + 1, 2 * i, z[: a1 - a0])
        xb = rec(l + 1, 2 * i + 1, z[a1 - a0:])
        rb = blk.Ub.shape[1]
        w = np.concatenate([blk.Vba.T @ xa, blk.Vab.T @ xb], axis=0)
        if w.shape[0] == 0:
            return np.concatenate([xa, xb], axis=0)
        y = lu_solve(*F.S_lu[(l, i)], w)
        y1, y2 = y[:rb], y[rb:]
        return np.concatenate([xa - F.d[(l + 1, 2 * i)] @ y2,
                               xb - F.d[(l + 1, 2 * i + 1)] @ y1], axis=0)

    X = rec(0, 0, Z)
    return X[:, 0] if vec else X


# --------------------------------------------------------------------------- GMRES
@dataclass
class GMRESResult:
    x: np.ndarray
    iters: int
    est_relres: float
    true_relres: float
    converged: bool
    history: list


def gmres(A: np.ndarray, b: np.ndarray, prec=None, tol: float = 1e-12,
          max_iter: int = 1000, restart: int = 0) -> GMRESResult:
    """GMRES (Section 3) with right preconditioning M^-1 = `prec` (identity if None).

    Arnoldi with modified Gram-Schmidt on A M^-1, Givens rotations on the
    Hessenberg columns, stop when the estimated residual |g_{j+1}| <= tol ||b||;
    then x = x0 + M^-1 (V_j y) and the true residual ||b - A x|| / ||b|| is checked,
    restarting from x when it misses tol (also every `restart` steps if > 0).
    M^-1 (V_j y) is formed as Z_j y with the stored z_i = M^-1 v_i (the flexible
    form), equal to it in exact arithmetic for a fixed linear preconditioner."""
    P = prec if prec is not None else (lambda v: v)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(n)
    hist = []
    if bnorm == 0.0:
        return GMRESResult(x, 0, 0.0, 0.0, True, hist)
    total = 0
    m = restart if restart > 0 else max_iter
    est = 1.0
    while True:
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm or total >= max_iter:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j = 0
        while j < m and total < max_iter:
            Z.append(P(V[j]))
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            hnext = float(np.linalg.norm(w))
            H[j + 1, j] = hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = math.hypot(H[j, j], H[j + 1, j])
            if rho == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            est = abs(g[j + 1]) / bnorm
            hist.append(est)
            breakdown = H[j, j] == 0.0
            j += 1
            if est <= tol or breakdown:
                break
            V.append(w / hnext)
        # y = H(1:j,1:j)^-1 g(1:j), back substitution
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j] @ y[i + 1:j]) / H[i, i]
        x = x + np.stack(Z[:j], axis=1) @ y
        if est > tol and total >= max_iter:
            break
    true = float(np.linalg.norm(b - A @ x)) / bnorm
    return GMRESResult(x, total, est, true, true <= tol, hist)


# --------------------------------------------------------------------------- diagnostics
def precond_error(A: np.ndarray, prec, Omega: np.ndarray) -> float:
    """||(I - P^-1 A) Omega||_F / ||Omega||_F for a given probe block Omega."""
    E = Omega - prec(A @ Omega)
    return float(np.linalg.norm(E) / np.linalg.norm(Omega))


def precond_error_2norm(A: np.ndarray, prec) -> float:
    """The exact ||I - P^-1 A||_2: P^-1 applied to every column of A, then the
    largest singular value (dense SVD; for n up to a few thousand)."""
    E = np.eye(A.shape[0]) - prec(A)
    return float(np.linalg.svd(E, compute_uv=False)[0])


def dense_floor(A: np.ndarray, b: np.ndarray) -> float:
    """||b - A x_LU|| / ||b|| for the FP64 dense partial-pivoting LU solution."""
    x = dense_lu_solve(A, b)
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


def hodlr_precond(A, tree, method="aca", tol=1e-6, rank_cap=1 << 30, graph=None,
                  depth=-1, symmetric=False, dtype=np.float64):
    """Convenience: build + factor, returning (blocks, factors, apply function)."""
    blocks = build(A, tree, method, tol, rank_cap, graph, depth, symmetric, dtype)
    F = factor(A, tree, blocks)
    return blocks, F, (lambda v: solve(F, v))
