"""Seeded synthetic frontal matrices: the inputs of the solver, and nothing of its method.

The paper applies its solver to the dense frontal matrices of a multifrontal
elimination of 3D finite-element stiffness matrices (Section 6, Table 3).  Those
matrices are not public, so the workloads here are their closest synthetic
stand-in with the same structure: the exact Schur complement of a 3D
variable-coefficient 7-point diffusion operator onto the separator plane in the
middle of a box, i.e. a dense SPD front whose rows are the vertices of a 2D grid.

Everything in this module is input preparation, shared by the CPU oracle, the
CUDA path, the tests and the benchmark:

* a counter-based normal generator (SplitMix64 finaliser + Box-Muller), so that
  every coefficient and right-hand side is a pure function of (seed, index);
* the coefficient fields (lognormal and checkerboard);
* the exact FP64 block-tridiagonal elimination of the box onto its middle
  plane (across the planes, or across the lines of thin slabs);
* the recursive-bisection ordering of the plane (every HODLR node is then a
  rectangle of the plane and a contiguous index range), the plane's 5-point
  adjacency graph in that order (the sparse graph the BDLR row/column selection
  of Section 5.3 walks), and the leaf boundaries of the resulting tree.

No HODLR compression, factorisation, preconditioning or Krylov arithmetic is here.
The elimination runs in PyTorch FP64 on whatever device it is given (CPU for the
small cases, a GPU to make the large fronts quickly); the solver only ever sees the
finished matrix.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "splitmix64", "uniform01", "normal", "coefficient_lognormal",
    "coefficient_checkerboard", "face_coefficients", "plane_front",
    "bisection_order", "plane_graph", "Front", "make_front", "rhs",
    "WORKLOADS", "octree_boxes", "elastic_operator", "elastic_front", "make_elastic_front",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) applied to counters x.

    z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
    z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31   (all mod 2^64).
    """
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counter: np.ndarray) -> np.ndarray:
    """U(0,1) doubles from the counter-based stream (seed, counter).

    The 64-bit counter word is seed * 2^40 + counter; the top 53 bits of its
    SplitMix64 image give a double in [0, 1)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        word = np.uint64(seed) * np.uint64(1 << 40) + c
    bits = splitmix64(word) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, index: np.ndarray) -> np.ndarray:
    """N(0,1) doubles: Box-Muller on the uniforms at counters 2g and 2g+1."""
    g = np.asarray(index, dtype=np.uint64)
    u1 = uniform01(seed, np.uint64(2) * g)
    u2 = uniform01(seed, np.uint64(2) * g + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- fields
def coefficient_lognormal(nx: int, ny: int, nz: int, sigma: float, seed: int = 0,
                          origin=(0, 0, 0), full_shape=None) -> np.ndarray:
    """Node coefficients a = exp(sigma * z), z ~ N(0,1) from the global node index.

    The field is defined on a (possibly larger) grid `full_shape` with x-fastest
    global index g = i + X*(j + Y*k); the returned array is the box of size
    nx*ny*nz starting at `origin`, indexed [k, j, i]."""
    X, Y, _ = full_shape if full_shape is not None else (nx, ny, nz)
    i = np.arange(nx) + origin[0]
    j = np.arange(ny) + origin[1]
    k = np.arange(nz) + origin[2]
    g = i[None, None, :] + X * (j[None, :, None] + Y * k[:, None, None])
    return np.exp(sigma * normal(seed, g.astype(np.uint64)))


def coefficient_checkerboard(nx: int, ny: int, nz: int, cell: int = 8,
                             contrast: float = 1e6) -> np.ndarray:
    """a = 1 where (i//cell + j//cell + k//cell) is even, `contrast` where odd."""
    i = np.arange(nx) // cell
    j = np.arange(ny) // cell
    k = np.arange(nz) // cell
    par = (i[None, None, :] + j[None, :, None] + k[:, None, None]) % 2
    return np.where(par == 1, contrast, 1.0)


def face_coefficients(a: np.ndarray):
    """Face coefficients of the 7-point finite-volume operator, h = 1.

    Interior faces take the harmonic mean 2ab/(a+b) of the two nodes; a face to
    the outside of the box (Dirichlet) takes the node's own coefficient.
    Returns (fx, fy, fz) of shapes (nz,ny,nx+1), (nz,ny+1,nx), (nz+1,ny,nx)."""
    nz, ny, nx = a.shape

    def faces(axis):
        lo = np.take(a, range(0, a.shape[axis] - 1), axis=axis)
        hi = np.take(a, range(1, a.shape[axis]), axis=axis)
        inner = 2.0 * lo * hi / (lo + hi)
        first = np.take(a, [0], axis=axis)
        last = np.take(a, [a.shape[axis] - 1], axis=axis)
        return np.concatenate([first, inner, last], axis=axis)

    return faces(2), faces(1), faces(0)


# --------------------------------------------------------------------------- front
def _plane_matrix(fx, fy, fz, k, dev):
    """T_k: the 2D block of plane k of the box operator (x-fastest order); its
    diagonal carries all six face coefficients of each node."""
    import torch
    f64 = torch.float64
    ny, nx = fx.shape[1], fx.shape[2] - 1
    n = nx * ny
    diag = (fx[k, :, :-1] + fx[k, :, 1:] + fy[k, :-1, :] + fy[k, 1:, :]
            + fz[k] + fz[k + 1]).reshape(-1)
    t = torch.diag(torch.as_tensor(diag, dtype=f64, device=dev))
    idx = np.arange(n).reshape(ny, nx)
    for r_, c_, v_ in ((idx[:, :-1], idx[:, 1:], fx[k, :, 1:-1]),      # x-neighbours
                       (idx[:-1, :], idx[1:, :], fy[k, 1:-1, :])):     # y-neighbours
        r = torch.as_tensor(r_.reshape(-1), device=dev)
        c = torch.as_tensor(c_.reshape(-1), device=dev)
        v = torch.as_tensor(v_.reshape(-1), dtype=f64, device=dev)
        t[r, c] = -v
        t[c, r] = -v
    return t


def _slab_inverse_planes(fx, fy, fz, planes, dev):
    """(A_slab^-1) on the last plane of `planes` (ordered away from the front):
    S_0 = T_first, S_{k+1} = T_{k+1} - C_k S_k^-1 C_k, result S_last^-1."""
    import torch
    f64 = torch.float64
    s = None
    for step, k in enumerate(planes):
        t = _plane_matrix(fx, fy, fz, k, dev)
        if s is not None:
            prev = planes[step - 1]
            c = torch.as_tensor(fz[max(prev, k)].reshape(-1), dtype=f64, device=dev)
            t -= c[:, None] * torch.cholesky_inverse(torch.linalg.cholesky(s)) * c[None, :]
        s = t
    return torch.cholesky_inverse(torch.linalg.cholesky(s))


def _slab_inverse_rows(fx, fy, fz, planes, adj, dev):
    """The same block, (A_slab^-1) on plane `adj`, by a block-tridiagonal
    elimination across the y-lines of the slab instead of across its planes.

    Block j holds the slab's nodes with y = j (local order q*nx + x, q the
    plane's position in sorted `planes`), nb = p*nx of them; neighbouring blocks
    couple through the diagonal y-face coefficients F_j.  With the block pivots
    Sigma_0 = B_0, Sigma_j = B_j - F_{j-1} Sigma_{j-1}^-1 F_{j-1}, the columns
    E of the identity on plane `adj` are solved for by
      forward   W_j = Sigma_j^-1 (E_j + F_{j-1} W_{j-1})
      backward  X_j = W_j + Sigma_j^-1 F_j X_{j+1}
    and the result is X restricted to the rows of plane `adj`.  Only the first
    nx*(j+1) columns of W_j are non-zero (E_j is non-zero in the columns of line
    j alone), which the forward sweep exploits.  About 3 ny nb^2 n flops against
    p n^3 for the plane recursion: the cheaper one for thin slabs."""
    import torch
    f64 = torch.float64
    planes = sorted(planes)
    p = len(planes)
    ny, nx = fx.shape[1], fx.shape[2] - 1
    n = nx * ny
    nb = p * nx
    zl = planes.index(adj)
    q = np.repeat(np.arange(p), nx)          # local plane of each block row
    x = np.tile(np.arange(nx), p)
    z = np.asarray(planes)[q]

    def block(j):
        d = (fx[z, j, x] + fx[z, j, x + 1] + fy[z, j, x] + fy[z, j + 1, x] + fz[z, j, x] + fz[z + 1, j, x])
        b = np.diag(d)
        r = np.nonzero(x < nx - 1)[0]                      # x-neighbours
        b[r, r + 1] = b[r + 1, r] = -fx[z[r], j, x[r] + 1]
        r = np.nonzero((q < p - 1))[0]                     # z-neighbours, consecutive planes only
        r = r[np.asarray(planes)[q[r] + 1] == z[r] + 1]
        b[r, r + nx] = b[r + nx, r] = -fz[z[r] + 1, j, x[r]]
        return torch.as_tensor(b, dtype=f64, device=dev)

    def couple(j):                                         # F_j between lines j and j+1
        return torch.as_tensor(fy[z, j + 1, x], dtype=f64, device=dev)

    sinv, W = [], []
    for j in range(ny):
        b = block(j)
        if j > 0:
            f = couple(j - 1)
            b -= f[:, None] * sinv[-1] * f[None, :]
        si = torch.cholesky_inverse(torch.linalg.cholesky(b))
        rhs = torch.zeros(nb, nx * (j + 1), dtype=f64, device=dev)
        if j > 0:
            rhs[:, :nx * j] = couple(j - 1)[:, None] * W[-1]
        rhs[zl * nx + np.arange(nx), nx * j + np.arange(nx)] += 1.0
        W.append(si @ rhs)
        sinv.append(si)
    G = torch.empty(n, n, dtype=f64, device=dev)
    X = None
    for j in range(ny - 1, -1, -1):
        Xj = torch.zeros(nb, n, dtype=f64, device=dev)
        Xj[:, :nx * (j + 1)] = W[j]
        if X is not None:
            Xj += sinv[j] @ (couple(j)[:, None] * X)
        W[j] = None
        X = Xj
        G[j * nx:(j + 1) * nx] = X[zl * nx:(zl + 1) * nx]
    return G


def _transpose_faces(fx, fy, fz):
    """Faces of the box with x and y exchanged (so that lines run along the
    other axis)."""
    return (np.ascontiguousarray(fy.transpose(0, 2, 1)), np.ascontiguousarray(fx.transpose(0, 2, 1)),
            np.ascontiguousarray(fz.transpose(0, 2, 1)))


def plane_front(a: np.ndarray, n_below: int, device="cpu", method="auto") -> np.ndarray:
    """Exact FP64 Schur complement of the box operator onto plane k = n_below.

    The front is T_m - C_below G_below C_below - C_above G_above C_above, where
    T_m is the 2D block of the middle plane, C the diagonal z-face coefficients
    to its neighbouring planes and G the block, on the neighbouring plane, of the
    inverse of the operator restricted to the slab of planes on that side.
    G comes from one of two exact eliminations of the slab (same values up to
    rounding):
      "planes": one plane at a time, S_0 = T_0, S_{k+1} = T_{k+1} - C_k S_k^-1 C_k,
                G = S_last^-1 (about p n^3 flops for p planes);
      "rows":   block-tridiagonal across the lines of the slab along its longer
                side (about 3 ny nb^2 n flops, nb = p * shorter side);
      "auto":   "rows" when it is at least four times cheaper, else "planes".
    Returned in the plane's natural x-fastest order, symmetrised exactly."""
    import torch

    nz, ny, nx = a.shape
    n = nx * ny
    m = n_below
    fx, fy, fz = face_coefficients(a)
    dev = torch.device(device)
    f64 = torch.float64

    def side(planes, adj):
        p = len(planes)
        lines, short = max(nx, ny), min(nx, ny)
        rows_cost = 3.0 * lines * (p * short) ** 2 * n
        use_rows = method == "rows" or (method == "auto" and 4.0 * rows_cost < p * float(n) ** 3)
        if not use_rows:
            return _slab_inverse_planes(fx, fy, fz, planes, dev)
        if ny >= nx:
            return _slab_inverse_rows(fx, fy, fz, planes, adj, dev)
        # lines along x: exchange the axes, eliminate, and map back to x-fastest order
        G = _slab_inverse_rows(*_transpose_faces(fx, fy, fz), planes, adj, dev)
        t = torch.as_tensor(np.arange(n).reshape(nx, ny).T.reshape(-1), device=dev)   # natural -> exchanged
        return G.index_select(0, t).index_select(1, t)

    front = _plane_matrix(fx, fy, fz, m, dev)
    if m > 0:
        G = side(list(range(0, m)), m - 1)
        c = torch.as_tensor(fz[m].reshape(-1), dtype=f64, device=dev)
        front -= c[:, None] * G * c[None, :]
        del G
    if m < nz - 1:
        G = side(list(range(nz - 1, m, -1)), m + 1)
        c = torch.as_tensor(fz[m + 1].reshape(-1), dtype=f64, device=dev)
        front -= c[:, None] * G * c[None, :]
        del G
    front = 0.5 * (front + front.T)
    return front.cpu().numpy() if dev.type == "cpu" else front


# --------------------------------------------------------------------------- elasticity
def elastic_operator(mu: np.ndarray, nu: float = 0.3):
    """The 3-dof Navier-Cauchy operator -mu Lap u - (lambda + mu) grad div u on a
    box of nodes (nz, ny, nx) = mu.shape, h = 1, Dirichlet outside the box, as
    the sum of two positive semi-definite forms (so the matrix is SPD):
      * sum over the 6 faces of every node of mu_f |u_p - u_q|^2 / 2 per
        component (node coefficients mu, harmonic mean on interior faces, the
        node's own on boundary faces), the vector Laplacian of the
        finite-volume scalar operator;
      * sum over the (nx+1)(ny+1)(nz+1) cells between nodes of (lambda +
        mu)_c (div_c u)^2, div_c the one-point divergence of the trilinear
        cell: du_a/dx_a = 1/4 sum over the cell's 4 edges along a of the
        difference of u_a across the edge (outside nodes are zero);
    lambda = 2 mu nu / (1 - 2 nu), cell values the mean of the cell's nodes.
    Dofs are ordered 3 * (x + nx (y + ny z)) + component.  Returns a
    scipy.sparse CSR matrix."""
    import scipy.sparse as sp
    nz, ny, nx = mu.shape
    N = nx * ny * nz
    fx, fy, fz = face_coefficients(mu)
    rows, cols, vals = [], [], []

    def node(i, j, k):
        return i + nx * (j + ny * k)

    # vector Laplacian (same scalar stencil on each component)
    diag = np.zeros(N)
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    pidx = node(ii, jj, kk)
    diag += (fx[kk, jj, ii] + fx[kk, jj, ii + 1] + fy[kk, jj, ii] + fy[kk, jj + 1, ii]
             + fz[kk, jj, ii] + fz[kk + 1, jj, ii])
    for (di, dj, dk, f) in ((1, 0, 0, fx[kk, jj, ii + 1]), (0, 1, 0, fy[kk, jj + 1, ii]), (0, 0, 1, fz[kk + 1, jj, ii])):
        ok = (ii + di < nx) & (jj + dj < ny) & (kk + dk < nz)
        a, b = pidx[ok], node(ii[ok] + di, jj[ok] + dj, kk[ok] + dk)
        for c in range(3):
            rows += [3 * a + c, 3 * b + c]
            cols += [3 * b + c, 3 * a + c]
            vals += [-f[ok], -f[ok]]
    for c in range(3):
        rows.append(3 * pidx + c)
        cols.append(3 * pidx + c)
        vals.append(diag)
    lap = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * N, 3 * N))
    # grad-div: B^T W B over the cells
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    pad = np.pad(lam + mu, 1, mode="edge")   # cell value: mean of the 8 (padded) nodes around it
    cw = sum(pad[dk:dk + nz + 1, dj:dj + ny + 1, di:di + nx + 1]
             for dk in (0, 1) for dj in (0, 1) for di in (0, 1)) / 8.0
    ci, cj, ck = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    cidx = ci + (nx + 1) * (cj + (ny + 1) * ck)
    brow, bcol, bval = [], [], []
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                xi, yj, zk = ci - 1 + di, cj - 1 + dj, ck - 1 + dk   # corner node of the cell
                ok = (xi >= 0) & (xi < nx) & (yj >= 0) & (yj < ny) & (zk >= 0) & (zk < nz)
                nd = node(xi[ok], yj[ok], zk[ok])
                for c, d in ((0, di), (1, dj), (2, dk)):
                    brow.append(cidx[ok])
                    bcol.append(3 * nd + c)
                    bval.append(np.full(ok.sum(), 0.25 if d == 1 else -0.25))
    ncell = (nx + 1) * (ny + 1) * (nz + 1)
    B = sp.csr_matrix((np.concatenate(bval), (np.concatenate(brow), np.concatenate(bcol))), shape=(ncell, 3 * N))
    W = sp.diags(cw[ck, cj, ci])
    return (lap + B.T @ W @ B).tocsr()


def elastic_front(mu: np.ndarray, n_below: int, nu: float = 0.3, device="cpu") -> np.ndarray:
    """Exact FP64 Schur complement of the elasticity operator onto plane
    n_below (3 dofs per node, x-fastest node order): the planes on each side
    are eliminated one at a time, S_0 = T_0, S_{k+1} = T_{k+1} - C_k^T S_k^-1
    C_k, with C_k the (sparse) coupling of planes k and k+1; symmetrised
    exactly."""
    import torch
    nz, ny, nx = mu.shape
    K = elastic_operator(mu, nu)
    m = 3 * nx * ny
    dev = torch.device(device)

    def blk(a, b):
        return torch.as_tensor(K[a * m:(a + 1) * m, b * m:(b + 1) * m].toarray(), dtype=torch.float64, device=dev)

    def side(planes):
        s = None
        for step, k in enumerate(planes):
            t = blk(k, k)
            if s is not None:
                C = blk(planes[step - 1], k)
                t -= C.T @ torch.cholesky_solve(C, torch.linalg.cholesky(s))
            s = t
        return s

    front = blk(n_below, n_below)
    if n_below > 0:
        s = side(list(range(0, n_below)))
        C = blk(n_below - 1, n_below)
        front -= C.T @ torch.cholesky_solve(C, torch.linalg.cholesky(s))
    if n_below < nz - 1:
        s = side(list(range(nz - 1, n_below, -1)))
        C = blk(n_below + 1, n_below)
        front -= C.T @ torch.cholesky_solve(C, torch.linalg.cholesky(s))
    front = 0.5 * (front + front.T)
    return front.cpu().numpy() if dev.type == "cpu" else front


def make_elastic_front(nx, ny, below, above, sigma=0.5, nu=0.3, leaf_nodes=64, seed=0, device="cpu"):
    """An elasticity front on an nx x ny x (below + 1 + above) box: shear modulus
    mu = exp(sigma z), z ~ N(0,1) per node (counter stream `seed`), Poisson
    ratio nu, in the recursive-bisection order of the plane with the 3 dofs of
    a node kept together (leaves of at most `leaf_nodes` nodes).  The graph is
    the plane's 5-point adjacency between nodes, every dof of a node joined to
    the other dofs of that node and to every dof of the neighbouring nodes."""
    nz = below + 1 + above
    mu = coefficient_lognormal(nx, ny, nz, sigma, seed)
    A_nat = elastic_front(mu, below, nu, device=device)
    perm_n, bounds_n, L, _ = bisection_order(nx, ny, leaf_nodes)
    perm = (3 * perm_n[:, None] + np.arange(3)[None, :]).reshape(-1)
    if isinstance(A_nat, np.ndarray):
        A = np.ascontiguousarray(A_nat[np.ix_(perm, perm)])
    else:
        import torch
        p = torch.as_tensor(perm, device=A_nat.device)
        A = A_nat.index_select(0, p).index_select(1, p).contiguous()
    rp_n, ci_n = plane_graph(nx, ny, perm_n)
    rows = []
    for v in range(len(perm_n)):
        nb = [int(w) for w in ci_n[rp_n[v]:rp_n[v + 1]]] + [v]
        for c in range(3):
            rows.append(sorted(3 * w + d for w in nb for d in range(3) if (w, d) != (v, c)))
    rowptr = np.zeros(len(rows) + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.asarray([c for r in rows for c in r], dtype=np.int32)
    return Front(A, 3 * nx * ny, nx, ny, perm, 3 * bounds_n, L, rowptr, colind,
                 dict(nz=nz, below=below, above=above, field="elastic", sigma=sigma, nu=nu, seed=seed))


# --------------------------------------------------------------------------- ordering
def bisection_order(nx: int, ny: int, leaf: int):
    """Recursive bisection of the nx-by-ny plane rectangle.

    Each node is split across its longer side (x on ties) into a lower half of
    floor(len/2) lines and an upper half; all nodes of a level are split together
    until every node holds at most `leaf` vertices, giving a complete binary tree
    of depth L.  Inside a leaf the order is lexicographic (x fastest).

    Returns (perm, bounds, L, rects): perm[new] = natural index x + nx*y,
    bounds = the 2^L + 1 leaf boundary offsets, rects = per-level rectangles."""
    rects = [[(0, nx, 0, ny)]]
    while max((x1 - x0) * (y1 - y0) for x0, x1, y0, y1 in rects[-1]) > leaf:
        nxt = []
        for x0, x1, y0, y1 in rects[-1]:
            if (x1 - x0) >= (y1 - y0):
                xm = x0 + (x1 - x0) // 2
                nxt += [(x0, xm, y0, y1), (xm, x1, y0, y1)]
            else:
                ym = y0 + (y1 - y0) // 2
                nxt += [(x0, x1, y0, ym), (x0, x1, ym, y1)]
        rects.append(nxt)
    perm = []
    bounds = [0]
    for x0, x1, y0, y1 in rects[-1]:
        for y in range(y0, y1):
            for x in range(x0, x1):
                perm.append(x + nx * y)
        bounds.append(len(perm))
    return np.asarray(perm, dtype=np.int64), np.asarray(bounds, dtype=np.int64), len(rects) - 1, rects


def plane_graph(nx: int, ny: int, perm: np.ndarray):
    """5-point adjacency of the plane (the sparsity of the front's own block of the
    3D operator) in the permuted order, as CSR (rowptr, colind) int32, columns
    sorted ascending within each row."""
    n = nx * ny
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    rows = [[] for _ in range(n)]
    for new, old in enumerate(perm):
        x, y = old % nx, old // nx
        for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            xx, yy = x + dx, y + dy
            if 0 <= xx < nx and 0 <= yy < ny:
                rows[new].append(int(inv[xx + nx * yy]))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.asarray([c for r in rows for c in sorted(r)], dtype=np.int32)
    return rowptr, colind


# --------------------------------------------------------------------------- workloads
@dataclass
class Front:
    """A dense front in tree order plus everything a solver needs about it."""
    A: object                 # n x n FP64 (numpy, or torch tensor when built on a GPU)
    n: int
    nx: int
    ny: int
    perm: np.ndarray          # tree order -> natural plane index
    bounds: np.ndarray        # leaf boundaries (2^L + 1)
    levels: int
    rowptr: np.ndarray        # plane graph, CSR, tree order
    colind: np.ndarray
    meta: dict = field(default_factory=dict)


def _finish(A_nat, nx, ny, leaf, meta):
    perm, bounds, L, _ = bisection_order(nx, ny, leaf)
    if isinstance(A_nat, np.ndarray):
        A = np.ascontiguousarray(A_nat[np.ix_(perm, perm)])
    else:
        import torch
        p = torch.as_tensor(perm, device=A_nat.device)
        A = A_nat.index_select(0, p).index_select(1, p).contiguous()
    rowptr, colind = plane_graph(nx, ny, perm)
    return Front(A, nx * ny, nx, ny, perm, bounds, L, rowptr, colind, meta)


# The five synthetic workloads: grid (nx, ny, planes below, planes above), field, leaf.
WORKLOADS = {
    "plane576":  dict(nx=24, ny=24, below=8, above=8, field="lognormal", sigma=0.5, leaf=64),
    "plane4096": dict(nx=64, ny=64, below=32, above=32, field="lognormal", sigma=0.5, leaf=128),
    "checker16384": dict(nx=128, ny=128, below=16, above=16, field="checkerboard", leaf=256),
    "plane32768": dict(nx=128, ny=256, below=4, above=4, field="lognormal", sigma=0.5, leaf=256),
}


def default_cache_dir() -> str:
    """Directory for generated fronts: $HODLR_FRONT_CACHE or <tmp>/hodlr_fronts."""
    import tempfile
    return os.environ.get("HODLR_FRONT_CACHE", os.path.join(tempfile.gettempdir(), "hodlr_fronts"))


def make_front(nx, ny, below, above, field="lognormal", sigma=0.5, leaf=64, seed=0,
               device="cpu", cell=8, contrast=1e6, cache=False):
    """Build one plane front on an nx x ny x (below+1+above) box, in tree order.

    With cache=True the natural-order front is stored in default_cache_dir() and
    reloaded on the next call with the same parameters (the elimination is the
    slow part; the ordering and graph are recomputed)."""
    path = None
    if cache:
        key = f"front_{nx}x{ny}_{below}_{above}_{field}_{sigma}_{seed}_{cell}_{contrast}.npy"
        d = default_cache_dir()
        os.makedirs(d, exist_ok=True)
        path = os.path.join(d, key)
        if os.path.exists(path):
            A_nat = np.load(path)
            if device != "cpu":
                import torch
                A_nat = torch.as_tensor(A_nat, device=device)
            return _finish(A_nat, nx, ny, leaf, dict(nz=below + 1 + above, below=below, above=above,
                                                     field=field, sigma=sigma, seed=seed))
    nz = below + 1 + above
    if field == "lognormal":
        a = coefficient_lognormal(nx, ny, nz, sigma, seed)
    elif field == "checkerboard":
        a = coefficient_checkerboard(nx, ny, nz, cell, contrast)
    elif field == "constant":
        a = np.ones((nz, ny, nx))
    else:
        raise ValueError(field)
    A_nat = plane_front(a, below, device=device)
    if path is not None:
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, A_nat if isinstance(A_nat, np.ndarray) else A_nat.cpu().numpy())
        os.replace(tmp, path)
    return _finish(A_nat, nx, ny, leaf, dict(nz=nz, below=below, above=above,
                                             field=field, sigma=sigma, seed=seed))


def octree_boxes(side: int = 64, min_side: int = 8):
    """Octree reading of a nested-dissection tree of a side^3 grid: every box of
    side s = side, side/2, ..., min_side contributes the front of its middle z-plane
    (s/2 planes below it, s/2 - 1 above).  Returns [(s, (x0, y0, z0))] root first:
    1 + 8 + 64 + 512 = 585 boxes for 64 -> 8."""
    out = []
    s = side
    while s >= min_side:
        m = side // s
        for kz in range(m):
            for jy in range(m):
                for ix in range(m):
                    out.append((s, (ix * s, jy * s, kz * s)))
        s //= 2
    return out


def make_octree_front(s, origin, leaf, sigma=1.0, seed=0, side=64, device="cpu"):
    """Front of one octree box of side s inside a side^3 lognormal field."""
    a = coefficient_lognormal(s, s, s, sigma, seed, origin=origin, full_shape=(side, side, side))
    A_nat = plane_front(a, s // 2, device=device)
    return _finish(A_nat, s, s, leaf, dict(box=s, origin=origin, sigma=sigma, seed=seed))


def rhs(n: int, s: int, seed: int = 1) -> np.ndarray:
    """Right-hand sides B (n x s, column-major values) with B[i, c] ~ N(0,1) at
    counter i + n*c of stream `seed`; returned as a C-contiguous n x s array."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    c = np.arange(s, dtype=np.uint64)[None, :]
    return np.ascontiguousarray(normal(seed, i + np.uint64(n) * c))
