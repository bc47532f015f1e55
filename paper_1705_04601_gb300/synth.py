"""Seeded synthetic H^2 matrices shaped like the paper's workloads.

This module builds the *input* of the sparsification: an H^2 matrix given by
its parameters (cluster tree, nested cluster bases, transfer matrices,
coupling matrices and the close matrix, Definitions 4.1-4.9 of §4.1).  The
paper takes the H^2 matrix as given (§4.1) and builds it with an external
library; here it is built from Chebyshev interpolation on a quadtree/octree
and then recompressed to a tolerance.  Nothing in this module performs any
step of the sparsification, factorization or solve.  Both the CPU oracle and
the CUDA path consume what it produces.

Conventions (shared input format, consumed by both sides):

* The cluster tree is *level-uniform*: every leaf sits at depth ``D``.  A
  geometric leaf at a shallower depth is pushed down by a chain of virtual
  single-child clusters that keep the same cell and the same point range
  (their transfer matrices are identities up to the recompression).
* Clusters are numbered depth by depth; inside a depth, in the order of their
  parents, and inside a parent in Morton order of the child cells.  Children
  of a cluster therefore have consecutive numbers, and the points of the tree
  are ordered so that every cluster owns a contiguous index range.
* Admissibility is ``dist >= max diam`` evaluated exactly in integer units of
  the finest cell (per-axis gap between the cells).
* All dense blocks are stored column-major and packed in one flat float64
  array with an int64 offset per block.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import Callable, Optional

import numpy as np

SEED_BASE = 170504601

# --------------------------------------------------------------------------
# point sets
# --------------------------------------------------------------------------


def points_uniform(n: int, dim: int, rng: np.random.Generator) -> np.ndarray:
    return rng.random((n, dim))


def points_sphere_fibonacci(n: int, rng: np.random.Generator, jitter: float = 1e-3) -> np.ndarray:
    """Fibonacci lattice on the unit sphere plus uniform jitter (not re-projected)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    p = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return p + jitter * rng.uniform(-1.0, 1.0, size=p.shape)


def points_ellipse(n: int, rng: np.random.Generator) -> np.ndarray:
    """Points on a random ellipse curve centred at (0.5, 0.5), full axes in [0.2, 1]."""
    a = 0.5 * rng.uniform(0.2, 1.0)
    b = 0.5 * rng.uniform(0.2, 1.0)
    rot = rng.uniform(0.0, math.pi)
    th = rng.uniform(0.0, 2.0 * math.pi, size=n)
    x = a * np.cos(th)
    y = b * np.sin(th)
    c, s = math.cos(rot), math.sin(rot)
    return np.stack([0.5 + c * x - s * y, 0.5 + s * x + c * y], axis=1)


# --------------------------------------------------------------------------
# kernels
# --------------------------------------------------------------------------


def _pairdist(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    d = np.subtract.outer(x[:, 0], y[:, 0])
    r2 = d * d
    for k in range(1, x.shape[1]):
        d = np.subtract.outer(x[:, k], y[:, k])
        r2 += d * d
    return np.sqrt(r2)


def kernel_log(x, y):
    r = _pairdist(x, y)
    with np.errstate(divide="ignore"):
        return -np.log(r)


def kernel_inv(x, y):
    r = _pairdist(x, y)
    with np.errstate(divide="ignore"):
        return 1.0 / r


def kernel_yukawa(x, y):
    r = _pairdist(x, y)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.exp(-r) / r


def _pool():
    import concurrent.futures as cf
    return cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1))


def _sandwich_pairs(Lm, M, Rm, pairs, transpose_left):
    """[Lm[t] @ M[i] @ Rm[s].T] (or Lm[t].T @ M[i] @ Rm[s] with
    transpose_left) for pairs i = (t, s), batched by block shape."""
    out = [None] * len(pairs)
    groups = {}
    for i, (t, s) in enumerate(pairs):
        groups.setdefault((Lm[t].shape, M[i].shape, Rm[s].shape), []).append(i)
    for idx in groups.values():
        L = np.stack([Lm[pairs[i][0]] for i in idx])
        X = np.stack([M[i] for i in idx])
        Rr = np.stack([Rm[pairs[i][1]] for i in idx])
        if transpose_left:
            Y = np.matmul(np.matmul(L.transpose(0, 2, 1), X), Rr)
        else:
            Y = np.matmul(np.matmul(L, X), Rr.transpose(0, 2, 1))
        for z, i in enumerate(idx):
            out[i] = Y[z]
    return out


def _blocks_by_row(kf, rows_pts, cols_pts, pairs):
    """Kernel blocks K(rows_pts[t], cols_pts[s]) for a list of (t, s) pairs
    sorted by t: one kernel evaluation per row t over all its columns (the
    values are those of evaluating each block alone), split back per pair."""
    out = [None] * len(pairs)
    i = 0
    while i < len(pairs):
        t = int(pairs[i][0])
        j = i
        while j < len(pairs) and int(pairs[j][0]) == t:
            j += 1
        cols = [cols_pts(int(pairs[z][1])) for z in range(i, j)]
        K = kf(rows_pts(t), np.concatenate(cols, axis=0))
        o = 0
        for z, c in zip(range(i, j), cols):
            out[z] = K[:, o:o + c.shape[0]]
            o += c.shape[0]
        i = j
    return out


def kernel_gauss(x, y):
    """exp(-|x-y|^2); with 2 on the diagonal this is the SPD matrix of Example 5.2."""
    d = x[:, None, :] - y[None, :, :]
    return np.exp(-np.einsum("ijk,ijk->ij", d, d))


def kernel_log_skew(x, y):
    """A non-symmetric variant used to exercise separate row/column bases."""
    return kernel_log(x, y) + 0.1 * (x[:, None, 0] - y[None, :, 0])


def kernel_ifmm(d: float):
    """The matrix of the preconditioning example of §5.5: |x-y|/d for
    0 < |x-y| < d, d/|x-y| beyond (1 on the diagonal, from default_diag).
    Its condition number grows with d."""
    def k(x, y):
        r = _pairdist(x, y)
        with np.errstate(divide="ignore"):
            return np.where(r < d, r / d, d / r)
    return k


KERNELS = {"log": kernel_log, "inv": kernel_inv, "yukawa": kernel_yukawa, "log_skew": kernel_log_skew,
           "gauss": kernel_gauss, "ifmm_d1e-3": kernel_ifmm(1e-3), "ifmm_d1e-2": kernel_ifmm(1e-2)}


def default_diag(kernel: str, n: int, dim: int) -> float:
    if kernel in ("log", "log_skew"):
        return -math.log(0.5 / math.sqrt(n))
    if kernel == "inv":
        return 2.0 * math.sqrt(n)
    if kernel == "yukawa":
        return 2.0 * n ** (1.0 / 3.0)
    if kernel == "gauss":
        return 3.0
    if kernel.startswith("ifmm_"):
        return 1.0
    raise ValueError(kernel)


# --------------------------------------------------------------------------
# the H^2 container
# --------------------------------------------------------------------------


@dataclasses.dataclass
class H2Matrix:
    n: int
    dim: int
    depth: int                     # leaf depth D (level-uniform)
    level_ptr: np.ndarray          # int32[D+2]: clusters of depth d are [level_ptr[d], level_ptr[d+1])
    parent: np.ndarray             # int32[ncl], -1 for the root
    begin: np.ndarray              # int64[ncl]
    size: np.ndarray               # int64[ncl]
    rank: np.ndarray               # int32[ncl]  row rank k_t
    leaf_basis: np.ndarray         # float64 packed, n_t x k_t column-major per leaf
    leaf_basis_off: np.ndarray     # int64[nleaf]
    transfer: np.ndarray           # float64 packed, k_c x k_parent per non-root cluster
    transfer_off: np.ndarray       # int64[ncl] (root entry unused, 0)
    far_ptr: np.ndarray            # int64[ncl+1], CSR by row cluster (same depth)
    far_col: np.ndarray            # int32[nfar]
    coupling: np.ndarray           # float64 packed, k_t x kc_s per far pair
    coupling_off: np.ndarray       # int64[nfar]
    near_ptr: np.ndarray           # int64[nleaf+1], CSR by leaf (leaf index = cluster - level_ptr[D])
    near_col: np.ndarray           # int32[nnear], cluster ids of depth D
    near_block: np.ndarray         # float64 packed, n_t x n_s per near pair
    near_off: np.ndarray           # int64[nnear]
    col_rank: Optional[np.ndarray] = None          # None => column bases equal row bases
    col_leaf_basis: Optional[np.ndarray] = None
    col_leaf_basis_off: Optional[np.ndarray] = None
    col_transfer: Optional[np.ndarray] = None
    col_transfer_off: Optional[np.ndarray] = None
    points: Optional[np.ndarray] = None            # points in tree order (diagnostics only)
    cell_lo: Optional[np.ndarray] = None           # int64[ncl, dim] cell in finest units
    cell_hi: Optional[np.ndarray] = None
    kernel: str = ""
    diag: float = 0.0

    @property
    def ncl(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nleaf(self) -> int:
        return int(self.level_ptr[self.depth + 1] - self.level_ptr[self.depth])

    @property
    def symmetric_bases(self) -> bool:
        return self.col_rank is None

    def crank(self) -> np.ndarray:
        return self.rank if self.col_rank is None else self.col_rank

    # convenient block views -------------------------------------------------
    def leaf_R(self, t: int, col: bool = False) -> np.ndarray:
        lf = t - int(self.level_ptr[self.depth])
        if col and self.col_rank is not None:
            k, arr, off = int(self.col_rank[t]), self.col_leaf_basis, self.col_leaf_basis_off
        else:
            k, arr, off = int(self.rank[t]), self.leaf_basis, self.leaf_basis_off
        nt = int(self.size[t])
        o = int(off[lf])
        return arr[o:o + nt * k].reshape(k, nt).T

    def T(self, c: int, col: bool = False) -> np.ndarray:
        p = int(self.parent[c])
        if col and self.col_rank is not None:
            rk, arr, off = self.col_rank, self.col_transfer, self.col_transfer_off
        else:
            rk, arr, off = self.rank, self.transfer, self.transfer_off
        kc, kp = int(rk[c]), int(rk[p])
        o = int(off[c])
        return arr[o:o + kc * kp].reshape(kp, kc).T

    def D(self, idx: int, t: int, s: int) -> np.ndarray:
        kt, ks = int(self.rank[t]), int(self.crank()[s])
        o = int(self.coupling_off[idx])
        return self.coupling[o:o + kt * ks].reshape(ks, kt).T

    def C(self, idx: int, t: int, s: int) -> np.ndarray:
        nt, ns = int(self.size[t]), int(self.size[s])
        o = int(self.near_off[idx])
        return self.near_block[o:o + nt * ns].reshape(ns, nt).T

    def stats(self) -> dict:
        return {
            "n": self.n, "depth": self.depth, "clusters": self.ncl, "leaves": self.nleaf,
            "near_pairs": int(self.near_col.shape[0]), "far_pairs": int(self.far_col.shape[0]),
            "max_rank": int(self.rank.max()), "mean_leaf_size": float(self.n / self.nleaf),
            "near_bytes": int(self.near_block.nbytes),
        }


def _pack_colmajor(blocks) -> tuple[np.ndarray, np.ndarray]:
    offs = np.zeros(len(blocks), dtype=np.int64)
    tot = 0
    for i, b in enumerate(blocks):
        offs[i] = tot
        tot += b.size
    out = np.empty(tot, dtype=np.float64)
    for i, b in enumerate(blocks):
        if b.size:
            out[offs[i]:offs[i] + b.size] = np.asarray(b, dtype=np.float64).T.reshape(-1)
    return out, offs


# --------------------------------------------------------------------------
# tree
# --------------------------------------------------------------------------


@dataclasses.dataclass
class _Tree:
    depth: int
    level_ptr: np.ndarray
    parent: np.ndarray
    begin: np.ndarray
    size: np.ndarray
    cell_lo: np.ndarray     # int64[ncl, dim] in finest units
    cell_hi: np.ndarray
    box_lo: np.ndarray      # float cell corners (for Chebyshev nodes)
    box_hi: np.ndarray
    perm: np.ndarray        # tree position -> input index


def build_tree(points: np.ndarray, leaf_size: int, lo: np.ndarray, hi: np.ndarray, max_depth: int = 24) -> _Tree:
    """Quadtree/octree with empty children dropped, made level-uniform."""
    n, dim = points.shape
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = (points - lo) / (hi - lo)
    u = np.clip(u, 0.0, np.nextafter(1.0, 0.0))
    # real clusters: (point index array, depth, integer coords at that depth)
    real = [[(np.arange(n), np.zeros(dim, dtype=np.int64))]]
    real_children = [[]]   # per depth, per cluster: list of child indices at depth+1 (None if leaf)
    d = 0
    while True:
        nxt = []
        kids_here = []
        for idx, coord in real[d]:
            if idx.size <= leaf_size or d >= max_depth:
                kids_here.append(None)
                continue
            sub = np.floor(u[idx] * (1 << (d + 1))).astype(np.int64)
            bits = sub - 2 * coord[None, :]
            cid = np.zeros(idx.size, dtype=np.int64)
            for a in range(dim):
                cid |= bits[:, a] << a
            order = np.argsort(cid, kind="stable")
            cid_sorted = cid[order]
            mine = []
            for c in range(1 << dim):
                lo_i = np.searchsorted(cid_sorted, c, "left")
                hi_i = np.searchsorted(cid_sorted, c, "right")
                if hi_i > lo_i:
                    cc = 2 * coord + np.array([(c >> a) & 1 for a in range(dim)], dtype=np.int64)
                    mine.append(len(nxt))
                    nxt.append((idx[order[lo_i:hi_i]], cc))
            kids_here.append(mine)
        real_children[d] = kids_here
        if not nxt:
            break
        real.append(nxt)
        real_children.append([])
        d += 1
    D = len(real) - 1
    # level-uniform numbering: each entry refers to (real depth, real index)
    lvl = [[(0, 0)]]
    par = [[-1]]
    for dd in range(1, D + 1):
        cur, cpar = [], []
        base_prev = sum(len(x) for x in lvl[:dd - 1])
        for j, (rd, ri) in enumerate(lvl[dd - 1]):
            kids = real_children[rd][ri] if rd == dd - 1 else None
            if kids is None:      # a (possibly virtual) leaf: push down
                cur.append((rd, ri))
                cpar.append(base_prev + j)
            else:
                for k in kids:
                    cur.append((dd, k))
                    cpar.append(base_prev + j)
        lvl.append(cur)
        par.append(cpar)
    level_ptr = np.zeros(D + 2, dtype=np.int32)
    for dd in range(D + 1):
        level_ptr[dd + 1] = level_ptr[dd] + len(lvl[dd])
    ncl = int(level_ptr[-1])
    parent = np.array([p for pl in par for p in pl], dtype=np.int32)
    # point order from the leaves
    leaf_pts = [real[rd][ri][0] for (rd, ri) in lvl[D]]
    perm = np.concatenate(leaf_pts).astype(np.int64)
    size = np.zeros(ncl, dtype=np.int64)
    begin = np.zeros(ncl, dtype=np.int64)
    off = 0
    for j, p in enumerate(leaf_pts):
        size[level_ptr[D] + j] = p.size
        begin[level_ptr[D] + j] = off
        off += p.size
    for dd in range(D - 1, -1, -1):
        for j in range(level_ptr[dd], level_ptr[dd + 1]):
            pass
        kids_lo = level_ptr[dd + 1]
        for c in range(level_ptr[dd + 1], level_ptr[dd + 2]):
            p = parent[c]
            if size[p] == 0:
                begin[p] = begin[c]
            size[p] += size[c]
        del kids_lo
    cell_lo = np.zeros((ncl, dim), dtype=np.int64)
    cell_hi = np.zeros((ncl, dim), dtype=np.int64)
    box_lo = np.zeros((ncl, dim))
    box_hi = np.zeros((ncl, dim))
    w = hi - lo
    for dd in range(D + 1):
        for j, (rd, ri) in enumerate(lvl[dd]):
            cl = level_ptr[dd] + j
            coord = real[rd][ri][1]
            sh = D - rd
            cell_lo[cl] = coord << sh
            cell_hi[cl] = (coord + 1) << sh
            box_lo[cl] = lo + w * coord / (1 << rd)
            box_hi[cl] = lo + w * (coord + 1) / (1 << rd)
    return _Tree(D, level_ptr, parent, begin, size, cell_lo, cell_hi, box_lo, box_hi, perm)


def admissible(lo_t, hi_t, lo_s, hi_s) -> np.ndarray:
    """dist >= max diam on integer cells (vectorised over rows)."""
    gap = np.maximum(0, np.maximum(lo_s - hi_t, lo_t - hi_s))
    dist2 = np.sum(gap * gap, axis=-1)
    dt = np.sum((hi_t - lo_t) ** 2, axis=-1)
    ds = np.sum((hi_s - lo_s) ** 2, axis=-1)
    return dist2 >= np.maximum(dt, ds)


def block_lists(tree: _Tree):
    """Dual traversal from (root, root): far pairs per depth and leaf near pairs."""
    D = tree.depth
    ncl = tree.parent.shape[0]
    child_start = np.full(ncl, -1, dtype=np.int64)
    child_cnt = np.zeros(ncl, dtype=np.int64)
    for c in range(ncl - 1, 0, -1):
        p = tree.parent[c]
        child_start[p] = c
        child_cnt[p] += 1
    near = np.array([[0, 0]], dtype=np.int64)
    far_all = []
    for d in range(1, D + 1):
        p, q = near[:, 0], near[:, 1]
        nc_p, nc_q = child_cnt[p], child_cnt[q]
        tot = nc_p * nc_q
        rep = np.repeat(np.arange(p.size), tot)
        local = np.arange(tot.sum()) - np.repeat(np.cumsum(tot) - tot, tot)
        c = child_start[p][rep] + local // nc_q[rep]
        e = child_start[q][rep] + local % nc_q[rep]
        adm = admissible(tree.cell_lo[c], tree.cell_hi[c], tree.cell_lo[e], tree.cell_hi[e])
        far_all.append(np.stack([c[adm], e[adm]], axis=1))
        near = np.stack([c[~adm], e[~adm]], axis=1)
    far = np.concatenate(far_all) if far_all else np.zeros((0, 2), dtype=np.int64)
    # sort: far by (row, col); near by (row, col)
    far = far[np.lexsort((far[:, 1], far[:, 0]))]
    near = near[np.lexsort((near[:, 1], near[:, 0]))]
    return near, far


# --------------------------------------------------------------------------
# Chebyshev interpolation H^2
# --------------------------------------------------------------------------


def _cheb_nodes_1d(a: float, b: float, p: int) -> np.ndarray:
    c, h = 0.5 * (a + b), 0.5 * (b - a)
    return c + h * np.cos((2.0 * np.arange(p) + 1.0) * math.pi / (2.0 * p))


def _lagrange_1d(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[i, a] = prod_{b != a} (x_i - nodes_b) / (nodes_a - nodes_b)."""
    p = nodes.size
    out = np.ones((x.size, p))
    for a in range(p):
        for b in range(p):
            if b != a:
                out[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return out


def _tensor_nodes(lo: np.ndarray, hi: np.ndarray, p: int) -> np.ndarray:
    dim = lo.size
    ax = [_cheb_nodes_1d(lo[a], hi[a], p) for a in range(dim)]
    grids = np.meshgrid(*ax, indexing="ij")
    # index alpha = a0 + p*a1 + p^2*a2 (axis 0 fastest)
    return np.stack([g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grids], axis=1)


def _tensor_lagrange(lo: np.ndarray, hi: np.ndarray, p: int, x: np.ndarray) -> np.ndarray:
    dim = lo.size
    vals = [_lagrange_1d(_cheb_nodes_1d(lo[a], hi[a], p), x[:, a]) for a in range(dim)]
    out = vals[0]
    for a in range(1, dim):
        out = (vals[a][:, :, None] * out[:, None, :]).reshape(x.shape[0], -1)
    return out


def _orthogonalise(tree, kids, Rleaf, T):
    """Bottom-up QR of the nested basis: R_t = Q_t Z_t with orthonormal Q_t.

    Returns the orthonormal leaf bases, the transfers of the orthonormal basis
    and the coefficient maps Z_t (so that old basis = new basis @ Z_t)."""
    D = tree.depth
    lp = tree.level_ptr
    ncl = tree.parent.shape[0]
    Z = [None] * ncl
    Qleaf = {}
    Tq = [None] * ncl
    for t in range(lp[D], lp[D + 1]):
        q, z = np.linalg.qr(Rleaf[t])
        Qleaf[t], Z[t] = q, z
    for d in range(D - 1, -1, -1):
        for t in range(lp[d], lp[d + 1]):
            ks = kids[t]
            W = np.vstack([Z[c] @ T[c] for c in ks])
            q, z = np.linalg.qr(W)
            Z[t] = z
            r0 = 0
            for c in ks:
                rc = Z[c].shape[0]
                Tq[c] = q[r0:r0 + rc, :]
                r0 += rc
    return Qleaf, Tq, Z


def _truncation(tree, Tq, Z, far_pairs, Dorth, tol, col: bool):
    """Weight each orthonormal cluster basis by the far field it carries (its
    own couplings plus the parent's weight pushed down through the transfer,
    top-down) and keep the left singular vectors above ``tol`` times the
    largest singular value of that weight."""
    D = tree.depth
    lp = tree.level_ptr
    ncl = tree.parent.shape[0]
    rows_of = [[] for _ in range(ncl)]
    for i, (t, s) in enumerate(far_pairs):
        if col:
            rows_of[s].append(Dorth[i].T)
        else:
            rows_of[t].append(Dorth[i])
    G = [None] * ncl
    B = [None] * ncl
    R = [0] * ncl

    def one(t):
        p = tree.parent[t]
        kt = Z[t].shape[0]
        blocks = list(rows_of[t])
        if p >= 0 and G[p].shape[1] > 0:
            blocks.append(Tq[t] @ G[p])
        if not blocks or kt == 0:
            G[t] = np.zeros((kt, 0))
            B[t] = np.zeros((kt, 0))
            return
        Y = np.hstack(blocks)
        G[t] = np.linalg.qr(Y.T, mode="r").T
        u, sig, _ = np.linalg.svd(G[t], full_matrices=True)
        if sig.size == 0 or sig[0] == 0.0:
            G[t] = np.zeros((kt, 0))
            B[t] = np.zeros((kt, 0))
            return
        B[t] = u
        R[t] = int(np.sum(sig > tol * sig[0]))

    # the clusters of one depth are independent (each needs only its parent's G)
    with _pool() as ex:
        for d in range(D + 1):
            list(ex.map(one, range(lp[d], lp[d + 1])))
    return B, R


def build_h2(points: np.ndarray, kernel: str, leaf_size: int, p: int = 4, tol: Optional[float] = 1e-8,
             diag: Optional[float] = None, lo=None, hi=None, keep_points: bool = True) -> H2Matrix:
    n, dim = points.shape
    if lo is None:
        lo = np.zeros(dim)
    if hi is None:
        hi = np.ones(dim)
    kf: Callable = KERNELS[kernel]
    if diag is None:
        diag = default_diag(kernel, n, dim)
    tree = build_tree(points, leaf_size, np.asarray(lo, float), np.asarray(hi, float))
    D = tree.depth
    lp = tree.level_ptr
    ncl = tree.parent.shape[0]
    pts = points[tree.perm]
    kids = [[] for _ in range(ncl)]
    for c in range(1, ncl):
        kids[tree.parent[c]].append(c)
    near, far = block_lists(tree)
    # Chebyshev parameters
    nodes = [_tensor_nodes(tree.box_lo[t], tree.box_hi[t], p) for t in range(ncl)]
    Rleaf = {}
    for t in range(lp[D], lp[D + 1]):
        b, s = int(tree.begin[t]), int(tree.size[t])
        Rleaf[t] = _tensor_lagrange(tree.box_lo[t], tree.box_hi[t], p, pts[b:b + s])
    T = [None] * ncl
    for c in range(1, ncl):
        par = tree.parent[c]
        T[c] = _tensor_lagrange(tree.box_lo[par], tree.box_hi[par], p, nodes[c])
    Dfar = _blocks_by_row(kf, lambda t: nodes[t], lambda s: nodes[s], far)
    symmetric = kernel != "log_skew"
    col = None
    if tol is not None:
        Ql_r, Tq_r, Z_r = _orthogonalise(tree, kids, Rleaf, T)
        Ql_c, Tq_c, Z_c = (Ql_r, Tq_r, Z_r) if symmetric else _orthogonalise(tree, kids, Rleaf, T)
        Dorth = _sandwich_pairs(Z_r, Dfar, Z_c, far, transpose_left=False)
        U_r, r_r = _truncation(tree, Tq_r, Z_r, far, Dorth, tol, col=False)
        if symmetric:
            U_c, r_c = U_r, r_r
        else:
            U_c, r_c = _truncation(tree, Tq_c, Z_c, far, Dorth, tol, col=True)
        # one rank per cluster for rows and columns, so S has square diagonal blocks
        rk = [max(a, b) for a, b in zip(r_r, r_c)]
        B_r = [U_r[t][:, :rk[t]] for t in range(ncl)]
        B_c = B_r if symmetric else [U_c[t][:, :rk[t]] for t in range(ncl)]
        Dfar = _sandwich_pairs(B_r, Dorth, B_c, far, transpose_left=True)
        Rleaf = {t: Ql_r[t] @ B_r[t] for t in Ql_r}
        T = [None] + [B_r[c].T @ Tq_r[c] @ B_r[tree.parent[c]] for c in range(1, ncl)]
        rank = np.array([B_r[t].shape[1] for t in range(ncl)], dtype=np.int32)
        if not symmetric:
            col = ({t: Ql_c[t] @ B_c[t] for t in Ql_c},
                   [None] + [B_c[c].T @ Tq_c[c] @ B_c[tree.parent[c]] for c in range(1, ncl)],
                   np.array([B_c[t].shape[1] for t in range(ncl)], dtype=np.int32))
    else:
        rank = np.full(ncl, p ** dim, dtype=np.int32)
        if not symmetric:
            col = (dict(Rleaf), list(T), rank.copy())
    # pack
    leaf_ids = list(range(lp[D], lp[D + 1]))
    leaf_basis, leaf_basis_off = _pack_colmajor([Rleaf[t] for t in leaf_ids])
    tr_blocks = [np.zeros((0, 0))] + [T[c] for c in range(1, ncl)]
    transfer, transfer_off = _pack_colmajor(tr_blocks)
    far_ptr = np.zeros(ncl + 1, dtype=np.int64)
    np.add.at(far_ptr, far[:, 0] + 1, 1)
    far_ptr = np.cumsum(far_ptr)
    coupling, coupling_off = _pack_colmajor(Dfar)
    nleaf = len(leaf_ids)
    near_ptr = np.zeros(nleaf + 1, dtype=np.int64)
    np.add.at(near_ptr, near[:, 0] - lp[D] + 1, 1)
    near_ptr = np.cumsum(near_ptr)
    def leaf_pts(t):
        return pts[int(tree.begin[t]):int(tree.begin[t]) + int(tree.size[t])]

    blocks = _blocks_by_row(kf, leaf_pts, leaf_pts, near)
    for z, (t, s) in enumerate(near):
        if t == s:
            blocks[z] = np.array(blocks[z])
            np.fill_diagonal(blocks[z], diag)
    near_block, near_off = _pack_colmajor(blocks)
    h = H2Matrix(
        n=n, dim=dim, depth=D, level_ptr=lp.astype(np.int32), parent=tree.parent.astype(np.int32),
        begin=tree.begin.astype(np.int64), size=tree.size.astype(np.int64), rank=rank,
        leaf_basis=leaf_basis, leaf_basis_off=leaf_basis_off, transfer=transfer, transfer_off=transfer_off,
        far_ptr=far_ptr.astype(np.int64), far_col=far[:, 1].astype(np.int32), coupling=coupling,
        coupling_off=coupling_off, near_ptr=near_ptr.astype(np.int64), near_col=near[:, 1].astype(np.int32),
        near_block=near_block, near_off=near_off, points=pts if keep_points else None,
        cell_lo=tree.cell_lo, cell_hi=tree.cell_hi, kernel=kernel, diag=float(diag),
    )
    if col is not None:
        leaf_c, T_c, crank = col
        h.col_rank = crank
        h.col_leaf_basis, h.col_leaf_basis_off = _pack_colmajor([leaf_c[t] for t in leaf_ids])
        h.col_transfer, h.col_transfer_off = _pack_colmajor([np.zeros((0, 0))] + [T_c[c] for c in range(1, ncl)])
    return h


def tree_arrays(points: np.ndarray, leaf_size: int, lo=None, hi=None) -> tuple[dict, np.ndarray]:
    """The cluster tree and the close / admissible lists build_h2 uses, as the
    host arrays of a GPU construction (boxes, CSR lists), and the points in
    tree order."""
    n, dim = points.shape
    lo = np.zeros(dim) if lo is None else np.asarray(lo, float)
    hi = np.ones(dim) if hi is None else np.asarray(hi, float)
    tree = build_tree(points, leaf_size, lo, hi)
    D = tree.depth
    lp = tree.level_ptr
    ncl = tree.parent.shape[0]
    near, far = block_lists(tree)
    far_ptr = np.zeros(ncl + 1, dtype=np.int64)
    np.add.at(far_ptr, far[:, 0] + 1, 1)
    nleaf = int(lp[D + 1] - lp[D])
    near_ptr = np.zeros(nleaf + 1, dtype=np.int64)
    np.add.at(near_ptr, near[:, 0] - lp[D] + 1, 1)
    t = dict(depth=D, level_ptr=lp.astype(np.int32), parent=tree.parent.astype(np.int32),
             begin=tree.begin.astype(np.int64), size=tree.size.astype(np.int64),
             box_lo=np.ascontiguousarray(tree.box_lo, np.float64), box_hi=np.ascontiguousarray(tree.box_hi, np.float64),
             far_ptr=np.cumsum(far_ptr).astype(np.int64), far_col=far[:, 1].astype(np.int32),
             near_ptr=np.cumsum(near_ptr).astype(np.int64), near_col=near[:, 1].astype(np.int32))
    return t, np.ascontiguousarray(points[tree.perm])


def workload_points(name: str, n: Optional[int] = None, seed: Optional[int] = None):
    """(points, lo, hi, config) of a named single-system workload: the same
    seeded points make_workload builds its H^2 matrix from."""
    cfg = dict(WORKLOADS[name])
    if n is not None:
        cfg["n"] = n
    rng = np.random.default_rng(SEED_BASE + cfg["index"] if seed is None else seed)
    if cfg.get("points", "uniform") == "sphere":
        pts = points_sphere_fibonacci(cfg["n"], rng)
        lo, hi = np.full(3, -1.01), np.full(3, 1.01)
    else:
        pts = points_uniform(cfg["n"], cfg["dim"], rng)
        lo, hi = np.zeros(cfg["dim"]), np.ones(cfg["dim"])
    return pts, lo, hi, cfg


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    # 2D -log r, N=4096, leaf<=64, Chebyshev 4x4 recompressed to 1e-8, one RHS
    "log2d_n4096": dict(kernel="log", n=4096, dim=2, leaf=64, tol=1e-8, nrhs=1, index=1),
    # 2D -log r, N=65536, leaf<=64, tol 1e-6, 16 RHS
    "log2d_n65536": dict(kernel="log", n=65536, dim=2, leaf=64, tol=1e-6, nrhs=16, index=2),
    # 3D 1/r on a jittered Fibonacci sphere, N=262144, leaf<=128, Chebyshev 4^3 to 1e-6
    "inv3d_sphere_n262144": dict(kernel="inv", n=262144, dim=3, leaf=128, tol=1e-6, nrhs=1, index=3,
                                 points="sphere"),
    # 3D Yukawa, N=1048576 uniform in the cube, leaf<=128, tol 1e-4
    "yukawa3d_n1048576": dict(kernel="yukawa", n=1048576, dim=3, leaf=128, tol=1e-4, nrhs=1, index=5),
    # batched form: 256 independent 2D -log r systems on random ellipses, N_k ~ U[2048, 32768], leaf<=64,
    # tol 1e-6, one forest (n = the systems' total; "n" overrides the count of systems)
    "batched_ellipse_256": dict(kernel="log", n=256, dim=2, leaf=64, tol=1e-6, nrhs=1, index=4,
                                batched=(2048, 32768), points="ellipses"),
}


def make_workload(name: str, n: Optional[int] = None, seed: Optional[int] = None, tol: Optional[float] = "cfg",
                  leaf: Optional[int] = None, kernel: Optional[str] = None):
    """Return (H2Matrix, rhs) for a named workload; ``n``/``leaf``/``tol`` override for small cases."""
    cfg = dict(WORKLOADS[name])
    if n is not None:
        cfg["n"] = n
    if "batched" in cfg:
        # n counts systems; the size range may be narrowed through leaf/tol-free overrides of the caller
        lo, hi = cfg["batched"]
        _, forest, b = make_batched(cfg["n"], lo, hi, seed=SEED_BASE + cfg["index"] if seed is None else seed,
                                    leaf=cfg["leaf"] if leaf is None else leaf,
                                    tol=cfg["tol"] if tol == "cfg" else tol, nrhs=cfg["nrhs"])
        return forest, b
    if leaf is not None:
        cfg["leaf"] = leaf
    if tol != "cfg":
        cfg["tol"] = tol
    if kernel is not None:
        cfg["kernel"] = kernel
    rng = np.random.default_rng(SEED_BASE + cfg["index"] if seed is None else seed)
    kind = cfg.get("points", "uniform")
    if kind == "sphere":
        pts = points_sphere_fibonacci(cfg["n"], rng)
        lo, hi = np.full(3, -1.01), np.full(3, 1.01)
    else:
        pts = points_uniform(cfg["n"], cfg["dim"], rng)
        lo, hi = np.zeros(cfg["dim"]), np.ones(cfg["dim"])
    h = build_h2(pts, cfg["kernel"], cfg["leaf"], tol=cfg["tol"], lo=lo, hi=hi)
    b = rng.standard_normal((cfg["n"], cfg["nrhs"]))
    return h, b


def make_small(n: int = 512, kernel: str = "log", leaf: int = 32, tol: Optional[float] = 1e-8, seed: int = 7,
               dim: int = 2, nrhs: int = 1):
    rng = np.random.default_rng(SEED_BASE + seed)
    pts = points_uniform(n, dim, rng)
    h = build_h2(pts, kernel, leaf, tol=tol)
    b = rng.standard_normal((n, nrhs))
    return h, b


# --------------------------------------------------------------------------
# batched form: several independent H^2 matrices as one forest
# --------------------------------------------------------------------------


def _push_down(h: H2Matrix, D: int) -> dict:
    """Per-depth cluster lists of h extended to leaf depth D: every leaf gets a
    chain of virtual single-child clusters with an identity transfer."""
    lp = h.level_ptr
    d0 = h.depth
    kids = [[] for _ in range(h.ncl)]
    for c in range(1, h.ncl):
        kids[int(h.parent[c])].append(c)
    # node = (orig cluster id, virtual level offset)
    levels = [[(t, 0) for t in range(lp[d], lp[d + 1])] for d in range(d0 + 1)]
    for dd in range(d0 + 1, D + 1):
        levels.append([(t, v + 1) for (t, v) in levels[dd - 1]])
    return {"levels": levels}


def make_forest(systems: list) -> H2Matrix:
    """Concatenate independent H^2 matrices into one forest descriptor.

    Depth 0 holds one root per system; every tree is pushed down to the
    deepest leaf depth by virtual single-child chains (identity transfers,
    same points); clusters are renumbered depth by depth, system by system,
    so the children of a cluster stay consecutive and every system owns a
    contiguous range of rows.  No pair of clusters of different systems is
    close or admissible, so A is block diagonal with the given blocks."""
    D = max(h.depth for h in systems)
    sym = all(h.col_rank is None for h in systems)
    if not sym and any(h.col_rank is None for h in systems):
        raise ValueError("mixed symmetric / non-symmetric systems")
    ext = [_push_down(h, D) for h in systems]
    # new ids
    newid = []     # per system: dict (depth, t, v) -> new id
    level_ptr = [0]
    order = []     # per depth: list of (sys, t, v)
    for d in range(D + 1):
        lst = []
        for k, h in enumerate(systems):
            lst.extend((k, t, v) for (t, v) in ext[k]["levels"][d])
        order.append(lst)
        level_ptr.append(level_ptr[-1] + len(lst))
    ids = [dict() for _ in systems]
    for d in range(D + 1):
        for j, (k, t, v) in enumerate(order[d]):
            ids[k][(d, t, v)] = level_ptr[d] + j
    ncl = level_ptr[-1]
    parent = np.full(ncl, -1, dtype=np.int32)
    begin = np.zeros(ncl, dtype=np.int64)
    size = np.zeros(ncl, dtype=np.int64)
    rank = np.zeros(ncl, dtype=np.int32)
    crank = np.zeros(ncl, dtype=np.int32)
    orig = [None] * ncl
    row0 = np.cumsum([0] + [h.n for h in systems])
    for d in range(D + 1):
        for (k, t, v) in order[d]:
            h = systems[k]
            nid = ids[k][(d, t, v)]
            orig[nid] = (k, t, v, d)
            begin[nid] = row0[k] + h.begin[t]
            size[nid] = h.size[t]
            rank[nid] = h.rank[t]
            crank[nid] = h.crank()[t]
            if d > 0:
                if v == 0:
                    parent[nid] = ids[k][(d - 1, int(h.parent[t]), 0)]
                else:
                    parent[nid] = ids[k][(d - 1, t, v - 1)]
    leaf0 = level_ptr[D]
    # bases and transfers
    lb, lbc, tr, trc = [], [], [np.zeros((0, 0))], [np.zeros((0, 0))]
    for nid in range(leaf0, ncl):
        k, t, v, d = orig[nid]
        lb.append(systems[k].leaf_R(t))
        lbc.append(systems[k].leaf_R(t, col=True))
    for nid in range(1, ncl):
        k, t, v, d = orig[nid]
        if parent[nid] < 0:
            tr.append(np.zeros((rank[nid], 0)))
            trc.append(np.zeros((crank[nid], 0)))
        elif v == 0:
            tr.append(systems[k].T(t))
            trc.append(systems[k].T(t, col=True))
        else:
            tr.append(np.eye(rank[nid]))
            trc.append(np.eye(crank[nid]))
    leaf_basis, leaf_basis_off = _pack_colmajor(lb)
    transfer, transfer_off = _pack_colmajor(tr)
    # far pairs keep their depth; close pairs move to the new leaf depth
    far_rows = [[] for _ in range(ncl)]
    for k, h in enumerate(systems):
        for t in range(h.ncl):
            d = int(np.searchsorted(h.level_ptr, t, side="right") - 1)
            for i in range(int(h.far_ptr[t]), int(h.far_ptr[t + 1])):
                s = int(h.far_col[i])
                far_rows[ids[k][(d, t, 0)]].append((ids[k][(d, s, 0)], h.D(i, t, s)))
    far_ptr = np.zeros(ncl + 1, dtype=np.int64)
    far_col, Dl = [], []
    for r in range(ncl):
        far_rows[r].sort(key=lambda x: x[0])
        far_ptr[r + 1] = far_ptr[r] + len(far_rows[r])
        for (s, blk) in far_rows[r]:
            far_col.append(s)
            Dl.append(blk)
    coupling, coupling_off = _pack_colmajor(Dl)
    near_rows = [[] for _ in range(ncl - leaf0)]
    for k, h in enumerate(systems):
        hl0 = int(h.level_ptr[h.depth])
        off = D - h.depth
        for lf in range(h.nleaf):
            t = hl0 + lf
            for i in range(int(h.near_ptr[lf]), int(h.near_ptr[lf + 1])):
                s = int(h.near_col[i])
                near_rows[ids[k][(D, t, off)] - leaf0].append((ids[k][(D, s, off)], h.C(i, t, s)))
    near_ptr = np.zeros(ncl - leaf0 + 1, dtype=np.int64)
    near_col, Cl = [], []
    for r in range(ncl - leaf0):
        near_rows[r].sort(key=lambda x: x[0])
        near_ptr[r + 1] = near_ptr[r] + len(near_rows[r])
        for (s, blk) in near_rows[r]:
            near_col.append(s)
            Cl.append(blk)
    near_block, near_off = _pack_colmajor(Cl)
    out = H2Matrix(
        n=int(row0[-1]), dim=systems[0].dim, depth=D, level_ptr=np.array(level_ptr, dtype=np.int32), parent=parent,
        begin=begin, size=size, rank=rank, leaf_basis=leaf_basis, leaf_basis_off=leaf_basis_off,
        transfer=transfer, transfer_off=transfer_off, far_ptr=far_ptr, far_col=np.array(far_col, dtype=np.int32),
        coupling=coupling, coupling_off=coupling_off, near_ptr=near_ptr, near_col=np.array(near_col, dtype=np.int32),
        near_block=near_block, near_off=near_off, kernel=systems[0].kernel, diag=float("nan"),
    )
    if not sym:
        out.col_rank = crank
        out.col_leaf_basis, out.col_leaf_basis_off = _pack_colmajor(lbc)
        out.col_transfer, out.col_transfer_off = _pack_colmajor(trc)
    out.points = np.concatenate([h.points for h in systems]) if all(h.points is not None for h in systems) else None
    return out


def make_batched(nsys: int, n_lo: int, n_hi: int, seed: int = SEED_BASE + 4, leaf: int = 64, tol: float = 1e-6,
                 nrhs: int = 1):
    """Independent 2D -log r systems on random ellipses (the batched workload).

    N_k ~ U[n_lo, n_hi]; ellipse centre (0.5, 0.5), full axes ~ U[0.2, 1],
    random rotation; diagonal -log(0.5/sqrt(N_k)).  Returns (systems, forest, b)."""
    rng = np.random.default_rng(seed)
    sizes = [int(rng.integers(n_lo, n_hi + 1)) for _ in range(nsys)]
    jobs = [(nk, seed + 1000 * (k + 1), leaf, tol) for k, nk in enumerate(sizes)]
    workers = min(len(jobs), os.cpu_count() or 1, int(os.environ.get("H2SP_GEN_WORKERS", "16")))
    if workers > 1 and sum(sizes) > 200000:
        # the systems are independent: build them in worker processes (spawned,
        # so that no CUDA state is inherited), each from its own seed as below
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            systems = list(ex.map(_ellipse_system, jobs, chunksize=max(1, len(jobs) // (4 * workers))))
    else:
        systems = [_ellipse_system(j) for j in jobs]
    forest = make_forest(systems)
    b = rng.standard_normal((forest.n, nrhs))
    return systems, forest, b


def _ellipse_system(job):
    nk, sd, leaf, tol = job
    pts = points_ellipse(nk, np.random.default_rng(sd))
    return build_h2(pts, "log", leaf, tol=tol)
