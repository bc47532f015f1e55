"""Block LU of the sparse S and the solve S y = U^T b, x = V y (§1, Eq. sp0).

The paper factors S with a sparse direct package (§5.3-5.4) and says nothing
about the order of elimination or about pivoting.  The readings taken:

* Ordering -- nested dissection along the cluster tree.  Every S node
  v = (l, t) below the top gets the *closure* cluster
      closure(v) = LCA of t and every level-l close neighbour e of t with
                   e > t (cluster number),
  and every top node gets the root.  Two nodes whose closures lie in
  disjoint subtrees are never coupled in S (and never become coupled by
  fill), so the nodes are eliminated by closure depth, deepest first; the
  nodes that share a closure form one supernode; supernodes of one closure
  depth are independent.  Order key: (-depth(closure), closure, node id).
* Pivoting -- partial pivoting restricted to the rows of the supernode's own
  diagonal block (LAPACK getrf semantics: the first row of largest modulus).
* Symbolic factorization -- plain graph elimination on the node graph of S
  (made structurally symmetric): eliminating a supernode joins its remaining
  neighbours (its *boundary*) into a clique.

The numeric factorization is the right-looking block elimination written on
a dictionary of dense node-by-node blocks:
      F11 = P L11 U11          (dense LU of the supernode block, getrf)
      U12 = L11^-1 P^T F12,    L21 = F21 U11^-1
      M[w1, w2] -= L21[w1] U12[w2]   for all boundary pairs (w1, w2).
The dense LU of the pivot block is the LAPACK routine (scipy) used as one
step; everything else is written out.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .sparsify import Sparsified


def _depths(h) -> np.ndarray:
    dep = np.zeros(h.ncl, dtype=np.int64)
    for d in range(h.depth + 1):
        dep[h.level_ptr[d]:h.level_ptr[d + 1]] = d
    return dep


def lca(h, dep, a: int, b: int) -> int:
    while dep[a] > dep[b]:
        a = int(h.parent[a])
    while dep[b] > dep[a]:
        b = int(h.parent[b])
    while a != b:
        a, b = int(h.parent[a]), int(h.parent[b])
    return a


@dataclasses.dataclass
class Symbolic:
    closure: np.ndarray       # int64[nnodes]
    order: np.ndarray         # elimination order of the nodes
    sn_ptr: np.ndarray        # supernodes as ranges of ``order``
    sn_closure: np.ndarray    # closure cluster of each supernode
    sn_depth: np.ndarray      # depth of that closure
    boundary: list            # per supernode: node ids (ascending elimination position)
    flops: float              # (2/3)s^3 + 2 s^2 b + 2 s b^2 summed over supernodes (scalar sizes)


def node_graph(sp: Sparsified) -> list:
    nn = sp.sch.node_size.shape[0]
    adj = [set() for _ in range(nn)]
    for (i, j) in sp.blocks.keys():
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    return adj


def symbolic(h, sp: Sparsified) -> Symbolic:
    sch = sp.sch
    nn = sch.node_size.shape[0]
    dep = _depths(h)
    close = [dict() for _ in range(sch.lstop + 1)]
    for l in range(sch.lstop):
        for (t, e) in sch.near[l]:
            close[l].setdefault(int(t), []).append(int(e))
    clo = np.zeros(nn, dtype=np.int64)
    for v in range(nn):
        l, t = int(sch.node_level[v]), int(sch.node_cluster[v])
        if l == sch.lstop:
            clo[v] = 0
            continue
        c = t
        for e in close[l].get(t, []):
            if e > t:
                c = lca(h, dep, c, e)
        clo[v] = c
    order = np.array(sorted(range(nn), key=lambda v: (-dep[clo[v]], clo[v], v)), dtype=np.int64)
    sn_ptr = [0]
    for i in range(1, nn):
        if clo[order[i]] != clo[order[i - 1]]:
            sn_ptr.append(i)
    sn_ptr.append(nn)
    sn_ptr = np.array(sn_ptr, dtype=np.int64)
    pos = np.empty(nn, dtype=np.int64)
    pos[order] = np.arange(nn)
    adj = node_graph(sp)
    boundary = []
    size = sch.node_size
    flops = 0.0
    for k in range(sn_ptr.size - 1):
        sn = [int(v) for v in order[sn_ptr[k]:sn_ptr[k + 1]]]
        sset = set(sn)
        bnd = set()
        for v in sn:
            bnd |= adj[v]
        bnd -= sset
        bl = sorted(bnd, key=lambda w: pos[w])
        assert all(pos[w] >= sn_ptr[k + 1] for w in bl)
        boundary.append(np.array(bl, dtype=np.int64))
        for w in bl:
            adj[w] |= bnd
            adj[w].discard(w)
            adj[w] -= sset
        s = float(sum(size[v] for v in sn))
        b = float(sum(size[w] for w in bl))
        flops += (2.0 / 3.0) * s ** 3 + 2.0 * s * s * b + 2.0 * s * b * b
    sn_closure = np.array([clo[order[sn_ptr[k]]] for k in range(sn_ptr.size - 1)], dtype=np.int64)
    return Symbolic(clo, order, sn_ptr, sn_closure, dep[sn_closure], boundary, flops)


@dataclasses.dataclass
class Factors:
    sym: Symbolic
    node_off: np.ndarray
    lu: list       # per supernode: (lu, piv) from getrf
    L21: list
    U12: list


def _rows(node_off, nodes):
    if len(nodes) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.concatenate([np.arange(node_off[v], node_off[v + 1]) for v in nodes])


def _gather(M: dict, rows: list, cols: list, size) -> np.ndarray:
    ro = np.concatenate([[0], np.cumsum([size[v] for v in rows])]).astype(np.int64)
    co = np.concatenate([[0], np.cumsum([size[v] for v in cols])]).astype(np.int64)
    out = np.zeros((ro[-1], co[-1]))
    for a, v in enumerate(rows):
        for b, w in enumerate(cols):
            blk = M.get((v, w))
            if blk is not None:
                out[ro[a]:ro[a + 1], co[b]:co[b + 1]] = blk
    return out


def getrf_tile(F: np.ndarray, nb: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """P F = L U with the pivot of column j searched only among rows j .. the
    end of the nb-row diagonal tile that holds j (LAPACK ipiv convention,
    L unit lower and U in one array).  A further restriction of the pivoting
    reading above, for the FP32 preconditioner: a panel's pivots then come
    from its own diagonal tile, so the rows below need no search.  With
    nb >= the block size it is getrf's partial pivoting.  Plain unblocked
    right-looking elimination; a zero pivot raises LinAlgError.
    """
    A = np.array(F, dtype=np.float64, copy=True)
    s = A.shape[0]
    piv = np.arange(s)
    for j in range(s):
        t_end = min((j // nb + 1) * nb, s)
        p = j + int(np.argmax(np.abs(A[j:t_end, j])))
        piv[j] = p
        if p != j:
            A[[j, p]] = A[[p, j]]
        if A[j, j] == 0.0:
            raise np.linalg.LinAlgError("zero pivot in column %d" % j)
        A[j + 1:, j] /= A[j, j]
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    return A, piv


def factor(h, sp: Sparsified, sym: Symbolic | None = None, pivot: str = "supernode") -> Factors:
    """Block LU of S; pivot = "supernode" (getrf on each pivot block) or
    "tile" (getrf_tile, the pivot of each column from its 64-row diagonal tile)."""
    if sym is None:
        sym = symbolic(h, sp)
    size = sp.sch.node_size
    M = {k: v.copy() for k, v in sp.blocks.items()}
    LU, L21s, U12s = [], [], []
    for k in range(sym.sn_ptr.size - 1):
        sn = [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]]
        bd = [int(w) for w in sym.boundary[k]]
        F11 = _gather(M, sn, sn, size)
        F12 = _gather(M, sn, bd, size)
        F21 = _gather(M, bd, sn, size)
        lu, piv = sla.lu_factor(F11, check_finite=True) if pivot == "supernode" else getrf_tile(F11)
        if np.any(np.diag(lu) == 0.0):
            raise np.linalg.LinAlgError("zero pivot in supernode %d" % k)
        F12p = F12.copy()
        for i, p in enumerate(piv):
            if p != i:
                F12p[[i, p]] = F12p[[p, i]]
        U12 = sla.solve_triangular(lu, F12p, lower=True, unit_diagonal=True) if F12p.size else F12p
        L21 = sla.solve_triangular(lu, F21.T, trans="T", lower=False).T if F21.size else F21
        LU.append((lu, piv))
        L21s.append(L21)
        U12s.append(U12)
        if bd:
            upd = L21 @ U12
            bo = np.concatenate([[0], np.cumsum([size[w] for w in bd])]).astype(np.int64)
            for a, w1 in enumerate(bd):
                for b, w2 in enumerate(bd):
                    blk = upd[bo[a]:bo[a + 1], bo[b]:bo[b + 1]]
                    if (w1, w2) in M:
                        M[(w1, w2)] = M[(w1, w2)] - blk
                    else:
                        M[(w1, w2)] = -blk
        for v in sn:
            for w in list(bd) + sn:
                M.pop((v, w), None)
                M.pop((w, v), None)
    return Factors(sym, sp.sch.node_off, LU, L21s, U12s)


def solve_S(fa: Factors, c: np.ndarray) -> np.ndarray:
    """y = S^{-1} c by the stored block factors (forward then backward sweep)."""
    sym = fa.sym
    y = np.array(c, dtype=np.float64, copy=True).reshape(c.shape[0], -1)
    rows = [_rows(fa.node_off, [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]])
            for k in range(sym.sn_ptr.size - 1)]
    brows = [_rows(fa.node_off, [int(w) for w in sym.boundary[k]]) for k in range(sym.sn_ptr.size - 1)]
    for k in range(len(rows)):
        lu, piv = fa.lu[k]
        ys = y[rows[k]]
        for i, p in enumerate(piv):
            if p != i:
                ys[[i, p]] = ys[[p, i]]
        ys = sla.solve_triangular(lu, ys, lower=True, unit_diagonal=True)
        y[rows[k]] = ys
        if brows[k].size:
            y[brows[k]] -= fa.L21[k] @ ys
    for k in range(len(rows) - 1, -1, -1):
        lu, _ = fa.lu[k]
        ys = y[rows[k]]
        if brows[k].size:
            ys = ys - fa.U12[k] @ y[brows[k]]
        y[rows[k]] = sla.solve_triangular(lu, ys, lower=False)
    return y.reshape(np.shape(c))


@dataclasses.dataclass
class CholFactors:
    sym: Symbolic
    node_off: np.ndarray
    L11: list      # per supernode: lower Cholesky factor of its pivot block
    L21: list      # per supernode: boundary rows x supernode columns


def cholesky(h, sp: Sparsified, sym: Symbolic | None = None) -> CholFactors:
    """Block Cholesky S = L L^T for a symmetric positive definite S.

    The sparse package the paper factors S with (§5.3-5.4) is a Cholesky
    code, and an SPD A gives an SPD S (Proposition 2.1: S = U^T A U with U
    orthogonal).  Same supernodes, elimination order and boundaries as
    factor(); per supernode, right-looking:
        F11 = L11 L11^T          (dense Cholesky of the pivot block, LAPACK potrf)
        L21 = F21 L11^-T
        M[w1, w2] -= L21[w1] L21[w2]^T   for all boundary pairs (w1, w2).
    No pivoting: a pivot block that is not positive definite raises
    LinAlgError.
    """
    if sym is None:
        sym = symbolic(h, sp)
    size = sp.sch.node_size
    M = {k: v.copy() for k, v in sp.blocks.items()}
    L11s, L21s = [], []
    for k in range(sym.sn_ptr.size - 1):
        sn = [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]]
        bd = [int(w) for w in sym.boundary[k]]
        F11 = _gather(M, sn, sn, size)
        F21 = _gather(M, bd, sn, size)
        L11 = sla.cholesky(F11, lower=True, check_finite=True)
        L21 = sla.solve_triangular(L11, F21.T, lower=True).T if F21.size else F21
        L11s.append(L11)
        L21s.append(L21)
        if bd:
            upd = L21 @ L21.T
            bo = np.concatenate([[0], np.cumsum([size[w] for w in bd])]).astype(np.int64)
            for a, w1 in enumerate(bd):
                for b, w2 in enumerate(bd):
                    blk = upd[bo[a]:bo[a + 1], bo[b]:bo[b + 1]]
                    if (w1, w2) in M:
                        M[(w1, w2)] = M[(w1, w2)] - blk
                    else:
                        M[(w1, w2)] = -blk
        for v in sn:
            for w in list(bd) + sn:
                M.pop((v, w), None)
                M.pop((w, v), None)
    return CholFactors(sym, sp.sch.node_off, L11s, L21s)


def solve_S_chol(fa: CholFactors, c: np.ndarray) -> np.ndarray:
    """y = S^{-1} c = L^-T L^-1 c by the block Cholesky factors."""
    sym = fa.sym
    y = np.array(c, dtype=np.float64, copy=True).reshape(c.shape[0], -1)
    rows = [_rows(fa.node_off, [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]])
            for k in range(sym.sn_ptr.size - 1)]
    brows = [_rows(fa.node_off, [int(w) for w in sym.boundary[k]]) for k in range(sym.sn_ptr.size - 1)]
    for k in range(len(rows)):
        ys = sla.solve_triangular(fa.L11[k], y[rows[k]], lower=True)
        y[rows[k]] = ys
        if brows[k].size:
            y[brows[k]] -= fa.L21[k] @ ys
    for k in range(len(rows) - 1, -1, -1):
        ys = y[rows[k]]
        if brows[k].size:
            ys = ys - fa.L21[k].T @ y[brows[k]]
        y[rows[k]] = sla.solve_triangular(fa.L11[k], ys, lower=True, trans="T")
    return y.reshape(np.shape(c))


def logdet_chol(fa: CholFactors) -> float:
    """log det S = log det A (> 0 for SPD A, V = U) = 2 sum_j log l_jj (§5.3)."""
    return 2.0 * sum(float(np.sum(np.log(np.diag(L)))) for L in fa.L11)


def logdet(fa: Factors) -> tuple[float, int]:
    """log|det A| and the sign of det S of one system, from the block LU of S.

    §5.3 proposes the factorization of the sparse S as the way to the
    determinant of the dense matrix (the use HODLR factorizations are put to).
    U and V are orthogonal (Eq. main_uv), so A = U S V^T (Eq. main_fact) has
    |det A| = |det S|; with symmetric bases (V = U) also det A = det U^2 det S
    = det S.  Block elimination factors det S into the determinants of the
    supernodes' pivot blocks after the Schur updates from the supernodes
    eliminated before them, and getrf's F11 = P L U gives
    det F11 = (-1)^(number of interchanges) * prod_j u_jj.  The logarithms are
    summed in FP64 over all pivot blocks.
    """
    total = 0.0
    flips = 0
    for lu, piv in fa.lu:
        d = np.diag(lu)
        total += float(np.sum(np.log(np.abs(d))))
        flips += int(np.count_nonzero(d < 0.0)) + int(np.count_nonzero(piv != np.arange(piv.size)))
    return total, (-1 if flips % 2 else 1)


def solve(h, sp: Sparsified, fa: Factors, b: np.ndarray) -> np.ndarray:
    """x = V S^{-1} U^T b (Eq. sp0: S y = U^T b, x = V y)."""
    from .sparsify import apply_N, apply_T
    c = apply_T(sp, h, b, col=False)
    y = solve_S(fa, c)
    return apply_N(sp, h, y, col=True)
