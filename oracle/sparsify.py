"""Level-by-level sparsification A = U S V^T from H^2 parameters (§2, §4).

The construction follows §2.1-2.3 (compression at level zero, basis /
non-basis permutation, grouping into big blocks, recursion over all levels)
with the factors built from the H^2 parameters as §4.2-4.3 prescribe:

* level 0 (the leaves): the block rows of the close matrix C_0 and of the
  leaf cluster bases are transformed by the square orthogonal blocks Q_t that
  complete the leaf bases (§2.1, Eqs. q and v; §4.2).  After this every far
  block lives in the k' x k' "basis" corner (§2.1).
* the basis / non-basis permutation P_r1, P_c1 (§2.2) puts the non-basis rows
  and columns (the orthogonal complement of the basis) first; the non-basis
  part of cluster t at level l becomes the S node (l, t).
* the basis rows of the sons of a level-(l+1) cluster form its local space
  X_{l+1}(p) (grouping into big blocks, §2.2).  The far blocks between sons of
  a close big block move into the close matrix (Eq. cl1); those are exactly
  the couplings of the interaction list at level l projected on the basis,
  Rr_t D_ts Rr_s^T (§4.3: the F_ml matrices are the coupling matrices).
* the same step is repeated at every level (§2.3, Eq. fin).  Non-basis rows
  already final keep being transformed on the column side by the higher
  levels' blocks (the products of U_k in Eq. main_uv), which produces the
  mixed-level blocks S_ij of §3.
* the process stops at l_stop, the lowest level from which on no admissible
  pair exists; the remaining level-l_stop clusters are kept uncompressed and
  form the "top" nodes of S (the last term F_L of §4.3 is the projection of
  the couplings of level l_stop - 1).

Readings taken where the paper is silent or inconsistent:
* the factor direction is A = U S V^T with S = U^T A V (Eq. main_fact,
  §2.1); the pseudo-code's A_{j+1} = U_j A_j V_j^T is read as a typo.
* within a level, clusters are in tree order; within a cluster the
  non-basis columns follow Householder column order.  S node order: the
  non-basis nodes of level 0, then of level 1, ... then the top nodes.
* a cluster with k_t >= m_t keeps k' = min(k_t, m_t) basis columns and owns
  no S node at that level.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .householder import householder_complete


@dataclasses.dataclass
class Schedule:
    """Integer structure of the level recursion (a1)."""
    D: int
    lstop: int
    level: np.ndarray            # int64[ncl]: l = D - depth
    clusters: list               # per level l: array of cluster ids
    m: np.ndarray                # local size of X_l(t)
    kp: np.ndarray               # k' = min(k, m) (0 at and above l_stop)
    d: np.ndarray                # non-basis size m - k' (= m for top clusters)
    off: np.ndarray              # offset of t's basis block inside X_{l+1}(parent)
    xoff: np.ndarray             # offset of X_l(t) inside the level-l space
    near: list                   # per level l <= l_stop: int64 (P, 2) sorted pairs
    far: list                    # per level l < D+1: int64 (F, 3): (t, s, coupling index)
    node_of: dict                # (l, t) -> S node id
    node_level: np.ndarray
    node_cluster: np.ndarray
    node_size: np.ndarray
    node_off: np.ndarray         # int64[nnodes+1]


def schedule(h) -> Schedule:
    D = h.depth
    lp = h.level_ptr
    ncl = h.ncl
    level = np.zeros(ncl, dtype=np.int64)
    for d in range(D + 1):
        level[lp[d]:lp[d + 1]] = D - d
    clusters = [np.arange(lp[D - l], lp[D - l + 1], dtype=np.int64) for l in range(D + 1)]
    # interaction lists by level
    far = [[] for _ in range(D + 1)]
    for t in range(ncl):
        for i in range(int(h.far_ptr[t]), int(h.far_ptr[t + 1])):
            far[level[t]].append((t, int(h.far_col[i]), i))
    far = [np.array(f, dtype=np.int64).reshape(-1, 3) for f in far]
    lstop = 0
    for l in range(D + 1):
        if far[l].shape[0] > 0:
            lstop = l + 1
    # near lists: Near_0 from the close matrix, Near_{l+1} = parents of Near_l and Far_l
    base = int(lp[D])
    n0 = []
    for lf in range(h.nleaf):
        for i in range(int(h.near_ptr[lf]), int(h.near_ptr[lf + 1])):
            n0.append((base + lf, int(h.near_col[i])))
    near = [np.array(sorted(n0), dtype=np.int64).reshape(-1, 2)]
    for l in range(lstop):
        pairs = set()
        for (a, b) in near[l]:
            pairs.add((int(h.parent[a]), int(h.parent[b])))
        for (a, b, _) in far[l]:
            pairs.add((int(h.parent[a]), int(h.parent[b])))
        near.append(np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2))
    # sizes
    k = h.rank.astype(np.int64)
    m = np.zeros(ncl, dtype=np.int64)
    kp = np.zeros(ncl, dtype=np.int64)
    d_ = np.zeros(ncl, dtype=np.int64)
    off = np.zeros(ncl, dtype=np.int64)
    xoff = np.zeros(ncl, dtype=np.int64)
    for t in clusters[0]:
        m[t] = h.size[t]
    for l in range(lstop + 1):
        acc = 0
        for t in clusters[l]:
            xoff[t] = acc
            acc += m[t]
            if l < lstop:
                kp[t] = min(k[t], m[t])
                d_[t] = m[t] - kp[t]
            else:
                kp[t] = 0
                d_[t] = m[t]
        if l < lstop:
            for t in clusters[l]:
                p = int(h.parent[t])
                off[t] = m[p]
                m[p] += kp[t]
    node_of = {}
    nl, nc, ns = [], [], []
    for l in range(lstop + 1):
        for t in clusters[l]:
            if d_[t] > 0:
                node_of[(l, int(t))] = len(nl)
                nl.append(l)
                nc.append(int(t))
                ns.append(int(d_[t]))
    node_size = np.array(ns, dtype=np.int64)
    node_off = np.concatenate([[0], np.cumsum(node_size)]).astype(np.int64)
    assert node_off[-1] == h.n
    return Schedule(D, lstop, level, clusters, m, kp, d_, off, xoff, near, far, node_of,
                    np.array(nl, dtype=np.int64), np.array(nc, dtype=np.int64), node_size, node_off)


@dataclasses.dataclass
class Sparsified:
    sch: Schedule
    Q: dict          # cluster -> m x m row completion (levels < l_stop)
    Qc: dict         # column completion (same object as Q for symmetric bases)
    Rr: dict
    Rrc: dict
    blocks: dict     # (row node, col node) -> dense block of S


def _put(store: dict, key, shape, r0: int, c0: int, blk: np.ndarray):
    if key not in store:
        store[key] = np.zeros(shape)
    store[key][r0:r0 + blk.shape[0], c0:c0 + blk.shape[1]] = blk


def sparsify(h) -> Sparsified:
    """Run §2.1-2.3 on the H^2 parameters (§4.2-4.3) and return S block-wise."""
    sch = schedule(h)
    sym = h.symmetric_bases
    lstop = sch.lstop
    m, kp, d_, off = sch.m, sch.kp, sch.d, sch.off
    par = h.parent
    kids = [[] for _ in range(h.ncl)]
    for c in range(1, h.ncl):
        kids[int(par[c])].append(c)
    node = sch.node_of
    Q, Qc, Rr, Rrc = {}, {}, {}, {}
    S = {}
    # C_0: the close matrix, block by block over Near_0
    base = int(h.level_ptr[h.depth])
    C = {}
    for lf in range(h.nleaf):
        t = base + lf
        for i in range(int(h.near_ptr[lf]), int(h.near_ptr[lf + 1])):
            s = int(h.near_col[i])
            C[(t, s)] = h.C(i, t, s).copy()
    rowpan, colpan = {}, {}
    for l in range(lstop):
        # a2: orthogonal completion of the level-l bases (§4.2)
        for t in sch.clusters[l]:
            t = int(t)
            if l == 0:
                W = h.leaf_R(t)
                Wc = None if sym else h.leaf_R(t, col=True)
            else:
                W = np.vstack([Rr[c] @ h.T(c) for c in kids[t]]) if kids[t] else np.zeros((0, h.rank[t]))
                Wc = None if sym else np.vstack([Rrc[c] @ h.T(c, col=True) for c in kids[t]])
            Q[t], Rr[t] = householder_complete(W)
            if sym:
                Qc[t], Rrc[t] = Q[t], Rr[t]
            else:
                Qc[t], Rrc[t] = householder_complete(Wc)
        Cn, rpn, cpn = {}, {}, {}
        # a3: far blocks of the interaction list become close blocks of the
        #     next level (Eq. cl1), projected on the basis corner.
        for (p, q, i) in sch.far[l]:
            p, q, i = int(p), int(q), int(i)
            F = Rr[p] @ h.D(i, p, q) @ Rrc[q].T
            _put(Cn, (int(par[p]), int(par[q])), (m[par[p]], m[par[q]]), off[p], off[q], F)
        # a4: close blocks, B = Q_p^T C_l(p,q) Q_q split into the four parts
        for (p, q) in sch.near[l]:
            p, q = int(p), int(q)
            B = Q[p].T @ C.get((p, q), np.zeros((m[p], m[q]))) @ Qc[q]
            a, b = kp[p], kp[q]
            if d_[p] and d_[q]:
                S[(node[(l, p)], node[(l, q)])] = B[a:, b:]
            if d_[p]:
                _put(rpn, (node[(l, p)], int(par[q])), (d_[p], m[par[q]]), 0, off[q], B[a:, :b])
            if d_[q]:
                _put(cpn, (int(par[p]), node[(l, q)]), (m[par[p]], d_[q]), off[p], 0, B[:a, b:])
            _put(Cn, (int(par[p]), int(par[q])), (m[par[p]], m[par[q]]), off[p], off[q], B[:a, :b])
        # a5: non-basis rows (columns) of lower levels see the level-l column
        #     (row) transforms of the clusters they touch (Eq. main_uv products)
        for (v, q), P in rowpan.items():
            T = P @ Qc[q]
            b = kp[q]
            if d_[q]:
                S[(v, node[(l, q)])] = T[:, b:]
            _put(rpn, (v, int(par[q])), (P.shape[0], m[par[q]]), 0, off[q], T[:, :b])
        for (p, w), P in colpan.items():
            T = Q[p].T @ P
            a = kp[p]
            if d_[p]:
                S[(node[(l, p)], w)] = T[a:, :]
            _put(cpn, (int(par[p]), w), (m[par[p]], P.shape[1]), off[p], 0, T[:a, :])
        C, rowpan, colpan = Cn, rpn, cpn
    # top: the level-l_stop clusters stay uncompressed
    for (p, q) in sch.near[lstop]:
        p, q = int(p), int(q)
        if m[p] and m[q]:
            S[(node[(lstop, p)], node[(lstop, q)])] = C.get((p, q), np.zeros((m[p], m[q])))
    for (v, q), P in rowpan.items():
        if (lstop, q) in node:
            S[(v, node[(lstop, q)])] = P
    for (p, w), P in colpan.items():
        if (lstop, p) in node:
            S[(node[(lstop, p)], w)] = P
    return Sparsified(sch, Q, Qc, Rr, Rrc, S)


# ---------------------------------------------------------------------------
# VBR layout of S
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class VBR:
    node_size: np.ndarray
    node_off: np.ndarray
    brow_ptr: np.ndarray   # int64[nnodes+1]
    bcol_idx: np.ndarray   # int32[nnzb]
    val_off: np.ndarray    # int64[nnzb]
    vals: np.ndarray       # float64, each block column-major


def to_vbr(sp: Sparsified) -> VBR:
    sch = sp.sch
    nn = sch.node_size.shape[0]
    keys = sorted(sp.blocks.keys())
    brow_ptr = np.zeros(nn + 1, dtype=np.int64)
    for (i, _) in keys:
        brow_ptr[i + 1] += 1
    brow_ptr = np.cumsum(brow_ptr)
    bcol_idx = np.array([j for (_, j) in keys], dtype=np.int32)
    sizes = np.array([sch.node_size[i] * sch.node_size[j] for (i, j) in keys], dtype=np.int64)
    val_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if keys else np.zeros(0, np.int64)
    vals = np.zeros(int(sizes.sum()))
    for n_, key in enumerate(keys):
        blk = sp.blocks[key]
        vals[val_off[n_]:val_off[n_] + blk.size] = blk.T.reshape(-1)
    return VBR(sch.node_size, sch.node_off, brow_ptr, bcol_idx, val_off, vals)


def pattern_rule(h, sch: Schedule) -> set:
    """The block pattern of S predicted from the close lists (§3, the
    statement bsp(S_ij) = bsp(C) at block sizes 2^i B x 2^j B): node (i, c)
    couples with node (j, q), j >= i, iff q is the level-j ancestor of a
    level-i close neighbour of c; j < i by transposition; top x top dense."""
    par = h.parent
    anc = {}
    out = set()
    node = sch.node_of

    def up(e, i, j):
        while i < j:
            e = int(par[e])
            i += 1
        return e
    del anc
    for i in range(sch.lstop + 1):
        for (c, e) in sch.near[i]:
            c, e = int(c), int(e)
            for j in range(i, sch.lstop + 1):
                q = up(e, i, j)
                if (i, c) in node and (j, q) in node:
                    out.add((node[(i, c)], node[(j, q)]))
                    out.add((node[(j, q)], node[(i, c)]))
    return out


def dense_S(sp: Sparsified) -> np.ndarray:
    sch = sp.sch
    N = int(sch.node_off[-1])
    S = np.zeros((N, N))
    for (i, j), blk in sp.blocks.items():
        S[sch.node_off[i]:sch.node_off[i + 1], sch.node_off[j]:sch.node_off[j + 1]] = blk
    return S


# ---------------------------------------------------------------------------
# applies of U^T, V (and U, V^T) -- the products of Eq. main_uv
# ---------------------------------------------------------------------------


def _level_width(sch: Schedule, l: int) -> int:
    return int(sum(sch.m[t] for t in sch.clusters[l]))


def apply_T(sp: Sparsified, h, b: np.ndarray, col: bool = False) -> np.ndarray:
    """U^T b (or V^T b with col=True): point space (tree order) -> S node space."""
    sch = sp.sch
    Qd = sp.Qc if col else sp.Q
    b2 = np.asarray(b, dtype=np.float64).reshape(h.n, -1)
    out = np.zeros_like(b2)
    x = b2
    for l in range(sch.lstop):
        xn = np.zeros((_level_width(sch, l + 1), b2.shape[1]))
        for t in sch.clusters[l]:
            t = int(t)
            z = Qd[t].T @ x[sch.xoff[t]:sch.xoff[t] + sch.m[t]]
            a = sch.kp[t]
            if sch.d[t]:
                v = sch.node_of[(l, t)]
                out[sch.node_off[v]:sch.node_off[v + 1]] = z[a:]
            p = int(h.parent[t])
            xn[sch.xoff[p] + sch.off[t]: sch.xoff[p] + sch.off[t] + a] = z[:a]
        x = xn
    for t in sch.clusters[sch.lstop]:
        t = int(t)
        if sch.m[t]:
            v = sch.node_of[(sch.lstop, t)]
            out[sch.node_off[v]:sch.node_off[v + 1]] = x[sch.xoff[t]:sch.xoff[t] + sch.m[t]]
    return out.reshape(np.shape(b))


def apply_N(sp: Sparsified, h, y: np.ndarray, col: bool = True) -> np.ndarray:
    """V y (col=True) or U y (col=False): S node space -> point space."""
    sch = sp.sch
    Qd = sp.Qc if col else sp.Q
    y2 = np.asarray(y, dtype=np.float64).reshape(h.n, -1)
    x = np.zeros((_level_width(sch, sch.lstop), y2.shape[1]))
    for t in sch.clusters[sch.lstop]:
        t = int(t)
        if sch.m[t]:
            v = sch.node_of[(sch.lstop, t)]
            x[sch.xoff[t]:sch.xoff[t] + sch.m[t]] = y2[sch.node_off[v]:sch.node_off[v + 1]]
    for l in range(sch.lstop - 1, -1, -1):
        xl = np.zeros((_level_width(sch, l), y2.shape[1]))
        for t in sch.clusters[l]:
            t = int(t)
            a = sch.kp[t]
            p = int(h.parent[t])
            z = np.zeros((sch.m[t], y2.shape[1]))
            z[:a] = x[sch.xoff[p] + sch.off[t]: sch.xoff[p] + sch.off[t] + a]
            if sch.d[t]:
                v = sch.node_of[(l, t)]
                z[a:] = y2[sch.node_off[v]:sch.node_off[v + 1]]
            xl[sch.xoff[t]:sch.xoff[t] + sch.m[t]] = Qd[t] @ z
        x = xl
    return x.reshape(np.shape(y))
