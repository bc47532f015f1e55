"""The H^2 matrix itself (Definition 4.9, §4.1), written out plainly.

A = C + sum over admissible pairs b=(t,s) of R_t D_b E_s^T, where C is the
close matrix (Definition 4.8), R_t / E_s are the row / column cluster basis
matrices (Definition 4.7) and D_b the coupling matrices.  The cluster bases of
internal clusters are nested: R_t = [R_c T_c] stacked over the sons c of t.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def children(h) -> list[list[int]]:
    kids = [[] for _ in range(h.ncl)]
    for c in range(1, h.ncl):
        kids[int(h.parent[c])].append(c)
    return kids


def expanded_basis(h, col: bool = False) -> list[np.ndarray]:
    """R_t for every cluster t as an explicit (|t| x k_t) matrix, built from
    the leaf bases and the transfer matrices by the nestedness relation."""
    D = h.depth
    lp = h.level_ptr
    kids = children(h)
    R = [None] * h.ncl
    for t in range(lp[D], lp[D + 1]):
        R[t] = h.leaf_R(t, col)
    for d in range(D - 1, -1, -1):
        for t in range(lp[d], lp[d + 1]):
            R[t] = np.vstack([R[c] @ h.T(c, col) for c in kids[t]])
    return R


def dense(h) -> np.ndarray:
    """The full N x N matrix of Definition 4.9 (small N only)."""
    A = np.zeros((h.n, h.n))
    R = expanded_basis(h)
    E = R if h.symmetric_bases else expanded_basis(h, col=True)
    D = h.depth
    base = int(h.level_ptr[D])
    for lf in range(h.nleaf):
        t = base + lf
        bt, nt = int(h.begin[t]), int(h.size[t])
        for i in range(int(h.near_ptr[lf]), int(h.near_ptr[lf + 1])):
            s = int(h.near_col[i])
            bs, ns = int(h.begin[s]), int(h.size[s])
            A[bt:bt + nt, bs:bs + ns] += h.C(i, t, s)
    for t in range(h.ncl):
        bt, nt = int(h.begin[t]), int(h.size[t])
        for i in range(int(h.far_ptr[t]), int(h.far_ptr[t + 1])):
            s = int(h.far_col[i])
            bs, ns = int(h.begin[s]), int(h.size[s])
            A[bt:bt + nt, bs:bs + ns] += R[t] @ h.D(i, t, s) @ E[s].T
    return A


class Matvec:
    """y = A x with A given by Definition 4.9, block by block (no dense A).

    The expanded bases are formed once; each admissible block contributes
    R_t (D_ts (E_s^T x_s)) and each close block C_ts x_s."""

    def __init__(self, h):
        self.h = h
        self.R = expanded_basis(h)
        self.E = self.R if h.symmetric_bases else expanded_basis(h, col=True)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        h = self.h
        x2 = x.reshape(h.n, -1)
        y = np.zeros_like(x2, dtype=np.float64)
        D = h.depth
        base = int(h.level_ptr[D])
        for lf in range(h.nleaf):
            t = base + lf
            bt, nt = int(h.begin[t]), int(h.size[t])
            for i in range(int(h.near_ptr[lf]), int(h.near_ptr[lf + 1])):
                s = int(h.near_col[i])
                bs, ns = int(h.begin[s]), int(h.size[s])
                y[bt:bt + nt] += h.C(i, t, s) @ x2[bs:bs + ns]
        for t in range(h.ncl):
            lo, hi = int(h.far_ptr[t]), int(h.far_ptr[t + 1])
            if lo == hi:
                continue
            bt, nt = int(h.begin[t]), int(h.size[t])
            acc = np.zeros((self.R[t].shape[1], x2.shape[1]))
            for i in range(lo, hi):
                s = int(h.far_col[i])
                bs, ns = int(h.begin[s]), int(h.size[s])
                acc += h.D(i, t, s) @ (self.E[s].T @ x2[bs:bs + ns])
            y[bt:bt + nt] += self.R[t] @ acc
        return y.reshape(x.shape)
