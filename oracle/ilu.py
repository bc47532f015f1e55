"""Threshold incomplete LU of S, the preconditioner of §5.5.

§5.5 preconditions GMRES on the H^2 product with the sparsified matrix
factored by an incomplete LU with a drop tolerance (ILUt; its experiments
take tau = 1e-2 and 2e-2).  The paper names the method and its parameter
only.  The reading taken is the threshold incomplete LU with the threshold
rule alone (no cap on the entries kept per row), restated:

    for each row i of A, in order:
        w = A[i, :],  tau_i = tau * ||A[i, :]||_2
        for k < i with w_k != 0, in increasing k:
            w_k = w_k / u_kk
            if |w_k| < tau_i:  w_k = 0              (the multiplier is dropped)
            else:              w[k+1:] -= w_k U[k, k+1:]
        w_j = 0 for every j != i with |w_j| < tau_i
        L[i, :i] = w[:i] (unit diagonal),  U[i, i:] = w[i:]

There is no pivoting; a zero u_ii raises LinAlgError.  A is S with its rows
and columns in the elimination order of the block LU (nodes in closure order,
the rows of a node kept together), so tau = 0 gives the exact LU without
pivoting of that matrix.  Dense arrays throughout: for small cases only.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .factor import _rows, symbolic
from .sparsify import Sparsified, apply_N, apply_T, dense_S


def ilut(A: np.ndarray, tau: float) -> tuple[np.ndarray, np.ndarray]:
    """(L, U) of the threshold incomplete LU of A (dense), as restated above."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        w = A[i].copy()
        tau_i = tau * float(np.linalg.norm(A[i]))
        for k in range(i):
            if w[k] == 0.0:
                continue
            w[k] /= U[k, k]
            if abs(w[k]) < tau_i:
                w[k] = 0.0
            else:
                w[k + 1:] -= w[k] * U[k, k + 1:]
        small = np.abs(w) < tau_i
        small[i] = False
        w[small] = 0.0
        if w[i] == 0.0:
            raise np.linalg.LinAlgError("zero pivot in row %d" % i)
        L[i, :i] = w[:i]
        U[i, i:] = w[i:]
    return L, U


@dataclasses.dataclass
class IluFactors:
    perm: np.ndarray   # scalar rows of S in elimination order
    L: np.ndarray
    U: np.ndarray
    tau: float


def factor_ilut(h, sp: Sparsified, tau: float) -> IluFactors:
    """ILUt of S in the elimination order of the block LU."""
    sym = symbolic(h, sp)
    perm = np.concatenate([_rows(sp.sch.node_off, [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]])
                           for k in range(sym.sn_ptr.size - 1)])
    S = dense_S(sp)
    L, U = ilut(S[np.ix_(perm, perm)], tau)
    return IluFactors(perm, L, U, tau)


def solve_S_ilu(fa: IluFactors, c: np.ndarray) -> np.ndarray:
    """y = (P^T L U P)^{-1} c, the incomplete factors applied to c."""
    c2 = np.asarray(c, dtype=np.float64).reshape(c.shape[0], -1)
    z = sla.solve_triangular(fa.L, c2[fa.perm], lower=True, unit_diagonal=True)
    z = sla.solve_triangular(fa.U, z, lower=False)
    y = np.empty_like(c2)
    y[fa.perm] = z
    return y.reshape(np.shape(c))


def precondition(h, sp: Sparsified, fa: IluFactors, r: np.ndarray) -> np.ndarray:
    """M^{-1} r = V (L U)^{-1} U^T r: the ILUt preconditioner of §5.5."""
    return apply_N(sp, h, solve_S_ilu(fa, apply_T(sp, h, r, col=False)), col=True)
