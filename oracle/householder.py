"""Householder QR with square orthogonal completion (§4.2).

§4.2 builds the square orthogonal diagonal blocks of U_k from the rectangular
cluster basis blocks: orthogonalise each block and complete it to a square
orthogonal matrix by a QR decomposition with the square Q factor.  The paper
fixes no convention; the reading taken here is LAPACK's (the one dgeqrf /
dorgqr use):

  for j = 0 .. k'-1 (k' = min(m, k)):
    x = A[j:, j];  alpha = x[0];  s = ||x[1:]||
    if s == 0:  tau_j = 0 (H_j = I)
    else:       beta = -sign(alpha) * hypot(alpha, s)   (sign(0) = +1)
                tau_j = (beta - alpha) / beta
                v_j = x / (alpha - beta), v_j[0] = 1
    A[j:, j:] <- (I - tau_j v_j v_j^T) A[j:, j:]
  Rr = upper trapezoid of A[:k', :]            (k' x k)
  Q  = H_0 H_1 ... H_{k'-1} applied to I_m     (m x m)

so that W = Q[:, :k'] Rr.  Columns [0, k') of Q span the basis (the "basis"
rows of §2.2); columns [k', m) are the orthogonal complement (the
"non-basis" rows).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np


def householder_complete(W: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Return (Q, Rr): Q is m x m orthogonal, Rr is k' x k, W = Q[:, :k'] @ Rr."""
    W = np.asarray(W, dtype=np.float64)
    m, k = W.shape
    kp = min(m, k)
    A = W.copy()
    vs, taus = [], []
    for j in range(kp):
        x = A[j:, j].copy()
        alpha = x[0]
        s = math.sqrt(float(np.dot(x[1:], x[1:]))) if x.size > 1 else 0.0
        if s == 0.0:
            tau = 0.0
            v = np.zeros_like(x)
            v[0] = 1.0
        else:
            beta = -math.copysign(math.hypot(alpha, s), alpha)
            tau = (beta - alpha) / beta
            v = x / (alpha - beta)
            v[0] = 1.0
        if tau != 0.0:
            A[j:, j:] -= tau * np.outer(v, v @ A[j:, j:])
        vs.append(v)
        taus.append(tau)
    Rr = np.triu(A[:kp, :])
    Q = np.eye(m)
    for j in range(kp - 1, -1, -1):
        if taus[j] != 0.0:
            v = vs[j]
            Q[j:, :] -= taus[j] * np.outer(v, v @ Q[j:, :])
    return Q, Rr
