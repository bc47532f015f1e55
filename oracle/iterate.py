"""Iterative solves with the factored sparsification as preconditioner (§5.5).

§5.5 runs GMRES on the H^2 matrix-vector product, preconditioned by the
sparsified and factored H^2 matrix, to a relative residual of 1e-10.  Here
the preconditioner is M^{-1} = V S^{-1} U^T (the direct solve of Eq. sp0) and
two drivers are written out: iterative refinement and restarted GMRES with
right preconditioning (Saad's formulation with Givens rotations).

Residuals are max_k ||b_k - A x_k||_2 / ||b_k||_2 over the right-hand sides,
with A the FP64 H^2 matvec of Definition 4.9.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np


def rel_residual(matvec, b: np.ndarray, x: np.ndarray) -> float:
    r = b - matvec(x)
    b2 = b.reshape(b.shape[0], -1)
    r2 = r.reshape(b.shape[0], -1)
    return float(np.max(np.linalg.norm(r2, axis=0) / np.linalg.norm(b2, axis=0)))


def refine(matvec, precond, b: np.ndarray, tol: float = 1e-10, maxit: int = 50):
    """x_0 = M^-1 b;  x_{i+1} = x_i + M^-1 (b - A x_i) until the residual <= tol."""
    x = precond(b)
    hist = []
    for _ in range(maxit + 1):
        res = rel_residual(matvec, b, x)
        hist.append(res)
        if res <= tol:
            break
        x = x + precond(b - matvec(x))
    return x, hist


def gmres(matvec, precond, b: np.ndarray, tol: float = 1e-10, restart: int = 30, maxit: int = 300):
    """Right-preconditioned restarted GMRES for one right-hand side."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    hist = []
    it = 0
    while it < maxit:
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) / bnorm <= tol or it >= maxit:
                break
        yk = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done]) if j_done else np.zeros(0)
        x = x + Z[:j_done].T @ yk
    hist.append(rel_residual(matvec, b, x))
    return x, hist
