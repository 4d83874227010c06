"""Krylov solvers with a multigrid preconditioner (oracle, FP64; test
infrastructure only).  Paper Sec. 4.3: multigrid can be used as a
preconditioner inside a Krylov solver.

* fgmres: FGMRES(m) after Saad (1993): right preconditioning with a
  preconditioner that may change from step to step, modified Gram-Schmidt,
  Givens rotations, restart after m steps.
* pcg: preconditioned conjugate gradients (Hestenes & Stiefel 1952, in the
  preconditioned form of e.g. Saad, Iterative Methods for Sparse Linear
  Systems, Alg. 9.1) for a symmetric positive definite operator and a
  symmetric positive definite preconditioner (one symmetric V-cycle: forward
  Gauss-Seidel before, backward after, exact coarse solve).  flexible=True
  takes the Polak-Ribiere form of beta, z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k)
  (Notay 2000, "Flexible conjugate gradients"), which stays robust when the
  preconditioner varies slightly from step to step (a V-cycle in FP32); with
  r_{k+1} = r_k - alpha q_k it reads -alpha (q_k.z_{k+1}) / (z_k.r_k).

Vectors are full-length; inner products run over the free DoFs only
(Dirichlet entries of the Krylov vectors are zero).
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, precond, b, x0, free, m=20, tol=1e-10, max_iter=200, history=None):
    """Solve A x = b from x0.  apply_A(v) -> A v (zero Dirichlet rows);
    precond(v, j) -> z_j (the j-th preconditioner application).  Stops when
    ||b - A x|| <= tol ||b - A x0||.  Returns (x, residual history, steps)."""
    x = x0.copy()
    dot = lambda u, v: float(np.dot(u[free], v[free]))
    r = b - apply_A(x)
    r[~free] = 0.0
    r0 = np.sqrt(dot(r, r))
    hist = [r0] if history is None else history
    if history is not None:
        hist.append(r0)
    steps = 0
    beta = r0
    while beta > tol * r0 and steps < max_iter:
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = precond(V[j], steps)
            z[~free] = 0.0
            Z.append(z)
            w = apply_A(z)
            w[~free] = 0.0
            for i in range(j + 1):
                H[i, j] = dot(w, V[i])
                w = w - H[i, j] * V[i]
            h_next = np.sqrt(dot(w, w))
            H[j + 1, j] = h_next
            for i in range(j):                   # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            steps += 1
            k = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * r0 or steps >= max_iter or h_next == 0.0:
                break
            V.append(w / h_next)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        r[~free] = 0.0
        beta = np.sqrt(dot(r, r))
        hist[-1] = beta
    return x, hist, steps


def pcg(apply_A, precond, b, x0, free, tol=1e-10, max_iter=200, flexible=False):
    """Solve A x = b from x0 with preconditioner z = precond(r).  Stops when
    the updated residual satisfies ||r|| <= tol ||b - A x0||; the true
    residual is then recomputed and, should it miss the tolerance, the
    iteration restarts from it.  Returns (x, residual-norm history, steps)."""
    x = x0.copy()
    dot = lambda u, v: float(np.dot(u[free], v[free]))
    r = b - apply_A(x)
    r[~free] = 0.0
    r0 = np.sqrt(dot(r, r))
    hist = [r0]
    steps = 0
    if r0 == 0.0:
        return x, hist, steps
    z = precond(r)
    z[~free] = 0.0
    p = z.copy()
    rz = dot(r, z)
    while steps < max_iter:
        q = apply_A(p)
        q[~free] = 0.0
        alpha = rz / dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        steps += 1
        rn = np.sqrt(dot(r, r))
        if rn <= tol * r0:
            rt = b - apply_A(x)
            rt[~free] = 0.0
            rn = np.sqrt(dot(rt, rt))
            hist.append(rn)
            if rn <= tol * r0:
                break
            r = rt                       # restart from the true residual
            z = precond(r)
            z[~free] = 0.0
            p = z.copy()
            rz = dot(r, z)
            continue
        hist.append(rn)
        z = precond(r)
        z[~free] = 0.0
        rz_new = dot(r, z)
        beta = -alpha * dot(q, z) / rz if flexible else rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, hist, steps
