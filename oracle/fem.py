"""P1 finite elements on the refined mesh (oracle).

Paper Sec. 4.1 (P1 conforming elements, unknowns on the micro-vertices) and
Sec. 4.2 (matrix-free operator application; the stiffness matrix is never
stored on fine levels).  The oracle takes the plain definition:

  A_pq = sum over micro-triangles T of k_T * integral_T grad(phi_p).grad(phi_q)

with phi the P1 hat functions of the level-l mesh.  The element matrix of a
triangle with vertices a, b, c is k_T |T| G^T G, G = the 2x3 matrix of the
(constant) gradients of the barycentric coordinates.  Rows of Dirichlet DoFs
are dropped: the operator maps a full vector (Dirichlet values included) to
its free rows, and returns 0 at Dirichlet DoFs.

Also here: the consistent P1 mass matrix (|T|/12 [[2,1,1],[1,2,1],[1,1,2]]),
the load vector b = M f_I of an interpolated right-hand side, and the
discrete L2 error by Radon's 7-point degree-5 rule on every micro-triangle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Level


def element_geometry(level: Level):
    """Per element: area |T| (n_el,) and barycentric gradients (n_el, 2, 3)."""
    X = level.coords[level.elements]            # (n_el, 3, 2)
    D = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)   # columns b-a, c-a
    det = D[:, 0, 0] * D[:, 1, 1] - D[:, 0, 1] * D[:, 1, 0]
    area = 0.5 * np.abs(det)
    inv = np.empty_like(D)
    inv[:, 0, 0] = D[:, 1, 1] / det
    inv[:, 0, 1] = -D[:, 0, 1] / det
    inv[:, 1, 0] = -D[:, 1, 0] / det
    inv[:, 1, 1] = D[:, 0, 0] / det
    ref = np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])   # grads of barycentrics in reference coords
    G = np.einsum("eji,jk->eik", inv, ref)                # inv^T @ ref: physical gradients
    return area, G


def element_stiffness(level: Level, k_elem=None):
    """(n_el, 3, 3) element stiffness matrices k_T |T| G^T G."""
    area, G = element_geometry(level)
    K = area[:, None, None] * np.einsum("eia,eib->eab", G, G)
    if k_elem is not None:
        K = K * np.asarray(k_elem, dtype=np.float64)[:, None, None]
    return K


def assemble(level: Level, k_elem=None) -> sp.csr_matrix:
    """Brute-force assembled stiffness matrix over ALL unknowns (n x n)."""
    K = element_stiffness(level, k_elem)
    E = level.elements
    rows = np.repeat(E, 3, axis=1).ravel()
    cols = np.tile(E, (1, 3)).ravel()
    A = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(level.n, level.n)).tocsr()
    A.sum_duplicates()
    return A


def apply_element_loop(level: Level, x, k_elem=None, K=None):
    """y = A x by a loop over micro-triangles (each adds K_T x_T to y), then
    y = 0 at Dirichlet rows.  Independent of the CSR assembly above."""
    if K is None:
        K = element_stiffness(level, k_elem)
    E = level.elements
    xe = np.asarray(x, dtype=np.float64)[E]               # (n_el, 3)
    ye = np.einsum("eab,eb->ea", K, xe)
    y = np.bincount(E.ravel(), weights=ye.ravel(), minlength=level.n)
    y[~level.free] = 0.0
    return y


def free_rows(A: sp.csr_matrix, level: Level):
    """The operator restricted to free rows, as an n x n matrix whose
    Dirichlet rows are zero."""
    d = sp.diags(level.free.astype(np.float64))
    return (d @ A).tocsr()


def mass_matrix(level: Level) -> sp.csr_matrix:
    area, _ = element_geometry(level)
    loc = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0
    Me = area[:, None, None] * loc[None, :, :]
    E = level.elements
    rows = np.repeat(E, 3, axis=1).ravel()
    cols = np.tile(E, (1, 3)).ravel()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(level.n, level.n)).tocsr()
    M.sum_duplicates()
    return M


def load_vector(level: Level, f):
    """b = M f_I on free rows (f sampled at the unknowns), 0 at Dirichlet rows."""
    fI = f(level.coords[:, 0], level.coords[:, 1])
    b = mass_matrix(level) @ fI
    b[~level.free] = 0.0
    return b


def radon7():
    """Radon's 7-point rule on a triangle (exact to degree 5), written from
    its closed form: the centroid with weight 9/40 and two orbits
    (a, a, 1-2a), a = (6 -+ sqrt 15)/21, weights (155 -+ sqrt 15)/1200.
    Returns barycentric points (7, 3) and weights (7,) summing to 1."""
    s = np.sqrt(15.0)
    a1, w1 = (6.0 - s) / 21.0, (155.0 - s) / 1200.0
    a2, w2 = (6.0 + s) / 21.0, (155.0 + s) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3)]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        pts += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


def l2_error(level: Level, uh, u_exact):
    """sqrt( sum_T integral_T (u_h - u)^2 ) with Radon's rule per micro-triangle."""
    B, w = radon7()
    X = level.coords[level.elements]                        # (n_el, 3, 2)
    area, _ = element_geometry(level)
    P = np.einsum("qk,ekd->eqd", B, X)                      # (n_el, 7, 2)
    uq = np.einsum("qk,ek->eq", B, np.asarray(uh)[level.elements])
    err = (uq - u_exact(P[..., 0], P[..., 1])) ** 2
    return float(np.sqrt(np.sum(area[:, None] * w[None, :] * err)))
