"""P2 finite elements and p-multigrid on the refined mesh (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper Sec. 4.1 (conforming P2 elements), Sec. 4.2 (stencils of vertex DoFs
and of horizontal, vertical and diagonal edge DoFs), Sec. 3.1 (the edge
unknowns of a face in three subgroups) and Sec. 4.3 (p-refinement: transfer
between P1 and P2 on the same geometric level).

Unknowns.  P2 on level L has one unknown per micro-vertex and one per
micro-edge midpoint of the level-L mesh.  These are exactly the lattice
points of level L + 1, so the level-(L+1) ``Level`` numbers them: lattice
point (i, j) of level L + 1 is a micro-vertex DoF of level L when i and j
are both even, and the midpoint of a horizontal (i odd, j even), vertical
(i even, j odd) or diagonal (both odd) micro-edge otherwise.

Operator (plain definition): A_pq = sum over the level-L micro-triangles T
of k_T * integral_T grad(phi_p) . grad(phi_q), phi the P2 Lagrange basis.
The integrand is a polynomial of degree 2 on T, so the three-point
edge-midpoint rule (weights |T|/3) integrates it exactly.  Basis on T with
barycentric coordinates l_0, l_1, l_2 (constant gradients g_i):
vertex i: l_i (2 l_i - 1), gradient (4 l_i - 1) g_i; edge (i, j):
4 l_i l_j, gradient 4 (l_j g_i + l_i g_j).  Local node order: v0, v1, v2,
m01, m12, m02.

p-multigrid (Sec. 4.3, p-refinement on one geometric level; the paper gives
no cycle, so this reading): the P1 space of level L is a subspace of the P2
space of level L, and its embedding is linear interpolation onto the level
L + 1 lattice -- the P1 prolongation from level L to L + 1.  One cycle:
nu1 forward colour Gauss-Seidel sweeps on P2, the P2 residual restricted by
the transpose of that embedding, one P1 V(nu1c, nu2c) cycle on level L from
zero for the coarse correction, prolongation and correction, nu2 backward
sweeps.  The coarse operator is the P1 operator of level L with the same
per-element coefficient (equal to the Galerkin product, pinned).

Gauss-Seidel colour order (the paper names multi-colour Gauss-Seidel only;
this reading): free macro-vertices; free macro-edge points of the level-(L+1)
lattice, greedily coloured in canonical order by structural adjacency (two
unknowns are adjacent when a level-L micro-triangle holds both); then the
face-interior points in six sets: micro-vertex points by the level-L colour
(i/2 + 2 j/2) mod 3 = 0, 1, 2, then horizontal, vertical and diagonal edge
points.  Every set is independent (a micro-triangle has three vertices of
distinct colours and exactly one edge of each direction).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import Level, MacroMesh
from .multigrid import Hierarchy, prolongation, vcycle


# ------------------------------------------------------------------ elements
def p2_elements(lat: Level, L: int) -> np.ndarray:
    """(n_faces * N^2, 6) lattice ids (level L + 1 numbering) of the P2 nodes
    of every level-L micro-triangle in canonical element order (per face:
    upward triangles (a, b) row by row, then downward ones), node order
    v0, v1, v2, m01, m12, m02."""
    N = 1 << L
    assert lat.N == 2 * N
    out = []
    for G in lat.face_ids:
        up, dn = [], []
        for b in range(N):
            for a in range(N - b):
                I, J = 2 * a, 2 * b
                up.append([G[J, I], G[J, I + 2], G[J + 2, I],
                           G[J, I + 1], G[J + 1, I + 1], G[J + 1, I]])
        for b in range(N - 1):
            for a in range(N - 1 - b):
                I, J = 2 * a, 2 * b
                dn.append([G[J, I + 2], G[J + 2, I], G[J + 2, I + 2],
                           G[J + 1, I + 1], G[J + 2, I + 1], G[J + 1, I + 2]])
        out.append(np.array(up, dtype=np.int64).reshape(-1, 6))
        if dn:
            out.append(np.array(dn, dtype=np.int64).reshape(-1, 6))
    return np.concatenate(out, axis=0)


def barycentric_gradients(X):
    """X (n, 3, 2) triangle vertices -> area (n,), gradients g (n, 3, 2)."""
    d1, d2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    g1 = np.stack([d2[:, 1], -d2[:, 0]], axis=1) / det[:, None]
    g2 = np.stack([-d1[:, 1], d1[:, 0]], axis=1) / det[:, None]
    g0 = -g1 - g2
    return 0.5 * np.abs(det), np.stack([g0, g1, g2], axis=1)


def basis_gradients(lam, g):
    """Gradients (n, 6, 2) of the six P2 basis functions at barycentric point
    lam (3,), from the barycentric gradients g (n, 3, 2)."""
    out = [(4.0 * lam[i] - 1.0) * g[:, i] for i in range(3)]
    for i, j in ((0, 1), (1, 2), (0, 2)):
        out.append(4.0 * (lam[j] * g[:, i] + lam[i] * g[:, j]))
    return np.stack(out, axis=1)


def basis_values(lam):
    """Values (6,) of the P2 basis at barycentric point lam (3,)."""
    v = [lam[i] * (2.0 * lam[i] - 1.0) for i in range(3)]
    v += [4.0 * lam[i] * lam[j] for i, j in ((0, 1), (1, 2), (0, 2))]
    return np.array(v)


MIDPOINTS = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])


def element_stiffness(X, k=None):
    """(n, 6, 6) P2 element stiffness matrices of triangles X (n, 3, 2) by
    the edge-midpoint rule (exact for the degree-2 integrand)."""
    area, g = barycentric_gradients(np.asarray(X, dtype=np.float64))
    K = np.zeros((X.shape[0], 6, 6))
    for lam in MIDPOINTS:
        D = basis_gradients(lam, g)
        K += np.einsum("nad,nbd->nab", D, D)
    K *= (area / 3.0)[:, None, None]
    if k is not None:
        K *= np.asarray(k, dtype=np.float64)[:, None, None]
    return K


def element_mass(X):
    """(n, 6, 6) P2 element mass matrices by Radon's degree-5 rule (exact
    for the degree-4 integrand)."""
    area, _ = barycentric_gradients(np.asarray(X, dtype=np.float64))
    B, w = fem.radon7()
    Ml = sum(wq * np.outer(basis_values(lam), basis_values(lam)) for lam, wq in zip(B, w))
    return area[:, None, None] * Ml[None]


class P2Level:
    """P2 unknowns of level L of one macro mesh (numbered by the level-(L+1)
    lattice) with its level-L elements and the per-element coefficient."""

    def __init__(self, mesh: MacroMesh, L: int, k_elem=None):
        self.mesh, self.L = mesh, L
        self.lat = Level(mesh, L + 1)
        self.n, self.free, self.coords = self.lat.n, self.lat.free, self.lat.coords
        self.elements = p2_elements(self.lat, L)
        self.k = None if k_elem is None else np.asarray(k_elem, dtype=np.float64)
        self.X = self.coords[self.elements[:, :3]]

    def stiffness(self):
        return element_stiffness(self.X, self.k)


def assemble(p2: P2Level) -> sp.csr_matrix:
    """Brute-force assembled P2 stiffness over all unknowns (n x n)."""
    K = p2.stiffness()
    E = p2.elements
    rows = np.repeat(E, 6, axis=1).ravel()
    cols = np.tile(E, (1, 6)).ravel()
    A = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(p2.n, p2.n)).tocsr()
    A.sum_duplicates()
    return A


def apply_element_loop(p2: P2Level, x):
    """y = A x by a loop over the level-L micro-triangles, 0 at Dirichlet rows."""
    K = p2.stiffness()
    E = p2.elements
    ye = np.einsum("eab,eb->ea", K, np.asarray(x, dtype=np.float64)[E])
    y = np.bincount(E.ravel(), weights=ye.ravel(), minlength=p2.n)
    y[~p2.free] = 0.0
    return y


def load_vector(p2: P2Level, f):
    """b = M f_I (P2 mass matrix, f interpolated at the P2 nodes), 0 at
    Dirichlet rows."""
    fI = f(p2.coords[:, 0], p2.coords[:, 1])
    Me = element_mass(p2.X)
    E = p2.elements
    be = np.einsum("eab,eb->ea", Me, fI[E])
    b = np.bincount(E.ravel(), weights=be.ravel(), minlength=p2.n)
    b[~p2.free] = 0.0
    return b


def l2_error(p2: P2Level, uh, u_exact):
    """sqrt(sum_T integral_T (u_h - u)^2) with Radon's rule per element."""
    B, w = fem.radon7()
    area, _ = barycentric_gradients(p2.X)
    Phi = np.array([basis_values(lam) for lam in B])          # (7, 6)
    uq = np.einsum("qa,ea->eq", Phi, np.asarray(uh)[p2.elements])
    P = np.einsum("qk,ekd->eqd", B, p2.X)
    err = (uq - u_exact(P[..., 0], P[..., 1])) ** 2
    return float(np.sqrt(np.sum(area[:, None] * w[None, :] * err)))


# ------------------------------------------------------------------ smoother
def adjacency(p2: P2Level) -> sp.csr_matrix:
    """Structural adjacency: p, q adjacent when one level-L triangle holds both."""
    E = p2.elements
    rows = np.repeat(E, 6, axis=1).ravel()
    cols = np.tile(E, (1, 6)).ravel()
    A = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(p2.n, p2.n)).tocsr()
    A.sum_duplicates()
    return A


def gs_sets(p2: P2Level, adj=None):
    """The colour sets of the forward sweep, in order (free unknowns only)."""
    lat = p2.lat
    adj = adjacency(p2) if adj is None else adj
    nv = p2.mesh.nv
    sets = [np.nonzero(p2.free[:nv])[0]]
    # macro-edge points: greedy colouring in canonical order
    e_ids = np.arange(lat.edge_off, lat.face_off)
    e_ids = e_ids[p2.free[e_ids]]
    colour = {}
    for p in e_ids:
        used = {colour[q] for q in adj.indices[adj.indptr[p]:adj.indptr[p + 1]] if q in colour and q != p}
        c = 0
        while c in used:
            c += 1
        colour[p] = c
    nc = max(colour.values()) + 1 if colour else 0
    for c in range(nc):
        sets.append(np.array([p for p in e_ids if colour[p] == c], dtype=np.int64))
    # face interiors: six classes by the lattice position
    cls = np.full(p2.n, -1)
    for G in lat.face_ids:
        Np = lat.N
        for j in range(1, Np - 1):
            for i in range(1, Np - j):
                g = G[j, i]
                if i % 2 == 0 and j % 2 == 0:
                    cls[g] = (i // 2 + 2 * (j // 2)) % 3
                elif j % 2 == 0:
                    cls[g] = 3
                elif i % 2 == 0:
                    cls[g] = 4
                else:
                    cls[g] = 5
    for c in range(6):
        sets.append(np.nonzero(cls == c)[0])
    return [s for s in sets if s.size]


class P2Hierarchy:
    """P2 on level L plus the P1 hierarchy 0..L of the same mesh (the
    coarse space of p-multigrid), both with the same level-L coefficient."""

    def __init__(self, mesh: MacroMesh, L: int, k_elem=None):
        self.p2 = P2Level(mesh, L, k_elem)
        self.H1 = Hierarchy(mesh, L, k_elem)
        self.L = L
        self.A = assemble(self.p2)
        self.diag = self.A.diagonal()
        self.P = prolongation(self.H1.levels[L], self.p2.lat)   # P1(L) -> P2(L)
        self._sets = None

    def sets(self):
        if self._sets is None:
            self._sets = [(s, self.A[s, :].tocsr()) for s in gs_sets(self.p2)]
        return self._sets

    def apply(self, x):
        y = self.A @ x
        y[~self.p2.free] = 0.0
        return y

    def residual(self, x, b):
        r = b - self.A @ x
        r[~self.p2.free] = 0.0
        return r

    def norm(self, v):
        return float(np.sqrt(np.sum(v[self.p2.free] ** 2)))


def gs_sweep(PH: P2Hierarchy, x, b, forward=True):
    """One colour-ordered P2 Gauss-Seidel sweep, in place."""
    order = PH.sets() if forward else PH.sets()[::-1]
    d = PH.diag
    for S, AS in order:
        off = AS @ x - d[S] * x[S]
        x[S] = (b[S] - off) / d[S]
    return x


def pmg_cycle(PH: P2Hierarchy, x, b, nu1=2, nu2=2, nu1c=3, nu2c=3):
    """One p-multigrid cycle (reading in the module docstring), in place."""
    for _ in range(nu1):
        gs_sweep(PH, x, b, True)
    r = PH.residual(x, b)
    bc = PH.P.T @ r
    xc = np.zeros(PH.H1.levels[PH.L].n)
    vcycle(PH.H1, PH.L, xc, bc, nu1c, nu2c)
    x += PH.P @ xc
    for _ in range(nu2):
        gs_sweep(PH, x, b, False)
    return x


def solve(PH: P2Hierarchy, x, b, nu1=2, nu2=2, tol=1e-10, max_iter=100):
    """p-multigrid cycles until ||b - A x|| <= tol ||b - A x0|| (free DoFs)."""
    hist = [PH.norm(PH.residual(x, b))]
    for _ in range(max_iter):
        if hist[-1] <= tol * hist[0]:
            break
        pmg_cycle(PH, x, b, nu1, nu2)
        hist.append(PH.norm(PH.residual(x, b)))
    return x, hist


def direct_solve(PH: P2Hierarchy, b, x_dirichlet=None):
    """The exact discrete solution (free rows solved densely or by CG for
    checks): x = x_dirichlet on Dirichlet DoFs, A_ff x_f = b_f - A_fd x_d."""
    n = PH.p2.n
    xd = np.zeros(n) if x_dirichlet is None else np.asarray(x_dirichlet, dtype=np.float64).copy()
    fr = PH.p2.free
    xd[fr] = 0.0
    rhs = b - PH.A @ xd
    idx = np.nonzero(fr)[0]
    Aff = PH.A[idx][:, idx].tocsc()
    from scipy.sparse.linalg import spsolve
    xd[idx] = spsolve(Aff, rhs[idx])
    return xd
