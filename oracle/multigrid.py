"""Geometric multigrid on the HHG level hierarchy (oracle).

Paper Sec. 4.3: multigrid as solver (or Krylov preconditioner); interpolation
and restriction are non-square matrix-vector products; the smoothers are
point-wise and need the diagonal of A; multi-colour Gauss-Seidel is named in
Sec. 3.2.  The paper fixes none of the details below; the oracle takes these
readings (each one a plain definition or a textbook algorithm):

* Gauss-Seidel order (forward sweep): the free macro-vertex DoFs; then the
  free edge-interior DoFs colour by colour, where each edge DoF, visited in
  canonical order, takes the smallest colour not held by an already coloured
  edge DoF that shares a micro-edge with it; then the face-interior DoFs with
  (i + 2j) mod 3 = 0, 1, 2.  Every set is independent (no micro-edge inside
  a set), so updating a set at once equals updating its points one after
  another.  The backward sweep is the exact reverse order.  Point update:
  x_p <- (b_p - sum_{q != p} A_pq x_q) / A_pp.
* Damped Jacobi: x <- x + omega D^-1 (b - A x), omega = 2/3 by default.
* Prolongation: P_pq = phi^c_q(x_p), the coarse hat function of coarse DoF q
  evaluated at fine DoF p (linear interpolation between nested P1 spaces).
  Restriction: R = P^T.  Rows of Dirichlet DoFs are zero on both sides.
* Coarse operator: rediscretisation on the coarse mesh; a coarse element's
  coefficient is the mean of its four children.
* V(nu1, nu2): nu1 forward sweeps, residual, restriction, zero coarse guess,
  recursion, prolongation and correction, nu2 backward sweeps; on level 0
  plain conjugate gradients to 1e-14 relative residual or 2 n0 iterations.
* Solver: x0 = 0 on free DoFs (Dirichlet values kept), V-cycles until
  ||b - A x||_2 <= tol ||b - A x0||_2 over free DoFs, at most max_iter cycles.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Level, MacroMesh
from . import fem


# ----------------------------------------------------------------- colouring
def adjacency(level: Level) -> sp.csr_matrix:
    """Boolean adjacency of unknowns sharing a micro-edge (structure only)."""
    E = level.elements
    r = np.concatenate([E[:, 0], E[:, 1], E[:, 2], E[:, 1], E[:, 2], E[:, 0]])
    c = np.concatenate([E[:, 1], E[:, 2], E[:, 0], E[:, 0], E[:, 1], E[:, 2]])
    A = sp.coo_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(level.n, level.n)).tocsr()
    A.sum_duplicates()
    return A


def edge_colours(level: Level, adj=None) -> np.ndarray:
    """Greedy colouring of the free edge-interior DoFs in canonical order:
    colour(p) = smallest c >= 0 not taken by an already coloured neighbour.
    Returns (n,) int array, -1 where not an edge DoF or not free."""
    if adj is None:
        adj = adjacency(level)
    col = -np.ones(level.n, dtype=np.int64)
    ids = np.nonzero((level.kind == 1) & level.free)[0]
    indptr, indices = adj.indptr, adj.indices
    for p in ids:
        taken = {col[q] for q in indices[indptr[p]:indptr[p + 1]] if col[q] >= 0}
        c = 0
        while c in taken:
            c += 1
        col[p] = c
    return col


def face_colours(level: Level) -> np.ndarray:
    """(i + 2j) mod 3 for face-interior DoFs in the face frame, -1 elsewhere."""
    col = -np.ones(level.n, dtype=np.int64)
    N = level.N
    if N < 3:
        return col
    jj = np.concatenate([np.full(N - 1 - j, j) for j in range(1, N - 1)])
    ii = np.concatenate([np.arange(1, N - j) for j in range(1, N - 1)])
    for G in level.face_ids:
        col[G[jj, ii]] = (ii + 2 * jj) % 3
    return col


def gs_sets(level: Level):
    """The forward Gauss-Seidel order as a list of index arrays."""
    sets = [np.nonzero((level.kind == 0) & level.free)[0]]
    ec = edge_colours(level)
    for c in range(int(ec.max()) + 1 if (ec >= 0).any() else 0):
        sets.append(np.nonzero(ec == c)[0])
    fc = face_colours(level)
    for c in range(3):
        sets.append(np.nonzero(fc == c)[0])
    return [s for s in sets if s.size]


# -------------------------------------------------------------- hierarchy
class Hierarchy:
    """Levels 0..L of one macro mesh with the assembled operators used by the
    oracle's smoother (rows of the brute-force CSR matrix)."""

    def __init__(self, mesh: MacroMesh, L: int, k_elem_fine=None):
        self.mesh, self.L = mesh, L
        self.levels = [Level(mesh, l) for l in range(L + 1)]
        self.k = [None] * (L + 1)
        if k_elem_fine is not None:
            self.k[L] = np.asarray(k_elem_fine, dtype=np.float64)
            for l in range(L, 0, -1):
                self.k[l - 1] = coarsen_coefficient(self.levels[l - 1], self.k[l], mesh.nf)
        self.A = [fem.assemble(lv, self.k[l]) for l, lv in enumerate(self.levels)]
        self.diag = [A.diagonal() for A in self.A]
        self._sets = {}
        self._P = {}

    def sets(self, l):
        if l not in self._sets:
            S = gs_sets(self.levels[l])
            self._sets[l] = [(s, self.A[l][s, :].tocsr()) for s in S]
        return self._sets[l]

    def P(self, l):
        """Prolongation from level l-1 to level l."""
        if l not in self._P:
            self._P[l] = prolongation(self.levels[l - 1], self.levels[l])
        return self._P[l]

    def apply(self, l, x):
        y = self.A[l] @ x
        y[~self.levels[l].free] = 0.0
        return y

    def residual(self, l, x, b):
        r = b - self.A[l] @ x
        r[~self.levels[l].free] = 0.0
        return r


def coarsen_coefficient(coarse: Level, k_fine, nf):
    """Coarse element value = mean of its four children (index form of the
    refinement: coarse up (I,J) -> fine up (2I,2J), (2I+1,2J), (2I,2J+1) and
    down (2I,2J); coarse down (I,J) -> fine down (2I+1,2J), (2I,2J+1),
    (2I+1,2J+1) and up (2I+1,2J+1))."""
    Nc = coarse.N
    Nf = 2 * Nc
    k_fine = np.asarray(k_fine).reshape(nf, Nf * Nf)

    def up_index(N, i, j):    # row-major index of up (i,j) within a face
        return j * N - j * (j - 1) // 2 + i

    def dn_index(N, i, j):
        return N * (N + 1) // 2 + j * (N - 1) - j * (j - 1) // 2 + i
    out = np.zeros((nf, Nc * Nc))
    J = np.concatenate([np.full(Nc - j, j) for j in range(Nc)])
    I = np.concatenate([np.arange(Nc - j) for j in range(Nc)])
    ch = [up_index(Nf, 2 * I, 2 * J), up_index(Nf, 2 * I + 1, 2 * J),
          up_index(Nf, 2 * I, 2 * J + 1), dn_index(Nf, 2 * I, 2 * J)]
    out[:, up_index(Nc, I, J)] = sum(k_fine[:, c] for c in ch) / 4.0
    if Nc >= 2:
        J = np.concatenate([np.full(Nc - 1 - j, j) for j in range(Nc - 1)])
        I = np.concatenate([np.arange(Nc - 1 - j) for j in range(Nc - 1)])
        ch = [dn_index(Nf, 2 * I + 1, 2 * J), dn_index(Nf, 2 * I, 2 * J + 1),
              dn_index(Nf, 2 * I + 1, 2 * J + 1), up_index(Nf, 2 * I + 1, 2 * J + 1)]
        out[:, dn_index(Nc, I, J)] = sum(k_fine[:, c] for c in ch) / 4.0
    return out.ravel()


def prolongation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """P_pq = phi^c_q(x_p): every fine DoF on the closure of a coarse
    micro-triangle gets the barycentric coordinates of its position in that
    triangle (computed from coordinates, then set to the exact value 0, 1/2
    or 1 that nested refinement gives -- a check fails if one is off by more
    than 1e-9).  Rows of fine Dirichlet DoFs and
    columns of coarse Dirichlet DoFs are zeroed."""
    Nc = coarse.N
    C = coarse.coords[coarse.elements]                            # (n_el_c, 3, 2)
    # fine lattice points on the closure of every coarse element, in the
    # coarse element order (per face: up row by row, then down row by row)
    J = np.concatenate([np.full(Nc - j, j) for j in range(Nc)])
    I = np.concatenate([np.arange(Nc - j) for j in range(Nc)])
    up_a, up_b = 2 * I, 2 * J                  # up: corners (a,b),(a+2,b),(a,b+2)
    up_off = ((0, 0), (2, 0), (0, 2), (1, 0), (1, 1), (0, 1))
    if Nc >= 2:
        J = np.concatenate([np.full(Nc - 1 - j, j) for j in range(Nc - 1)])
        I = np.concatenate([np.arange(Nc - 1 - j) for j in range(Nc - 1)])
    else:
        I = J = np.zeros(0, dtype=np.int64)
    dn_a, dn_b = 2 * I + 1, 2 * J + 1          # down centred at (a,b)
    dn_off = ((1, -1), (-1, 1), (1, 1), (0, 0), (1, 0), (0, 1))
    F = []
    for Gf in fine.face_ids:
        F.append(np.stack([Gf[up_b + db, up_a + da] for (da, db) in up_off], axis=1))
        if dn_a.size:
            F.append(np.stack([Gf[dn_b + db, dn_a + da] for (da, db) in dn_off], axis=1))
    F = np.concatenate(F, axis=0).astype(np.int64)                # (n_el_c, 6)
    X = fine.coords[F]                                            # (n_el_c, 6, 2)
    a, b, c = C[:, 0], C[:, 1], C[:, 2]
    D = np.stack([b - a, c - a], axis=2)                          # (n, 2, 2)
    rhs = X - a[:, None, :]                                       # (n, 6, 2)
    lam = np.linalg.solve(D[:, None, :, :], rhs[..., None])[..., 0]  # (n, 6, 2) = (lam_b, lam_c)
    bary = np.concatenate([1.0 - lam.sum(axis=2, keepdims=True), lam], axis=2)  # (n, 6, 3)
    # nested spaces: every value is 0, 1/2 or 1; anything else means a fine
    # point outside its coarse triangle
    snapped = np.round(2.0 * bary) / 2.0
    if np.max(np.abs(bary - snapped)) > 1e-9:
        raise AssertionError("fine lattice point off the coarse element")
    bary = snapped
    E = coarse.elements
    p = np.broadcast_to(F[:, :, None], bary.shape).ravel()
    q = np.broadcast_to(E[:, None, :], bary.shape).ravel()
    w = bary.ravel()
    keep = np.abs(w) > 1e-12
    p, q, w = p[keep], q[keep], w[keep]
    _, first = np.unique(p * coarse.n + q, return_index=True)
    p, q, w = p[first], q[first], w[first]
    keep = fine.free[p] & coarse.free[q]
    return sp.coo_matrix((w[keep], (p[keep], q[keep])), shape=(fine.n, coarse.n)).tocsr()


# ---------------------------------------------------------------- smoothers
def gs_sweep(H: Hierarchy, l, x, b, forward=True):
    """One colour-ordered Gauss-Seidel sweep, in place."""
    sets = H.sets(l)
    d = H.diag[l]
    order = sets if forward else sets[::-1]
    for S, AS in order:
        off = AS @ x - d[S] * x[S]
        x[S] = (b[S] - off) / d[S]
    return x


def jacobi_sweep(H: Hierarchy, l, x, b, omega=2.0 / 3.0):
    r = H.residual(l, x, b)
    fr = H.levels[l].free
    x[fr] += omega * r[fr] / H.diag[l][fr]
    return x


def sequential_gs(A: sp.csr_matrix, order, x, b):
    """Point Gauss-Seidel visiting the DoFs of ``order`` one by one (pure
    Python; tiny meshes only)."""
    A = A.tocsr()
    for p in order:
        s, dpp = 0.0, 0.0
        for k in range(A.indptr[p], A.indptr[p + 1]):
            q = A.indices[k]
            if q == p:
                dpp = A.data[k]
            else:
                s += A.data[k] * x[q]
        x[p] = (b[p] - s) / dpp
    return x


# --------------------------------------------------------------- coarse CG
def cg(A: sp.csr_matrix, free, b, tol=1e-14, maxit=None):
    """Plain conjugate gradients on the free DoFs (x0 = 0)."""
    idx = np.nonzero(free)[0]
    Af = A[idx][:, idx].tocsr()
    bf = b[idx]
    n0 = idx.size
    maxit = 2 * n0 if maxit is None else maxit
    x = np.zeros(n0)
    r = bf.copy()
    p = r.copy()
    rr = r @ r
    stop = (tol * np.sqrt(bf @ bf)) ** 2
    it = 0
    while rr > stop and it < maxit:
        Ap = Af @ p
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    out = np.zeros_like(b)
    out[idx] = x
    return out


# ----------------------------------------------------------------- V-cycle
def restrict(H: Hierarchy, l, r):
    """b_{l-1} = P^T r (fine Dirichlet rows of r are 0; coarse Dirichlet = 0)."""
    return H.P(l).T @ r


def prolongate_add(H: Hierarchy, l, x, xc):
    x += H.P(l) @ xc
    return x


def vcycle(H: Hierarchy, l, x, b, nu1=2, nu2=2):
    if l == 0:
        lv = H.levels[0]
        x[lv.free] = cg(H.A[0], lv.free, b)[lv.free]
        return x
    for _ in range(nu1):
        gs_sweep(H, l, x, b, True)
    r = H.residual(l, x, b)
    bc = restrict(H, l, r)
    xc = np.zeros(H.levels[l - 1].n)
    vcycle(H, l - 1, xc, bc, nu1, nu2)
    prolongate_add(H, l, x, xc)
    for _ in range(nu2):
        gs_sweep(H, l, x, b, False)
    return x


def norm_free(H: Hierarchy, l, v):
    return float(np.sqrt(np.sum(v[H.levels[l].free] ** 2)))


def solve(H: Hierarchy, x, b, nu1=2, nu2=2, tol=1e-10, max_iter=100, level=None):
    """V-cycles on ``level`` (default: finest) until ||r|| <= tol ||r0||.
    Returns (x, residual-norm history)."""
    L = H.L if level is None else level
    hist = [norm_free(H, L, H.residual(L, x, b))]
    for _ in range(max_iter):
        if hist[-1] <= tol * hist[0]:
            break
        vcycle(H, L, x, b, nu1, nu2)
        hist.append(norm_free(H, L, H.residual(L, x, b)))
    return x, hist
