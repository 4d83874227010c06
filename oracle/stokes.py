"""Stokes flow with equal-order P1-P1 elements, PSPG pressure stabilisation,
and the all-at-once multigrid with a pointwise inexact Uzawa smoother
(oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 5.2 (isoviscous incompressible Stokes, velocity and pressure by
equal-order P1-P1 elements with a Petrov-Galerkin pressure stabilisation
(PSPG, Brezzi and Pitkaranta), homogeneous Dirichlet velocity, solved
monolithically by multigrid); Sec. 4.3 (an all-at-once multigrid with
pointwise inexact Uzawa smoothers for saddle-point problems).  The paper
gives neither the stabilisation parameter nor the smoother's steps; the
readings taken here:

  Discrete system (u = (u1, u2) velocity, p pressure, all P1 on level l):

      [ A    0    B1^T ] [u1]   [f1]
      [ 0    A    B2^T ] [u2] = [f2]
      [ B1   B2   -C   ] [p ]   [g ]

  A_ij   = integral grad(phi_i).grad(phi_j)                (the P1 Laplacian)
  Bd_qj  = - integral phi_q d(phi_j)/dx_d                  (d = 1, 2)
  C_qr   = delta * sum_T h_T^2 integral_T grad(phi_q).grad(phi_r)
           (h_T = longest edge of micro-triangle T; the PSPG term of the
           continuity equation for P1, where the element Laplacian of the
           velocity vanishes)

  Velocity rows of Dirichlet unknowns are dropped (their values are data);
  B acts on the full velocity vector, B^T is evaluated on free velocity
  rows only.  Every pressure unknown is free.  With velocity Dirichlet
  conditions on the whole boundary the constant pressure spans the null
  space; g must then sum to zero, and the solutions taken are those whose
  pressure sums to zero where the system is solved directly (level 0 and
  the reference solve).

  Uzawa smoothing step (forward):
      u_d <- nvel colour-ordered Gauss-Seidel sweeps on A u_d = f_d - Bd^T p
      p   <- p + omega * (B1 u1 + B2 u2 - C p - g) / s
  with s = diag(C) + sum_d (Bd o Bd) (D_A^-1 on free velocity), the diagonal of
  C + B D_A^-1 B^T (a Jacobi step on the Schur complement of the system with
  A replaced by its diagonal).  The backward step takes the same parts in
  the opposite order (pressure first, then backward velocity sweeps).

  Cycle: a variable V-cycle -- nu1 + growth (top - l) forward steps on level
  l of a cycle started on level top, residual, restriction by the transposed
  P1 prolongation (velocity: free rows and columns only; pressure: every
  unknown), the coarse cycle from zero, prolongation and correction, nu2 +
  growth (top - l) backward steps.  (With the same steps on every level the
  cycle's factor grows with the number of levels -- about 0.58, 0.67, 0.95
  and 1.2 on levels 6 to 9 of the unit square -- while two more steps per
  coarser level keep it near 0.49 on every level.)  On the coarsest level of the cycle (level 0 or a finer
  one, `coarse`: a macro mesh whose vertices nearly all lie on the Dirichlet
  boundary leaves level 0 almost no velocity unknowns) the correction is a
  direct solve of the saddle-point system for the residual.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import fem
from . import multigrid as mg
from .mesh import Level, MacroMesh


def div_matrices(level: Level):
    """(B1, B2) over ALL unknowns (n x n): Bd_qj = -integral phi_q dphi_j/dx_d
    = -(|T| / 3) G_T[d, j] summed over the micro-triangles T (the integral of
    a hat function over T is |T| / 3, its gradient G_T is constant there)."""
    area, G = fem.element_geometry(level)
    E = level.elements
    rows = np.repeat(E, 3, axis=1).ravel()       # test (pressure) vertex
    cols = np.tile(E, (1, 3)).ravel()            # trial (velocity) vertex
    out = []
    for d in range(2):
        val = -(area / 3.0)[:, None, None] * np.broadcast_to(G[:, d, None, :], (E.shape[0], 3, 3))
        B = sp.coo_matrix((val.ravel(), (rows, cols)), shape=(level.n, level.n)).tocsr()
        B.sum_duplicates()
        out.append(B)
    return out


def longest_edge_sq(level: Level):
    """h_T^2 per micro-triangle: the squared longest edge."""
    X = level.coords[level.elements]
    e = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 1], X[:, 0] - X[:, 2]], axis=1)
    return (e ** 2).sum(axis=-1).max(axis=-1)


def stabilisation(level: Level, delta: float):
    """C = delta * sum_T h_T^2 * (P1 stiffness of T)."""
    return fem.assemble(level, delta * longest_edge_sq(level))


def pressure_prolongation(mesh: MacroMesh, coarse: Level, fine: Level):
    """P1 prolongation from ``coarse`` to ``fine`` over every unknown (the
    pressure has no Dirichlet rows): the prolongation of the same mesh with
    no Dirichlet vertex."""
    free_mesh = MacroMesh(mesh.xy, mesh.tri, dirichlet_vertex=np.zeros(mesh.nv, dtype=bool))
    return mg.prolongation(Level(free_mesh, coarse.level), Level(free_mesh, fine.level))


class StokesHierarchy:
    """Levels 0..L of the P1-P1 PSPG Stokes system on one macro mesh."""

    def __init__(self, mesh: MacroMesh, L: int, delta: float = 0.3, omega: float = 0.4, nvel: int = 2,
                 coarse: int = 0, growth: int = 2):
        self.mesh, self.L = mesh, L
        self.delta, self.omega, self.nvel, self.coarse, self.growth = delta, omega, nvel, coarse, growth
        self.H = mg.Hierarchy(mesh, L)            # velocity: A, Gauss-Seidel sets, prolongation
        self.levels = self.H.levels
        self.B = [div_matrices(lv) for lv in self.levels]
        self.C = [stabilisation(lv, delta) for lv in self.levels]
        self.s = []
        for l, lv in enumerate(self.levels):
            dinv = np.where(lv.free, 1.0 / self.H.diag[l], 0.0)
            B1, B2 = self.B[l]
            self.s.append(self.C[l].diagonal() + B1.multiply(B1) @ dinv + B2.multiply(B2) @ dinv)
        self._Pp = {}

    def Pp(self, l):
        if l not in self._Pp:
            self._Pp[l] = pressure_prolongation(self.mesh, self.levels[l - 1], self.levels[l])
        return self._Pp[l]

    # ------------------------------------------------------------ operator
    def grad_rows(self, l, p):
        """(B1^T p, B2^T p) on free velocity rows (0 at Dirichlet rows)."""
        fr = self.levels[l].free
        out = []
        for B in self.B[l]:
            y = B.T @ p
            y[~fr] = 0.0
            out.append(y)
        return out

    def apply(self, l, u1, u2, p):
        """The system matrix times (u1, u2, p)."""
        g1, g2 = self.grad_rows(l, p)
        B1, B2 = self.B[l]
        return (self.H.apply(l, u1) + g1, self.H.apply(l, u2) + g2, B1 @ u1 + B2 @ u2 - self.C[l] @ p)

    def residual(self, l, u1, u2, p, f1, f2, g):
        y1, y2, yp = self.apply(l, u1, u2, p)
        fr = self.levels[l].free
        r1, r2 = f1 - y1, f2 - y2
        r1[~fr] = 0.0
        r2[~fr] = 0.0
        return r1, r2, g - yp

    def norm(self, l, r1, r2, rp):
        fr = self.levels[l].free
        return float(np.sqrt(np.sum(r1[fr] ** 2) + np.sum(r2[fr] ** 2) + np.sum(rp ** 2)))

    # ------------------------------------------------------------ smoother
    def uzawa_step(self, l, u1, u2, p, f1, f2, g, forward=True):
        """One inexact Uzawa step in place (forward or backward order)."""
        def velocity():
            g1, g2 = self.grad_rows(l, p)
            for u, f, gd in ((u1, f1, g1), (u2, f2, g2)):
                b = f - gd
                for _ in range(self.nvel):
                    mg.gs_sweep(self.H, l, u, b, forward)

        def pressure():
            B1, B2 = self.B[l]
            p[:] = p + self.omega * (B1 @ u1 + B2 @ u2 - self.C[l] @ p - g) / self.s[l]

        if forward:
            velocity()
            pressure()
        else:
            pressure()
            velocity()

    # ------------------------------------------------------------- cycles
    def coarse_solve(self, f1, f2, g, level=0):
        """The saddle-point system of ``level`` on free velocity and every
        pressure unknown, solved densely; the least-squares minimum-norm
        solution (pressure summing to zero when constants are in the null
        space)."""
        lv = self.levels[level]
        A = self.H.A[level].toarray()
        B1, B2 = (B.toarray() for B in self.B[level])
        C = self.C[level].toarray()
        fr = np.nonzero(lv.free)[0]
        n, m = fr.size, lv.n
        K = np.zeros((2 * n + m, 2 * n + m))
        K[:n, :n] = A[np.ix_(fr, fr)]
        K[n:2 * n, n:2 * n] = A[np.ix_(fr, fr)]
        K[:n, 2 * n:] = B1[:, fr].T
        K[n:2 * n, 2 * n:] = B2[:, fr].T
        K[2 * n:, :n] = B1[:, fr]
        K[2 * n:, n:2 * n] = B2[:, fr]
        K[2 * n:, 2 * n:] = -C
        rhs = np.concatenate([f1[fr], f2[fr], g])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
        u1, u2 = np.zeros(m), np.zeros(m)
        u1[fr], u2[fr] = sol[:n], sol[n:2 * n]
        return u1, u2, sol[2 * n:].copy()

    def vcycle(self, l, u1, u2, p, f1, f2, g, nu1=2, nu2=2, top=None):
        top = l if top is None else top
        if l <= self.coarse:
            c1, c2, cp = self.coarse_solve(*self.residual(l, u1, u2, p, f1, f2, g), level=l)
            u1 += c1
            u2 += c2
            p += cp
            return
        extra = self.growth * (top - l)
        for _ in range(nu1 + extra):
            self.uzawa_step(l, u1, u2, p, f1, f2, g, True)
        r1, r2, rp = self.residual(l, u1, u2, p, f1, f2, g)
        P, Pp = self.H.P(l), self.Pp(l)
        m = self.levels[l - 1].n
        c1, c2, cp = np.zeros(m), np.zeros(m), np.zeros(m)
        self.vcycle(l - 1, c1, c2, cp, P.T @ r1, P.T @ r2, Pp.T @ rp, nu1, nu2, top)
        u1 += P @ c1
        u2 += P @ c2
        p += Pp @ cp
        for _ in range(nu2 + extra):
            self.uzawa_step(l, u1, u2, p, f1, f2, g, False)

    def solve(self, u1, u2, p, f1, f2, g, nu1=2, nu2=2, tol=1e-8, max_iter=100, level=None):
        """V-cycles until ||r|| <= tol ||r0|| (norm over free velocity rows and
        every pressure row).  Returns the residual-norm history."""
        L = self.L if level is None else level
        hist = [self.norm(L, *self.residual(L, u1, u2, p, f1, f2, g))]
        for _ in range(max_iter):
            if hist[-1] <= tol * hist[0]:
                break
            self.vcycle(L, u1, u2, p, f1, f2, g, nu1, nu2)
            hist.append(self.norm(L, *self.residual(L, u1, u2, p, f1, f2, g)))
        return hist

    def direct_solve(self, f1, f2, g, level=None):
        """Sparse direct solve of the level's system; with the constant
        pressure in the null space the pressure is fixed by a zero-sum
        constraint (a bordered system).  Reference for pins only."""
        l = self.L if level is None else level
        lv = self.levels[l]
        fr = np.nonzero(lv.free)[0]
        n, m = fr.size, lv.n
        A = self.H.A[l][fr][:, fr]
        B1, B2 = (B[:, fr] for B in self.B[l])
        one = sp.csr_matrix(np.ones((1, m)))
        K = sp.bmat([[A, None, B1.T, None], [None, A, B2.T, None], [B1, B2, -self.C[l], one.T],
                     [None, None, one, None]], format="csc")
        sol = sla.spsolve(K, np.concatenate([f1[fr], f2[fr], g, [0.0]]))
        u1, u2 = np.zeros(m), np.zeros(m)
        u1[fr], u2[fr] = sol[:n], sol[n:2 * n]
        return u1, u2, sol[2 * n:2 * n + m]
