"""Macro-primitive graph, structured refinement and canonical numbering (oracle).

Paper Sec. 2.1: the input triangulation is a graph of macro-vertices,
macro-edges and macro-faces; a face has three edges and three vertices, an edge
one or two faces.  Sec. 3.1: every macro-face is refined by connecting edge
midpoints, so level l has N = 2^l intervals per macro-edge and N^2 congruent
micro-triangles per face.  Sec. 2.2: every unknown is owned by exactly one
primitive (the lowest-dimensional one it lies on); the others hold copies.

Canonical numbering of the level-l unknowns (the order in which vectors cross
between the oracle and the CUDA library):
  1. macro-vertices, in input order;
  2. each macro-edge, edges sorted by (min vertex id, max vertex id), its N-1
     interior points from the low-id end (t = 1..N-1);
  3. each macro-face, in input order, its interior points (i, j), i, j >= 1,
     i + j <= N - 1, row by row (j outer, i inner).
Face frame: x = v0 + (i/N)(v1 - v0) + (j/N)(v2 - v0) with (v0, v1, v2) the
face made counter-clockwise (v1 and v2 swapped if the input is clockwise).

Dirichlet DoFs: a macro-vertex flagged by the caller (default: every vertex on
the boundary); the interior points of a macro-edge that lies on the boundary
and whose two end vertices are both Dirichlet.
"""
from __future__ import annotations

import numpy as np


class MeshError(ValueError):
    pass


class MacroMesh:
    """Macro-vertices, macro-edges and macro-faces of a 2D triangulation."""

    def __init__(self, xy, tri, dirichlet_vertex=None):
        xy = np.asarray(xy, dtype=np.float64)
        tri = np.array(tri, dtype=np.int64, copy=True)
        if xy.ndim != 2 or xy.shape[1] != 2 or tri.ndim != 2 or tri.shape[1] != 3:
            raise MeshError("bad shapes")
        nv = xy.shape[0]
        if tri.size and (tri.min() < 0 or tri.max() >= nv):
            raise MeshError("vertex index out of range")
        for f in range(tri.shape[0]):
            a, b, c = xy[tri[f]]
            cross = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
            if cross == 0.0 or len(set(tri[f].tolist())) < 3:
                raise MeshError(f"degenerate face {f}")
            if cross < 0:
                tri[f, 1], tri[f, 2] = tri[f, 2], tri[f, 1]
        self.xy, self.tri, self.nv, self.nf = xy, tri, nv, tri.shape[0]
        faces_of = {}
        for f in range(self.nf):
            for (a, b) in ((0, 1), (1, 2), (0, 2)):
                va, vb = int(tri[f, a]), int(tri[f, b])
                faces_of.setdefault((min(va, vb), max(va, vb)), []).append(f)
        for e, fs in faces_of.items():
            if len(fs) > 2:
                raise MeshError(f"edge {e} shared by {len(fs)} faces")
        self.edges = sorted(faces_of)                      # (lo, hi) pairs
        self.edge_id = {e: k for k, e in enumerate(self.edges)}
        self.edge_faces = [faces_of[e] for e in self.edges]
        self.ne = len(self.edges)
        bnd_edge = np.array([len(fs) == 1 for fs in self.edge_faces], dtype=bool)
        on_bnd = np.zeros(nv, dtype=bool)
        for k, (a, b) in enumerate(self.edges):
            if bnd_edge[k]:
                on_bnd[a] = on_bnd[b] = True
        if dirichlet_vertex is None:
            dv = on_bnd.copy()
        else:
            dv = np.asarray(dirichlet_vertex).astype(bool).copy()
            if dv.shape != (nv,):
                raise MeshError("dirichlet mask has wrong length")
        self.dirichlet_vertex = dv
        self.boundary_edge = bnd_edge
        self.dirichlet_edge = np.array(
            [bnd_edge[k] and dv[a] and dv[b] for k, (a, b) in enumerate(self.edges)], dtype=bool)


def closed_points(N):
    """All (i, j) of the closed face lattice, i, j >= 0, i + j <= N."""
    return [(i, j) for j in range(N + 1) for i in range(N + 1 - j)]


class Level:
    """Unknowns of one refinement level with their canonical ids.

    Attributes
      N          intervals per macro-edge
      n          number of unknowns (all vertices, edge and face interiors)
      coords     (n, 2) owner coordinates of every unknown
      free       (n,) bool, False at Dirichlet unknowns
      face_ids   list over faces of an (N+1, N+1) int array G[j, i] giving the
                 canonical id of lattice point (i, j) (-1 where i + j > N)
      elements   (n_faces * N^2, 3) canonical ids of the micro-triangles in
                 canonical element order (per face: upward (i,j),(i+1,j),(i,j+1)
                 row by row, then downward (i+1,j),(i,j+1),(i+1,j+1) row by row)
      kind       (n,) 0 vertex, 1 edge interior, 2 face interior
    """

    def __init__(self, mesh: MacroMesh, level: int):
        self.mesh, self.level = mesh, level
        N = 1 << level
        self.N = N
        nv, ne, nf = mesh.nv, mesh.ne, mesh.nf
        n_e_int = max(N - 1, 0)
        n_f_int = (N - 1) * (N - 2) // 2 if N >= 3 else 0
        self.edge_off = nv
        self.face_off = nv + ne * n_e_int
        self.n = self.face_off + nf * n_f_int
        self.n_e_int, self.n_f_int = n_e_int, n_f_int
        xy = mesh.xy
        coords = np.zeros((self.n, 2))
        kind = np.zeros(self.n, dtype=np.int8)
        free = np.ones(self.n, dtype=bool)
        coords[:nv] = xy
        free[:nv] = ~mesh.dirichlet_vertex
        t = np.arange(1, N, dtype=np.float64)
        for k, (a, b) in enumerate(mesh.edges):
            g = nv + k * n_e_int + np.arange(n_e_int)
            coords[g] = xy[a][None, :] + (t / N)[:, None] * (xy[b] - xy[a])[None, :]
            kind[g] = 1
            free[g] = not mesh.dirichlet_edge[k]
        # interior lattice points in row-major order (j outer, i inner)
        jj = np.concatenate([np.full(N - 1 - j, j) for j in range(1, N - 1)]).astype(np.int64) if N >= 3 else np.zeros(0, np.int64)
        ii = np.concatenate([np.arange(1, N - j) for j in range(1, N - 1)]).astype(np.int64) if N >= 3 else np.zeros(0, np.int64)
        p = np.arange(1, N)
        self.face_ids = []
        for f in range(nf):
            v0, v1, v2 = (int(v) for v in mesh.tri[f])
            G = -np.ones((N + 1, N + 1), dtype=np.int64)
            base = self.face_off + f * n_f_int
            g = base + np.arange(n_f_int)
            G[jj, ii] = g
            coords[g] = (xy[v0][None, :] + (ii / N)[:, None] * (xy[v1] - xy[v0])[None, :]
                         + (jj / N)[:, None] * (xy[v2] - xy[v0])[None, :])
            kind[g] = 2
            G[0, 0], G[0, N], G[N, 0] = v0, v1, v2
            if N >= 2:
                G[0, p] = self._edge_point(v0, v1, p)          # side j = 0, v0 -> v1
                G[p, N - p] = self._edge_point(v1, v2, p)      # side i + j = N, v1 -> v2
                G[p, 0] = self._edge_point(v0, v2, p)          # side i = 0, v0 -> v2
            self.face_ids.append(G)
        self.coords, self.kind, self.free = coords, kind, free
        ju = np.concatenate([np.full(N - j, j) for j in range(N)]).astype(np.int64)
        iu = np.concatenate([np.arange(N - j) for j in range(N)]).astype(np.int64)
        if N >= 2:
            jd = np.concatenate([np.full(N - 1 - j, j) for j in range(N - 1)]).astype(np.int64)
            id_ = np.concatenate([np.arange(N - 1 - j) for j in range(N - 1)]).astype(np.int64)
        else:
            jd = id_ = np.zeros(0, np.int64)
        els = []
        for G in self.face_ids:
            up = np.stack([G[ju, iu], G[ju, iu + 1], G[ju + 1, iu]], axis=1)
            dn = np.stack([G[jd, id_ + 1], G[jd + 1, id_], G[jd + 1, id_ + 1]], axis=1)
            els.append(up)
            els.append(dn)
        self.elements = np.concatenate(els, axis=0)

    def _edge_point(self, va, vb, p):
        """Canonical id of the point at distance p (in lattice steps) from va
        on the macro-edge {va, vb}."""
        m = self.mesh
        k = m.edge_id[(min(va, vb), max(va, vb))]
        t = p if va < vb else self.N - p
        return self.edge_off + k * self.n_e_int + (t - 1)

    def face_point_coords(self, f, i, j):
        """Coordinates of lattice point (i, j) computed in face f's frame."""
        v0, v1, v2 = self.mesh.xy[self.mesh.tri[f]]
        N = self.N
        return v0 + (i / N) * (v1 - v0) + (j / N) * (v2 - v0)
