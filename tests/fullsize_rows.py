"""Single rows of the P1 operator, for checking GPU results on sampled
points of levels too large for the oracle's whole-level arrays.

The row of a face-interior lattice point p = (i, j) of face f is built from
the oracle's own element matrices (Sec. 4.2: A_pq = sum over the
micro-triangles T of k_T * integral_T grad(phi_p).grad(phi_q)) on the six
micro-triangles around p, all inside face f, translated so that p is at the
origin (the matrices do not change under translation).  Lattice point (a, b) of face f
sits at v0 + (a/N)(v1 - v0) + (b/N)(v2 - v0), (v0, v1, v2) the face's
counter-clockwise vertices; upward triangle (a, b) has the vertices
(a, b), (a+1, b), (a, b+1), downward triangle (a, b) the vertices
(a+1, b), (a, b+1), (a+1, b+1), each numbered row by row within its face
(the canonical element order).
"""
from types import SimpleNamespace

import numpy as np

from oracle import fem

# the seven stencil points as offsets from p; local id = position here
NEIGH = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]
# the six micro-triangles containing p: (kind, origin offset)
PATCH = [("up", 0, 0), ("up", -1, 0), ("up", 0, -1), ("dn", -1, 0), ("dn", 0, -1), ("dn", -1, -1)]


def tri_vertices(kind, a, b):
    if kind == "up":
        return [(a, b), (a + 1, b), (a, b + 1)]
    return [(a + 1, b), (a, b + 1), (a + 1, b + 1)]


def element_index(N, kind, a, b):
    """Position of a micro-triangle within its face in the canonical element
    order (all upward triangles row by row, then all downward ones)."""
    if kind == "up":
        return b * N - b * (b - 1) // 2 + a
    return N * (N + 1) // 2 + b * (N - 1) - b * (b - 1) // 2 + a


def row_weights(xy, tri, N, f, i, j, k_patch=None):
    """w (7,) with (A x)_p = sum_m w[m] x[p + NEIGH[m]]; k_patch: the six
    coefficients in PATCH order (None: k = 1)."""
    v0, v1, v2 = (np.asarray(xy[v], dtype=np.float64) for v in tri[f])
    pts = [(i + di, j + dj) for di, dj in NEIGH]
    local = {pt: m for m, pt in enumerate(pts)}
    # the element matrices depend on coordinate differences only: the patch
    # is placed relative to p, so that its edge vectors are (v1 - v0) / N and
    # (v2 - v0) / N to rounding (absolute coordinates would lose about
    # log2(N) bits of them to cancellation)
    coords = np.array([((a - i) / N) * (v1 - v0) + ((b - j) / N) * (v2 - v0) for a, b in pts])
    elems = np.array([[local[v] for v in tri_vertices(kind, i + da, j + db)] for kind, da, db in PATCH])
    k = np.ones(6) if k_patch is None else np.asarray(k_patch, dtype=np.float64)
    K = fem.element_stiffness(SimpleNamespace(coords=coords, elements=elems), k)
    w = np.zeros(7)
    for e in range(6):
        a_loc = int(np.where(elems[e] == 0)[0][0])
        for bpos in range(3):
            w[elems[e, bpos]] += K[e, a_loc, bpos]
    return w


def patch_element_ids(N, f, i, j):
    """Canonical element ids (6,) of the PATCH triangles of point (i, j) of face f."""
    return np.array([f * N * N + element_index(N, kind, i + da, j + db) for kind, da, db in PATCH])


# ------------------------------------------------------------------ P2
# P2 on level L: lattice point (I, J) of level L + 1; the level-L triangles
# holding it and their six nodes (v0, v1, v2, m01, m12, m02) relative to the
# triangle origin (2a, 2b), in the order of oracle.p2.
P2_UP = [(0, 0), (2, 0), (0, 2), (1, 0), (1, 1), (0, 1)]
P2_DN = [(2, 0), (0, 2), (2, 2), (1, 1), (1, 2), (2, 1)]


def p2_patch(I, J):
    """(kind, a, b) of the level-L triangles holding lattice point (I, J)."""
    if I % 2 == 0 and J % 2 == 0:
        a, b = I // 2, J // 2
        return [("up", a, b), ("up", a - 1, b), ("up", a, b - 1), ("dn", a - 1, b), ("dn", a, b - 1),
                ("dn", a - 1, b - 1)]
    if J % 2 == 0:                              # horizontal micro-edge midpoint
        return [("up", (I - 1) // 2, J // 2), ("dn", (I - 1) // 2, J // 2 - 1)]
    if I % 2 == 0:                              # vertical
        return [("up", I // 2, (J - 1) // 2), ("dn", I // 2 - 1, (J - 1) // 2)]
    return [("up", (I - 1) // 2, (J - 1) // 2), ("dn", (I - 1) // 2, (J - 1) // 2)]   # diagonal


def p2_row(xy, tri, N1, f, I, J):
    """{(dI, dJ): weight} with (A2 x)_p = sum w x[p + (dI, dJ)] for the
    face-interior point p = (I, J) of the level-(L+1) lattice (N1 = 2^(L+1)
    intervals), from the oracle's P2 element matrices on the triangles
    holding p, placed relative to p (the matrices do not change under
    translation)."""
    from oracle import p2
    v0, v1, v2 = (np.asarray(xy[v], dtype=np.float64) for v in tri[f])
    nodes, X = [], []
    for kind, a, b in p2_patch(I, J):
        pts = [(2 * a + dx, 2 * b + dy) for dx, dy in (P2_UP if kind == "up" else P2_DN)]
        nodes.append(pts)
        X.append([((p[0] - I) / N1) * (v1 - v0) + ((p[1] - J) / N1) * (v2 - v0) for p in pts[:3]])
    K = p2.element_stiffness(np.array(X))
    w = {}
    for t, pts in enumerate(nodes):
        c = pts.index((I, J))
        for n, p in enumerate(pts):
            key = (p[0] - I, p[1] - J)
            w[key] = w.get(key, 0.0) + K[t, c, n]
    return w


# ------------------------------------------------------------------ Stokes
def stokes_row_weights(xy, tri, N, f, i, j, delta):
    """Weights (7,) in NEIGH order of the face-interior point p = (i, j) of
    face f for the Stokes operators of oracle.stokes, from the element
    quantities of the six micro-triangles around p (placed relative to p):
    B1, B2 (the pressure row of p over velocity neighbours), B1T, B2T (the
    velocity row of p over pressure neighbours), C (delta h_T^2 stiffness,
    h_T the longest edge) and A (the P1 stiffness).  Returns a dict."""
    v0, v1, v2 = (np.asarray(xy[v], dtype=np.float64) for v in tri[f])
    pts = [(i + di, j + dj) for di, dj in NEIGH]
    local = {pt: m for m, pt in enumerate(pts)}
    coords = np.array([((a - i) / N) * (v1 - v0) + ((b - j) / N) * (v2 - v0) for a, b in pts])
    elems = np.array([[local[v] for v in tri_vertices(kind, i + da, j + db)] for kind, da, db in PATCH])
    patch = SimpleNamespace(coords=coords, elements=elems)
    area, G = fem.element_geometry(patch)
    X = coords[elems]
    e = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 1], X[:, 0] - X[:, 2]], axis=1)
    h2 = (e ** 2).sum(axis=-1).max(axis=-1)
    K = fem.element_stiffness(patch)
    out = {k: np.zeros(7) for k in ("B1", "B2", "B1T", "B2T", "C", "A")}
    for t in range(6):
        c = int(np.where(elems[t] == 0)[0][0])
        for n in range(3):
            m = elems[t, n]
            for d, name in ((0, "1"), (1, "2")):
                out["B" + name][m] += -(area[t] / 3.0) * G[t, d, n]
                out["B" + name + "T"][m] += -(area[t] / 3.0) * G[t, d, c]
            out["C"][m] += delta * h2[t] * K[t, c, n]
            out["A"][m] += K[t, c, n]
    return out
