"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the multigrid method itself: it only makes
macro meshes, random right-hand sides and random coefficient fields.

* ``unit_square_mesh``: the unit square cut into 2x2 quads, each split along
  its (x0,y0)-(x1,y1) diagonal (8 macro-triangles).
* ``annulus_mesh``: the straight-edged annulus r in [0.55, 1] meshed as
  n_ang x n_rad quads, each split along its (i,j)-(i+1,j+1) diagonal.  Its
  shape follows the annulus of the paper's energy-transport example (Sec. 5.2).
* ``random_square_mesh``: a seeded random valid triangulation of the unit
  square (point insertion, boundary splits, Lawson flips to Delaunay).
* ``splitmix64`` / ``uniform_pm1``: Vigna's SplitMix64 counter generator and
  its map to uniform doubles in [-1, 1); the value for canonical DoF p is drawn
  from ``splitmix64(seed ^ p)``.
* ``grf_coefficient``: k = exp(g) with g a Gaussian random field of
  squared-exponential covariance sigma^2 exp(-d^2 / (2 l^2)), drawn by random
  Fourier features (Rahimi & Recht 2007) and sampled at element centroids.
* ``element_centroids``: centroids of the fine micro-triangles of every face in
  the library's canonical element order (per face: upward triangles row by row,
  then downward triangles row by row) -- the sampling points of k.

Every mesh is returned with counter-clockwise triangles.
"""
from __future__ import annotations

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _ccw(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    tri = np.array(tri, dtype=np.int32, copy=True)
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = cross < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    return tri


def unit_square_mesh(nq: int = 2):
    """Unit square, nq x nq quads, each cut along its (x0,y0)-(x1,y1) diagonal."""
    g = np.linspace(0.0, 1.0, nq + 1)
    xy = np.array([[g[i], g[j]] for j in range(nq + 1) for i in range(nq + 1)], dtype=np.float64)
    vid = lambda i, j: j * (nq + 1) + i
    tri = []
    for j in range(nq):
        for i in range(nq):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tri.append((a, b, c))
            tri.append((a, c, d))
    return xy, _ccw(xy, np.array(tri))


def annulus_mesh(n_ang: int = 32, n_rad: int = 2, r0: float = 0.55, r1: float = 1.0):
    """Straight-edged annulus: vertices at r_j = r0 + (r1-r0) j / n_rad and
    theta_i = 2 pi i / n_ang (vertex id j*n_ang + i); quad (i,j),(i+1,j),
    (i+1,j+1),(i,j+1) split along its (i,j)-(i+1,j+1) diagonal."""
    xy = []
    for j in range(n_rad + 1):
        r = r0 + (r1 - r0) * j / n_rad
        for i in range(n_ang):
            th = 2.0 * np.pi * i / n_ang
            xy.append((r * np.cos(th), r * np.sin(th)))
    xy = np.array(xy, dtype=np.float64)
    vid = lambda i, j: j * n_ang + (i % n_ang)
    tri = []
    for j in range(n_rad):
        for i in range(n_ang):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tri.append((a, b, c))
            tri.append((a, c, d))
    return xy, _ccw(xy, np.array(tri))


def _min_angle(p, q, r):
    def ang(a, b, c):
        u, v = b - a, c - a
        cu = float(np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v)))
        return np.degrees(np.arccos(np.clip(cu, -1.0, 1.0)))
    return min(ang(p, q, r), ang(q, r, p), ang(r, p, q))


def random_square_mesh(seed: int, n_faces: int):
    """Seeded random valid triangulation of the unit square with n_faces >= 2
    triangles: start from the square cut by one diagonal; repeat interior point
    insertion into one of the three largest faces (+2 faces; barycentric
    weights drawn from [0.2, 0.6] and normalised) or a split of one of the two
    longest boundary edges at t in [0.3, 0.7] (+1 face) until the count is
    reached; then Lawson flips until the triangulation is Delaunay (every
    interior edge's two opposite angles sum to at most pi), and eight rounds
    of Laplacian smoothing of the interior points (moves that would flip or
    collapse a triangle are skipped), each followed by Delaunay flips."""
    if n_faces < 2:
        raise ValueError("n_faces must be >= 2")
    rng = np.random.default_rng(seed)
    pts = [np.array(p, dtype=np.float64) for p in ((0, 0), (1, 0), (1, 1), (0, 1))]
    tris = [[0, 1, 2], [0, 2, 3]]

    def edge_faces():
        m = {}
        for f, t in enumerate(tris):
            for s in range(3):
                a, b = t[s], t[(s + 1) % 3]
                m.setdefault((min(a, b), max(a, b)), []).append(f)
        return m

    while len(tris) < n_faces:
        need = n_faces - len(tris)
        if need >= 2 and rng.random() < 0.6:
            # one of the three largest faces, near its centroid
            areas = []
            for t in tris:
                p0, p1, p2 = pts[t[0]], pts[t[1]], pts[t[2]]
                areas.append(abs((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0])))
            order = np.argsort(areas)[::-1]
            f = int(order[int(rng.integers(min(3, len(order))))])
            w = rng.uniform(0.2, 0.6, size=3)
            w /= w.sum()
            a, b, c = tris[f]
            p = w[0] * pts[a] + w[1] * pts[b] + w[2] * pts[c]
            pts.append(p)
            n = len(pts) - 1
            tris[f] = [a, b, n]
            tris.append([b, c, n])
            tris.append([c, a, n])
        else:
            em = edge_faces()
            bnd = [e for e, fs in em.items() if len(fs) == 1]
            lens = [np.linalg.norm(pts[a] - pts[b]) for a, b in bnd]
            order = np.argsort(lens)[::-1]
            e = bnd[int(order[int(rng.integers(min(2, len(order))))])]   # one of the two longest
            f = em[e][0]
            t = rng.uniform(0.3, 0.7)
            a, b = e
            p = (1 - t) * pts[a] + t * pts[b]
            pts.append(p)
            n = len(pts) - 1
            tri = tris[f]
            # rotate so that (tri[0], tri[1]) is the split edge
            for s in range(3):
                if {tri[s], tri[(s + 1) % 3]} == {a, b}:
                    u, v, w_ = tri[s], tri[(s + 1) % 3], tri[(s + 2) % 3]
                    break
            tris[f] = [u, n, w_]
            tris.append([n, v, w_])
    # Lawson flips to the Delaunay triangulation of the points: an interior
    # edge is flipped while the two angles opposite to it sum to more than pi
    def opp_angle(t, e):
        c = [v for v in t if v not in e][0]
        u, w = pts[e[0]] - pts[c], pts[e[1]] - pts[c]
        return np.arccos(np.clip(np.dot(u, w) / (np.linalg.norm(u) * np.linalg.norm(w)), -1.0, 1.0))
    for _ in range(50 * n_faces):
        em = edge_faces()
        flipped = False
        for e, fs in em.items():
            if len(fs) != 2:
                continue
            f1, f2 = fs
            if opp_angle(tris[f1], e) + opp_angle(tris[f2], e) <= np.pi + 1e-12:
                continue
            a, b = e
            c = [v for v in tris[f1] if v not in e][0]
            d = [v for v in tris[f2] if v not in e][0]
            tris[f1], tris[f2] = [c, d, a], [d, c, b]
            flipped = True
            break
        if not flipped:
            break
    def delaunay():
        for _ in range(50 * n_faces):
            em = edge_faces()
            flipped = False
            for e, fs in em.items():
                if len(fs) != 2:
                    continue
                f1, f2 = fs
                if opp_angle(tris[f1], e) + opp_angle(tris[f2], e) <= np.pi + 1e-12:
                    continue
                a, b = e
                c = [v for v in tris[f1] if v not in e][0]
                d = [v for v in tris[f2] if v not in e][0]
                tris[f1], tris[f2] = [c, d, a], [d, c, b]
                flipped = True
                break
            if not flipped:
                return

    def signed_area(t):
        p0, p1, p2 = pts[t[0]], pts[t[1]], pts[t[2]]
        return (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0])
    # Laplacian smoothing of the interior points (a move is kept only if no
    # incident triangle flips or collapses), then Delaunay flips again
    for _ in range(8):
        em = edge_faces()
        on_bnd = set()
        nbrs = {}
        for (a, b), fs in em.items():
            if len(fs) == 1:
                on_bnd.update((a, b))
            nbrs.setdefault(a, set()).add(b)
            nbrs.setdefault(b, set()).add(a)
        for v in range(4, len(pts)):
            if v in on_bnd or v not in nbrs:
                continue
            inc = [t for t in tris if v in t]
            sign = [np.sign(signed_area(t)) for t in inc]
            old = pts[v].copy()
            pts[v] = np.mean([pts[u] for u in nbrs[v]], axis=0)
            if any(np.sign(signed_area(t)) != s0 or abs(signed_area(t)) < 1e-9 for t, s0 in zip(inc, sign)):
                pts[v] = old
        delaunay()
    xy = np.array(pts, dtype=np.float64)
    return xy, _ccw(xy, np.array(tris))


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Vigna 2015; Steele, Lea & Flood 2014)
    applied to 64-bit states ``x`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & MASK64
        return z ^ (z >> np.uint64(31))


def uniform_pm1(n: int, seed: int) -> np.ndarray:
    """n doubles uniform in [-1, 1): value p = (top 53 bits of
    splitmix64(seed ^ p)) * 2^-52 - 1."""
    p = np.arange(n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ p)
    u = (z >> np.uint64(11)).astype(np.float64)
    return u * (2.0 ** -52) - 1.0


def element_centroids(xy: np.ndarray, tri: np.ndarray, level: int, device=None):
    """Centroids (n_faces * N^2, 2) of the level-``level`` micro-triangles in
    canonical element order.  Face frame: x = v0 + (i/N)(v1-v0) + (j/N)(v2-v0),
    (v0,v1,v2) the counter-clockwise face.  Upward triangle (i,j): lattice
    points (i,j),(i+1,j),(i,j+1), i+j <= N-1; downward triangle (i,j):
    (i+1,j),(i,j+1),(i+1,j+1), i+j <= N-2; both row by row (j outer)."""
    tri = _ccw(xy, tri)
    N = 1 << level
    up = [(i, j) for j in range(N) for i in range(N - j)]
    dn = [(i, j) for j in range(N - 1) for i in range(N - 1 - j)]
    cu = np.array([(i + 1.0 / 3.0, j + 1.0 / 3.0) for i, j in up]).reshape(-1, 2) / N
    cd = np.array([(i + 2.0 / 3.0, j + 2.0 / 3.0) for i, j in dn]).reshape(-1, 2) / N
    loc = np.concatenate([cu, cd], axis=0)  # (N^2, 2) in (s,t) frame coordinates
    v0, v1, v2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    if device is not None:   # same arithmetic with torch (large levels)
        import torch
        T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
        lt, a0, a1, a2 = T(loc), T(v0), T(v1), T(v2)
        out = (a0[:, None, :] + lt[None, :, 0:1] * (a1 - a0)[:, None, :]
               + lt[None, :, 1:2] * (a2 - a0)[:, None, :])
        return out.reshape(-1, 2)
    out = (v0[:, None, :] + loc[None, :, 0:1] * (v1 - v0)[:, None, :]
           + loc[None, :, 1:2] * (v2 - v0)[:, None, :])
    return out.reshape(-1, 2)


def grf_coefficient(points: np.ndarray, seed: int = 42, length: float = 0.1,
                    sigma: float = 1.0, n_features: int = 512) -> np.ndarray:
    """k = exp(g(points)), g(x) = sigma sqrt(2/M) sum_m cos(w_m . x + phi_m),
    w_m ~ N(0, length^-2 I), phi_m ~ U[0, 2 pi): a random-Fourier-feature draw
    of a zero-mean Gaussian field with covariance sigma^2 exp(-d^2/(2 l^2))."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0 / length, size=(n_features, 2))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_features)
    if not isinstance(points, np.ndarray):   # torch tensor: same draw, evaluated with torch
        import torch
        wt = torch.as_tensor(w, dtype=torch.float64, device=points.device)
        pt = torch.as_tensor(phi, dtype=torch.float64, device=points.device)
        out = torch.empty(points.shape[0], dtype=torch.float64, device=points.device)
        step = 1 << 20
        for s0 in range(0, points.shape[0], step):
            pr = points[s0:s0 + step] @ wt.T + pt[None, :]
            out[s0:s0 + step] = sigma * np.sqrt(2.0 / n_features) * torch.cos(pr).sum(dim=1)
        return torch.exp(out)
    out = np.empty(points.shape[0], dtype=np.float64)
    step = 1 << 20
    for s in range(0, points.shape[0], step):
        pr = points[s:s + step] @ w.T + phi[None, :]
        out[s:s + step] = sigma * np.sqrt(2.0 / n_features) * np.cos(pr).sum(axis=1)
    return np.exp(out)


def batch_workload(n: int = 64, seed0: int = 1000, min_level: int = 6, max_level: int = 9):
    """n independent problems: problem k uses seed s = seed0 + k, a random
    triangulation of the unit square with 2 + (splitmix64(s) mod 63) faces
    and level min_level + (splitmix64(s ^ 0x5bd1e995) mod (max_level -
    min_level + 1)).  Returns [(xy, tri, level)]."""
    out = []
    span = max_level - min_level + 1
    for k in range(n):
        s = seed0 + k
        h1 = int(splitmix64(np.array([s], dtype=np.uint64))[0])
        h2 = int(splitmix64(np.array([s ^ 0x5BD1E995], dtype=np.uint64))[0])
        nf = 2 + h1 % 63
        L = min_level + h2 % span
        xy, tri = random_square_mesh(s, nf)
        out.append((xy, tri, L))
    return out
