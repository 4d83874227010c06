"""Pins of the oracle's mesh, layout and operator against closed forms,
invariants and brute force (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem
from oracle import mesh as om
from paper_1805_10167_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def meshes():
    out = {"square": inputs.unit_square_mesh(), "annulus": inputs.annulus_mesh(32, 2)}
    out["random"] = inputs.random_square_mesh(7, 11)
    return out


# ------------------------------------------------------------ layout (Sec. 3, 5.2)
def test_paper_face_unknown_count():
    """Sec. 5.2: 2145 unknowns per macro-face at level 6; 256 faces give more
    than half a million unknowns."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_sec5_2_annulus_counts.json")))
    N = 1 << g["level"]
    assert len(om.closed_points(N)) == g["unknowns_per_face_closed"]
    assert g["macro_faces"] * g["unknowns_per_face_closed"] > g["total_unknowns_lower_bound"]
    # the 32 x 4 annulus has exactly the paper's 256 macro-faces
    xy, tri = inputs.annulus_mesh(32, 4)
    assert tri.shape[0] == g["macro_faces"]


@pytest.mark.parametrize("name", ["square", "annulus", "random"])
@pytest.mark.parametrize("L", [1, 2, 3])
def test_unique_ownership_and_ghost_coordinates(name, L):
    """Sec. 2.2: every unknown has exactly one owner; the copies a face sees
    (its boundary lattice points) sit at the owner's coordinates."""
    xy, tri = meshes()[name]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, L)
    N = lv.N
    seen = np.zeros(lv.n, dtype=int)
    for f, G in enumerate(lv.face_ids):
        for (i, j) in om.closed_points(N):
            g = G[j, i]
            assert g >= 0
            np.testing.assert_allclose(lv.coords[g], lv.face_point_coords(f, i, j), atol=1e-14)
            if 0 < i and 0 < j and i + j < N:
                seen[g] += 1
    # every face-interior id owned once; the rest are vertices or edge points
    assert np.all(seen[lv.kind == 2] == 1)
    # count = vertices + edge interiors + face interiors; no duplicates in coords
    assert lv.n == M.nv + M.ne * (N - 1) + M.nf * (N - 1) * (N - 2) // 2
    uniq = np.unique(np.round(lv.coords, 12), axis=0)
    assert uniq.shape[0] == lv.n


def test_refinement_congruent_children():
    """Sec. 3.1: refinement by edge midpoints gives congruent children: all
    micro-triangles of a face have area |F| / N^2 and the same element matrix
    up to vertex order."""
    xy, tri = meshes()["random"]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 3)
    N = lv.N
    area, _ = fem.element_geometry(lv)
    K = fem.element_stiffness(lv)
    for f in range(M.nf):
        a, b, c = xy[M.tri[f]]
        Af = 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        sl = slice(f * N * N, (f + 1) * N * N)
        np.testing.assert_allclose(area[sl], Af / N ** 2, rtol=1e-12)
        ev = np.sort(np.linalg.eigvalsh(K[sl]), axis=1)
        np.testing.assert_allclose(ev, np.broadcast_to(ev[0], ev.shape), atol=1e-12)


# ------------------------------------------------------------ operator (Sec. 4.2)
@pytest.mark.parametrize("name", ["square", "annulus", "random"])
@pytest.mark.parametrize("vark", [False, True])
def test_element_loop_equals_csr(name, vark):
    """The matrix-free element-loop apply equals the brute-force assembled
    CSR matrix (restricted to free rows)."""
    xy, tri = meshes()[name]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 3)
    rng = np.random.default_rng(1)
    k = rng.uniform(0.5, 2.0, M.nf * lv.N ** 2) if vark else None
    A = fem.free_rows(fem.assemble(lv, k), lv)
    x = rng.standard_normal(lv.n)
    np.testing.assert_allclose(fem.apply_element_loop(lv, x, k), A @ x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", ["square", "annulus", "random"])
def test_row_sums_symmetry_definiteness(name):
    xy, tri = meshes()[name]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 2)
    k = np.random.default_rng(2).uniform(0.1, 10.0, M.nf * lv.N ** 2)
    for kk in (None, k):
        A = fem.assemble(lv, kk).toarray()
        np.testing.assert_allclose(A.sum(axis=1), 0.0, atol=1e-12)   # pure diffusion
        np.testing.assert_allclose(A, A.T, atol=1e-13)
        Af = A[np.ix_(lv.free, lv.free)]
        assert np.linalg.eigvalsh(Af).min() > 0.0


@pytest.mark.parametrize("name", ["square", "annulus", "random"])
def test_linear_functions_in_kernel(name):
    """Constant k: A applied to a global linear function vanishes at every
    unknown off the domain boundary."""
    xy, tri = meshes()[name]
    M = om.MacroMesh(xy, tri, dirichlet_vertex=np.zeros(xy.shape[0]))
    lv = om.Level(M, 3)
    A = fem.assemble(lv)
    u = 0.3 + 1.7 * lv.coords[:, 0] - 2.2 * lv.coords[:, 1]
    y = A @ u
    # unknowns on the domain boundary: boundary vertices and boundary-edge points
    on_b = np.zeros(lv.n, dtype=bool)
    for k_, (a, b) in enumerate(M.edges):
        if M.boundary_edge[k_]:
            on_b[a] = on_b[b] = True
            on_b[lv.edge_off + k_ * lv.n_e_int: lv.edge_off + (k_ + 1) * lv.n_e_int] = True
    np.testing.assert_allclose(y[~on_b], 0.0, atol=1e-12)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_unit_square_eigenpairs(L):
    """On the unit square cut into right isosceles triangles the P1 matrix is
    the unscaled 5-point Laplacian, so sin(k pi x) sin(l pi y) at the free
    nodes is an eigenvector with eigenvalue 4 sin^2(k pi h/2) + 4 sin^2(l pi h/2),
    h = 1/(2N)."""
    xy, tri = inputs.unit_square_mesh()
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, L)
    A = fem.assemble(lv)
    h = 1.0 / (2 * lv.N)
    fr = lv.free
    Af = A[fr][:, fr]
    X, Y = lv.coords[fr, 0], lv.coords[fr, 1]
    for (k, l) in ((1, 1), (2, 3), (5, 1)):
        v = np.sin(k * np.pi * X) * np.sin(l * np.pi * Y)
        lam = 4 * np.sin(k * np.pi * h / 2) ** 2 + 4 * np.sin(l * np.pi * h / 2) ** 2
        np.testing.assert_allclose(Af @ v, lam * v, atol=1e-12)


def _angle(p, q, r):
    """Angle at p of triangle p, q, r by atan2 (independent of the gradient
    formula used by the oracle's element matrices)."""
    u, v = q - p, r - p
    return math.atan2(abs(u[0] * v[1] - u[1] * v[0]), u[0] * v[0] + u[1] * v[1])


@pytest.mark.parametrize("name", ["annulus", "random"])
def test_face_interior_cotangent_stencil(name):
    """Face-interior rows equal the 7-point cotangent stencil of the macro
    face: w(+-e1) = -cot t2, w(+-e2) = -cot t1, w(+-(e1-e2)) = -cot t0,
    centre = 2 (cot t0 + cot t1 + cot t2); with a per-element coefficient each
    micro-edge weight is -1/2 cot(opposite angle) (k_T1 + k_T2)."""
    xy, tri = meshes()[name]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 3)
    N = lv.N
    rng = np.random.default_rng(3)
    k = rng.uniform(0.5, 2.0, M.nf * N * N)
    A1 = fem.assemble(lv).tocsr()
    Ak = fem.assemble(lv, k).tocsr()

    def up(f, i, j):
        return f * N * N + j * N - j * (j - 1) // 2 + i

    def dn(f, i, j):
        return f * N * N + N * (N + 1) // 2 + j * (N - 1) - j * (j - 1) // 2 + i
    for f in range(M.nf):
        v0, v1, v2 = xy[M.tri[f]]
        c0 = 1 / math.tan(_angle(v0, v1, v2))
        c1 = 1 / math.tan(_angle(v1, v2, v0))
        c2 = 1 / math.tan(_angle(v2, v0, v1))
        G = lv.face_ids[f]
        for (i, j) in ((1, 1), (2, 3), (N - 3, 2), (3, N - 4)):
            p = G[j, i]
            nb = {(1, 0): c2, (-1, 0): c2, (0, 1): c1, (0, -1): c1, (1, -1): c0, (-1, 1): c0}
            for (di, dj), c in nb.items():
                assert A1[p, G[j + dj, i + di]] == pytest.approx(-c, abs=1e-12)
            assert A1[p, p] == pytest.approx(2 * (c0 + c1 + c2), abs=1e-12)
            kk = {(1, 0): k[up(f, i, j)] + k[dn(f, i, j - 1)],
                  (-1, 0): k[up(f, i - 1, j)] + k[dn(f, i - 1, j - 1)],
                  (0, 1): k[up(f, i, j)] + k[dn(f, i - 1, j)],
                  (0, -1): k[up(f, i, j - 1)] + k[dn(f, i - 1, j - 1)],
                  (1, -1): k[up(f, i, j - 1)] + k[dn(f, i, j - 1)],
                  (-1, 1): k[up(f, i - 1, j)] + k[dn(f, i - 1, j)]}
            tot = 0.0
            for (di, dj), c in nb.items():
                w = -0.5 * c * kk[(di, dj)]
                assert Ak[p, G[j + dj, i + di]] == pytest.approx(w, abs=1e-12)
                tot += w
            assert Ak[p, p] == pytest.approx(-tot, abs=1e-12)


def test_constant_coefficient_scales():
    xy, tri = meshes()["annulus"]
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 2)
    A = fem.assemble(lv).toarray()
    Ac = fem.assemble(lv, np.full(M.nf * lv.N ** 2, 3.5)).toarray()
    np.testing.assert_allclose(Ac, 3.5 * A, atol=1e-12)


# ------------------------------------------------------------ mass, quadrature
def test_mass_matrix_total_is_area():
    for name, area in (("square", 1.0), ("annulus", 32 * 0.5 * math.sin(2 * math.pi / 32) * (1 - 0.55 ** 2))):
        xy, tri = meshes()[name]
        lv = om.Level(om.MacroMesh(xy, tri), 3)
        assert fem.mass_matrix(lv).sum() == pytest.approx(area, rel=1e-13)


def test_radon_rule_degree_five():
    """Radon's 7-point rule integrates x^a y^b, a + b <= 5, exactly on the
    reference triangle: integral = a! b! / (a + b + 2)!."""
    B, w = fem.radon7()
    x, y = B[:, 1], B[:, 2]
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert 0.5 * np.sum(w * x ** a * y ** b) == pytest.approx(exact, rel=1e-13, abs=1e-16)
    # not exact at degree 6
    assert abs(0.5 * np.sum(w * x ** 6) - math.factorial(6) / math.factorial(8)) > 1e-8


def test_interpolant_l2_error_order():
    """The L2 error of the nodal interpolant of a smooth function falls as h^2."""
    xy, tri = meshes()["square"]
    M = om.MacroMesh(xy, tri)
    u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    e = []
    for L in (2, 3, 4, 5):
        lv = om.Level(M, L)
        e.append(fem.l2_error(lv, u(lv.coords[:, 0], lv.coords[:, 1]), u))
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all((orders > 1.9) & (orders < 2.1))


def test_invalid_meshes_rejected():
    xy, tri = inputs.unit_square_mesh()
    with pytest.raises(om.MeshError):
        om.MacroMesh(xy, np.array([[0, 1, 1]]))
    with pytest.raises(om.MeshError):
        om.MacroMesh(xy, np.array([[0, 1, 99]]))
    bad = np.concatenate([tri, tri[:1]])     # an edge used by three faces
    with pytest.raises(om.MeshError):
        om.MacroMesh(xy, bad)
