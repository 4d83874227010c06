"""The sampled-row helper of the full-size GPU tests, pinned on the CPU: its
rows equal the oracle's element-loop operator at every face-interior point of
a small level (constant and random coefficient), and its element numbering is
the canonical one of the oracle's level."""
import numpy as np
import pytest

from oracle import fem
from oracle import mesh as om
from paper_1805_10167_gb300 import inputs

import fullsize_rows as fr


@pytest.mark.parametrize("name", ["annulus", "random"])
@pytest.mark.parametrize("vark", [False, True])
def test_rows_equal_element_loop(name, vark):
    xy, tri = inputs.annulus_mesh(32, 2) if name == "annulus" else inputs.random_square_mesh(5, 12)
    M = om.MacroMesh(xy, tri)
    L = 4
    lv = om.Level(M, L)
    N = lv.N
    rng = np.random.default_rng(3)
    k = rng.uniform(0.3, 3.0, size=lv.elements.shape[0]) if vark else None
    x = rng.standard_normal(lv.n)
    want = fem.apply_element_loop(lv, x, k)
    worst = 0.0
    for f in range(0, M.nf, max(1, M.nf // 6)):
        G = lv.face_ids[f]
        for j in range(1, N - 1):
            for i in range(1, N - j):
                kp = None if k is None else k[fr.patch_element_ids(N, f, i, j)]
                w = fr.row_weights(M.xy, M.tri, N, f, i, j, kp)
                ids = [G[j + dj, i + di] for di, dj in fr.NEIGH]
                got = w @ x[ids]
                worst = max(worst, abs(got - want[G[j, i]]))
    assert worst <= 1e-13 * np.abs(want).max()


def test_element_numbering_matches_oracle_level():
    xy, tri = inputs.annulus_mesh(32, 2)
    M = om.MacroMesh(xy, tri)
    lv = om.Level(M, 3)
    N = lv.N
    for f in (0, 7, M.nf - 1):
        G = lv.face_ids[f]
        for b in range(N):
            for a in range(N - b):
                e = f * N * N + fr.element_index(N, "up", a, b)
                assert list(lv.elements[e]) == [G[v[1], v[0]] for v in fr.tri_vertices("up", a, b)]
        for b in range(N - 1):
            for a in range(N - 1 - b):
                e = f * N * N + fr.element_index(N, "dn", a, b)
                assert list(lv.elements[e]) == [G[v[1], v[0]] for v in fr.tri_vertices("dn", a, b)]


@pytest.mark.parametrize("name,L", [("annulus", 2), ("random", 2)])
def test_p2_rows_equal_assembled_matrix(name, L):
    """The one-row P2 helper equals the rows of the oracle's assembled P2
    matrix at every face-interior lattice point (all four point types)."""
    from oracle import p2
    from oracle import mesh as om
    xy, tri = (inputs.annulus_mesh(32, 2) if name == "annulus" else inputs.random_square_mesh(5, 9))
    M = om.MacroMesh(xy, tri)
    P = p2.P2Level(M, L)
    A = p2.assemble(P).tocsr()
    N1 = P.lat.N
    for f, G in enumerate(P.lat.face_ids):
        for J in range(1, N1 - 1):
            for I in range(1, N1 - J):
                w = fr.p2_row(xy, M.tri, N1, f, I, J)
                row = A[G[J, I]]
                got = {}
                for (dI, dJ), v in w.items():
                    q = G[J + dJ, I + dI]
                    got[q] = got.get(q, 0.0) + v
                for q, v in zip(row.indices, row.data):
                    assert abs(got.pop(q, 0.0) - v) <= 1e-12 * abs(row.data).max()
                assert all(abs(v) <= 1e-12 * abs(row.data).max() for v in got.values())


@pytest.mark.parametrize("name", ["annulus", "random"])
def test_stokes_rows_equal_assembled_operators(name):
    """The one-row Stokes helper equals the rows of the oracle's assembled
    B1, B2, their transposes, C and A at every face-interior point of a small
    level."""
    from oracle import stokes
    xy, tri = inputs.annulus_mesh(32, 4) if name == "annulus" else inputs.random_square_mesh(5, 12)
    M = om.MacroMesh(xy, tri)
    L, delta = 3, 0.3
    lv = om.Level(M, L)
    N = lv.N
    B1, B2 = stokes.div_matrices(lv)
    mats = {"B1": B1, "B2": B2, "B1T": B1.T.tocsr(), "B2T": B2.T.tocsr(),
            "C": stokes.stabilisation(lv, delta), "A": fem.assemble(lv)}
    dense = {k: v.toarray() for k, v in mats.items()}
    worst = 0.0
    for f in range(M.nf):
        G = lv.face_ids[f]
        for j in range(1, N - 1):
            for i in range(1, N - j):
                w = fr.stokes_row_weights(M.xy, M.tri, N, f, i, j, delta)
                ids = [G[j + dj, i + di] for di, dj in fr.NEIGH]
                for k, D in dense.items():
                    row = D[G[j, i]]
                    scale = np.abs(row).max()
                    worst = max(worst, np.abs(row[ids] - w[k]).max() / scale)
                    # nothing outside the 7-point stencil
                    rest = np.delete(row, ids)
                    assert np.abs(rest).max(initial=0.0) <= 1e-14 * scale
    assert worst <= 1e-13
