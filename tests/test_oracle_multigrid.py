"""Pins of the oracle's smoother, transfers, coarse solver and V-cycle (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem
from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs


def mesh_of(name, **kw):
    if name == "square":
        xy, tri = inputs.unit_square_mesh()
    elif name == "annulus":
        xy, tri = inputs.annulus_mesh(32, 2)
    else:
        xy, tri = inputs.random_square_mesh(5, 9)
    return om.MacroMesh(xy, tri, **kw)


# ------------------------------------------------------------- Gauss-Seidel
@pytest.mark.parametrize("name,L", [("square", 3), ("annulus", 2), ("random", 3), ("random", 1)])
def test_colour_sets_are_independent_and_cover_free(name, L):
    M = mesh_of(name)
    lv = om.Level(M, L)
    adj = mg.adjacency(lv)
    sets = mg.gs_sets(lv)
    allidx = np.concatenate(sets)
    assert np.array_equal(np.sort(allidx), np.nonzero(lv.free)[0])
    for S in sets:
        sub = adj[S][:, S]
        assert sub.nnz == 0 or np.all(sub.diagonal() == sub.sum(axis=1).A1)


@pytest.mark.parametrize("name,L", [("square", 3), ("annulus", 2), ("random", 2)])
@pytest.mark.parametrize("vark", [False, True])
def test_colour_gs_equals_sequential_gs(name, L, vark):
    """A colour-ordered sweep equals point Gauss-Seidel visiting the DoFs one
    by one in the same (colour-major) order, forward and backward."""
    M = mesh_of(name)
    rng = np.random.default_rng(4)
    k = rng.uniform(0.5, 2.0, M.nf * (1 << L) ** 2) if vark else None
    H = mg.Hierarchy(M, L, k)
    lv = H.levels[L]
    x0 = rng.standard_normal(lv.n)
    b = rng.standard_normal(lv.n)
    order = np.concatenate(mg.gs_sets(lv))
    for fwd in (True, False):
        xa = mg.gs_sweep(H, L, x0.copy(), b, forward=fwd)
        xb = mg.sequential_gs(H.A[L], order if fwd else order[::-1], x0.copy(), b)
        np.testing.assert_allclose(xa, xb, rtol=0, atol=1e-13)


def test_gs_reduces_energy_error():
    """Each GS point update minimises the energy along its coordinate, so a
    sweep never increases the A-norm of the error."""
    M = mesh_of("annulus")
    H = mg.Hierarchy(M, 3)
    lv = H.levels[3]
    A = H.A[3][lv.free][:, lv.free]
    rng = np.random.default_rng(5)
    xs = np.zeros(lv.n)
    xs[lv.free] = rng.standard_normal(lv.free.sum())
    b = H.apply(3, xs)
    x = np.zeros(lv.n)
    e_prev = np.inf
    for _ in range(5):
        mg.gs_sweep(H, 3, x, b)
        e = (x - xs)[lv.free]
        en = e @ (A @ e)
        assert en <= e_prev
        e_prev = en


# ------------------------------------------------------------- transfers
@pytest.mark.parametrize("name", ["square", "annulus", "random"])
def test_prolongation_reproduces_linear_functions(name):
    M = mesh_of(name, dirichlet_vertex=np.zeros(len(mesh_of(name).xy)))
    for L in (1, 2, 3):
        c, f = om.Level(M, L - 1), om.Level(M, L)
        P = mg.prolongation(c, f)
        lin = lambda X: 0.7 - 1.3 * X[:, 0] + 2.9 * X[:, 1]
        np.testing.assert_allclose(P @ lin(c.coords), lin(f.coords), atol=1e-13)


@pytest.mark.parametrize("name", ["square", "annulus", "random"])
def test_galerkin_identity(name):
    """Nested P1 spaces with constant coefficient: P^T A_l P = A_{l-1} on the
    free DoFs."""
    M = mesh_of(name)
    for L in (1, 2, 3):
        c, f = om.Level(M, L - 1), om.Level(M, L)
        P = mg.prolongation(c, f)
        Af = fem.assemble(f)
        Ac = fem.assemble(c).toarray()
        G = (P.T @ Af @ P).toarray()
        fr = c.free
        np.testing.assert_allclose(G[np.ix_(fr, fr)], Ac[np.ix_(fr, fr)], atol=1e-12)


def test_restriction_stencil_closed_form():
    """Coarse face-interior (I, J) of P^T r is r(2I, 2J) plus half of r at the
    six fine lattice neighbours (full weighting written out by index)."""
    M = mesh_of("annulus")
    c, f = om.Level(M, 2), om.Level(M, 3)
    P = mg.prolongation(c, f)
    r = np.random.default_rng(6).standard_normal(f.n)
    r[~f.free] = 0.0
    bc = P.T @ r
    for fc in range(M.nf):
        Gc, Gf = c.face_ids[fc], f.face_ids[fc]
        I, J = 1, 1
        a, b_ = 2 * I, 2 * J
        nb = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]
        want = r[Gf[b_, a]] + 0.5 * sum(r[Gf[b_ + dj, a + di]] for di, dj in nb)
        assert bc[Gc[J, I]] == pytest.approx(want, abs=1e-14)


def test_coarsened_coefficient_children_by_centroid():
    """The index rule for the four children of a coarse element agrees with a
    geometric one (fine elements whose centroid lies inside the coarse one),
    and a constant coefficient stays constant."""
    M = mesh_of("random")
    L = 3
    c, f = om.Level(M, L - 1), om.Level(M, L)
    nf, Nf = M.nf, f.N
    rng = np.random.default_rng(7)
    k = rng.uniform(0.5, 2.0, nf * Nf * Nf)
    kc = mg.coarsen_coefficient(c, k, nf)
    cf = f.coords[f.elements].mean(axis=1)
    C = c.coords[c.elements]
    for e in range(C.shape[0]):
        a, b, cc = C[e]
        D = np.stack([b - a, cc - a], axis=1)
        lam = np.linalg.solve(D, (cf - a).T).T
        inside = (lam[:, 0] > 1e-9) & (lam[:, 1] > 1e-9) & (lam.sum(1) < 1 - 1e-9)
        assert inside.sum() == 4
        assert kc[e] == pytest.approx(k[inside].mean(), rel=1e-14)
    np.testing.assert_allclose(mg.coarsen_coefficient(c, np.full(k.size, 2.5), nf), 2.5)


# ------------------------------------------------------------- coarse solve
@pytest.mark.parametrize("name", ["square", "annulus", "random"])
def test_coarse_cg_equals_dense_solve(name):
    M = mesh_of(name)
    lv = om.Level(M, 0)
    A = fem.assemble(lv)
    b = np.random.default_rng(8).standard_normal(lv.n)
    x = mg.cg(A, lv.free, b)
    fr = lv.free
    ref = np.linalg.solve(A.toarray()[np.ix_(fr, fr)], b[fr])
    np.testing.assert_allclose(x[fr], ref, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------- V-cycle
def test_vcycle_level1_is_two_grid_with_exact_coarse_solve():
    M = mesh_of("annulus")
    H = mg.Hierarchy(M, 1)
    lv, lc = H.levels[1], H.levels[0]
    rng = np.random.default_rng(9)
    b = rng.standard_normal(lv.n)
    x = rng.standard_normal(lv.n)
    x[~lv.free] = 0
    got = mg.vcycle(H, 1, x.copy(), b, 2, 2)
    # two-grid written out with a dense coarse solve
    y = x.copy()
    for _ in range(2):
        mg.gs_sweep(H, 1, y, b, True)
    r = H.residual(1, y, b)
    P = H.P(1).toarray()
    rc = P.T @ r
    fr = lc.free
    ec = np.zeros(lc.n)
    ec[fr] = np.linalg.solve(H.A[0].toarray()[np.ix_(fr, fr)], rc[fr])
    y += P @ ec
    for _ in range(2):
        mg.gs_sweep(H, 1, y, b, False)
    np.testing.assert_allclose(got, y, atol=1e-12)


def _asymptotic_rate(H, L, nu, cycles=12):
    lv = H.levels[L]
    b = inputs.uniform_pm1(lv.n, 1234)
    b[~lv.free] = 0
    x = np.zeros(lv.n)
    x, hist = mg.solve(H, x, b, nu, nu, tol=0.0, max_iter=cycles, level=L)
    return hist[-1] / hist[-2]


@pytest.mark.parametrize("name", ["square", "annulus"])
def test_convergence_factor_level_independent(name):
    """V(3,3): the asymptotic residual reduction per cycle stays bounded and
    nearly constant as the mesh is refined (levels 3..6)."""
    M = mesh_of(name)
    H = mg.Hierarchy(M, 6)
    rates = [_asymptotic_rate(H, L, 3) for L in (3, 4, 5, 6)]
    assert max(rates) < 0.25
    assert max(rates) - min(rates) < 0.06


def test_manufactured_solution_second_order():
    """u = sin(pi x) sin(pi y) on the unit square, f = 2 pi^2 u, b = M f_I:
    the multigrid solution's L2 error falls with observed order in [1.9, 2.1]."""
    M = mesh_of("square")
    u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2 * np.pi ** 2 * u(x, y)
    H = mg.Hierarchy(M, 6)
    errs = []
    for L in (3, 4, 5, 6):
        lv = H.levels[L]
        b = fem.load_vector(lv, f)
        x, hist = mg.solve(H, np.zeros(lv.n), b, 2, 2, tol=1e-10, level=L)
        assert hist[-1] <= 1e-10 * hist[0]
        errs.append(fem.l2_error(lv, x, u))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 1.9) & (orders < 2.1)), orders


@pytest.mark.parametrize("omega", [2.0 / 3.0, 0.5, 1.0])
@pytest.mark.parametrize("L", [2, 3])
def test_jacobi_sweep_scales_eigenvector(omega, L):
    """Damped Jacobi on the unit square: the matrix is the 5-point Laplacian
    with diagonal 4 at every free node, and v = sin(k pi x) sin(l pi y) is an
    eigenvector with eigenvalue lam = 4 sin^2(k pi h/2) + 4 sin^2(l pi h/2),
    h = 1/(2N).  With b = 0 one sweep therefore multiplies v by exactly
    1 - omega lam / 4; from x = 0 with b = lam v it gives omega lam v / 4.
    A wrong damping convention or a wrong diagonal changes both."""
    M = mesh_of("square")
    H = mg.Hierarchy(M, L)
    lv = H.levels[L]
    h = 1.0 / (2 * lv.N)
    X, Y = lv.coords[:, 0], lv.coords[:, 1]
    for (k, l) in ((1, 1), (2, 3), (3, 1)):
        v = np.sin(k * np.pi * X) * np.sin(l * np.pi * Y)
        v[~lv.free] = 0.0
        lam = 4 * np.sin(k * np.pi * h / 2) ** 2 + 4 * np.sin(l * np.pi * h / 2) ** 2
        got = mg.jacobi_sweep(H, L, v.copy(), np.zeros(lv.n), omega)
        np.testing.assert_allclose(got, (1 - omega * lam / 4) * v, atol=1e-13)
        got = mg.jacobi_sweep(H, L, np.zeros(lv.n), lam * v, omega)
        np.testing.assert_allclose(got, (omega * lam / 4) * v, atol=1e-13)


def test_jacobi_sweep_keeps_dirichlet_values():
    """Dirichlet unknowns are not smoothed: their values in x pass through."""
    M = mesh_of("random")
    H = mg.Hierarchy(M, 2)
    lv = H.levels[2]
    rng = np.random.default_rng(10)
    x = rng.standard_normal(lv.n)
    got = mg.jacobi_sweep(H, 2, x.copy(), rng.standard_normal(lv.n))
    np.testing.assert_array_equal(got[~lv.free], x[~lv.free])
    assert np.abs(got[lv.free] - x[lv.free]).min() > 0
