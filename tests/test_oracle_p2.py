"""Pins of the P2 / p-multigrid oracle (CPU): element matrices by exact
symbolic integration, assembly invariants, the Galerkin identity against the
(pinned) P1 operator, exact reproduction of quadratic solutions, third-order
L2 convergence, independent colour sets, colour Gauss-Seidel = sequential
Gauss-Seidel, and a level-independent p-multigrid convergence factor."""
import numpy as np
import pytest

from oracle import fem
from oracle import mesh as om
from oracle import multigrid as mg
from oracle import p2
from paper_1805_10167_gb300 import inputs


def mesh_of(name):
    if name == "square":
        return om.MacroMesh(*inputs.unit_square_mesh())
    if name == "annulus":
        return om.MacroMesh(*inputs.annulus_mesh(32, 2))
    return om.MacroMesh(*inputs.random_square_mesh(5, 9))


def _sympy_p2_stiffness(tri):
    """Exact P2 stiffness of a triangle with rational vertices: basis in
    reference coordinates (s, t), gradients by the chain rule, integral over
    the reference triangle times |det J|."""
    sympy = pytest.importorskip("sympy")
    s, t = sympy.symbols("s t")
    (x0, y0), (x1, y1), (x2, y2) = [tuple(sympy.Rational(c) for c in v) for v in tri]
    J = sympy.Matrix([[x1 - x0, x2 - x0], [y1 - y0, y2 - y0]])
    l0, l1, l2 = 1 - s - t, s, t
    phis = [l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1), 4 * l0 * l1, 4 * l1 * l2, 4 * l0 * l2]
    JinvT = J.inv().T
    grads = [JinvT * sympy.Matrix([sympy.diff(p, s), sympy.diff(p, t)]) for p in phis]
    K = np.zeros((6, 6))
    for a in range(6):
        for b in range(a, 6):
            integrand = (grads[a].T * grads[b])[0, 0] * abs(J.det())
            v = sympy.integrate(sympy.integrate(integrand, (t, 0, 1 - s)), (s, 0, 1))
            K[a, b] = K[b, a] = float(v)
    return K


@pytest.mark.parametrize("tri", [[(0, 0), (1, 0), (0, 1)], [(0, 0), (3, 1), (1, 2)],
                                 [("1/2", "1/3"), ("7/5", "-1/4"), ("2/7", "9/8")]])
def test_element_stiffness_equals_exact_integral(tri):
    want = _sympy_p2_stiffness(tri)
    X = np.array([[[float(eval(str(c))) if isinstance(c, str) else float(c) for c in v] for v in tri]])
    got = p2.element_stiffness(X)[0]
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(want).max())


def test_element_stiffness_vertex_opposite_midpoint_zero():
    """A known property of P2: a vertex function and the function of the
    opposite edge's midpoint have orthogonal gradients on any triangle."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((50, 3, 2))
    K = p2.element_stiffness(X)
    np.testing.assert_allclose(K[:, 0, 4], 0.0, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(K[:, 1, 5], 0.0, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(K[:, 2, 3], 0.0, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("name,L", [("square", 1), ("annulus", 1), ("random", 2)])
def test_elements_cover_lattice_and_are_congruent(name, L):
    """Every level-(L+1) lattice point is a node of some level-L element; the
    vertex nodes are the level-L lattice and the midpoints sit halfway."""
    P = p2.P2Level(mesh_of(name), L)
    assert np.array_equal(np.unique(P.elements), np.arange(P.n))
    C = P.coords
    E = P.elements
    for a, b, m in ((0, 1, 3), (1, 2, 4), (0, 2, 5)):
        np.testing.assert_allclose(C[E[:, m]], 0.5 * (C[E[:, a]] + C[E[:, b]]), atol=1e-14)


@pytest.mark.parametrize("name,L", [("square", 2), ("annulus", 1), ("random", 2)])
def test_assembly_invariants(name, L):
    """Symmetry, zero row sums (constants in the kernel of the unconstrained
    operator), positive definiteness on free DoFs, element loop = CSR."""
    P = p2.P2Level(mesh_of(name), L)
    A = p2.assemble(P)
    assert abs(A - A.T).max() < 1e-12
    np.testing.assert_allclose(A @ np.ones(P.n), 0.0, atol=1e-11)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(P.n)
    y = A @ x
    y[~P.free] = 0.0
    np.testing.assert_allclose(p2.apply_element_loop(P, x), y, atol=1e-12 * np.abs(y).max())
    fr = P.free
    ev = np.linalg.eigvalsh(A[fr][:, fr].toarray())
    assert ev.min() > 0


@pytest.mark.parametrize("name,L", [("square", 2), ("annulus", 1), ("random", 2)])
@pytest.mark.parametrize("vark", [False, True])
def test_galerkin_identity_against_p1(name, L, vark):
    """P1 of level L is a subspace of P2 of level L with the embedding P =
    linear interpolation onto the level-(L+1) lattice; with the same
    per-element coefficient the Galerkin product P^T A2 P is the P1 operator
    of level L on free DoFs."""
    M = mesh_of(name)
    N = 1 << L
    k = np.random.default_rng(2).uniform(0.5, 2.0, M.nf * N * N) if vark else None
    PH = p2.P2Hierarchy(M, L, k)
    lv = PH.H1.levels[L]
    fr = lv.free
    A1 = fem.assemble(lv, k)[fr][:, fr].toarray()
    G = (PH.P.T @ PH.A @ PH.P).toarray()[fr][:, fr]
    np.testing.assert_allclose(G, A1, atol=1e-12 * np.abs(A1).max())


@pytest.mark.parametrize("name,L", [("square", 2), ("annulus", 1), ("random", 2)])
def test_quadratic_solution_reproduced_exactly(name, L):
    """u = a quadratic polynomial lies in the P2 space: with its values on the
    boundary and b = M2 (-lap u)_I (constant), the discrete solution equals u
    at every node (to rounding)."""
    PH = p2.P2Hierarchy(mesh_of(name), L)
    u = lambda x, y: 0.3 + 1.1 * x - 0.7 * y + 0.9 * x * x - 0.4 * x * y + 1.7 * y * y
    lap = 2 * 0.9 + 2 * 1.7
    C = PH.p2.coords
    b = p2.load_vector(PH.p2, lambda x, y: -lap + 0.0 * x)
    x = p2.direct_solve(PH, b, u(C[:, 0], C[:, 1]))
    np.testing.assert_allclose(x, u(C[:, 0], C[:, 1]), atol=1e-11)


def test_l2_error_third_order():
    """Manufactured solution sin(pi x) sin(pi y) on the unit square: the P2 L2
    error falls by 8 per level (observed order in [2.8, 3.2])."""
    M = mesh_of("square")
    u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2 * np.pi ** 2 * u(x, y)
    errs = []
    for L in (1, 2, 3, 4):
        PH = p2.P2Hierarchy(M, L)
        x = p2.direct_solve(PH, p2.load_vector(PH.p2, f))
        errs.append(p2.l2_error(PH.p2, x, u))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 2.8) & (orders < 3.2)), orders


@pytest.mark.parametrize("name,L", [("square", 2), ("annulus", 1), ("random", 2), ("random", 1)])
def test_colour_sets_independent_and_cover_free(name, L):
    P = p2.P2Level(mesh_of(name), L)
    adj = p2.adjacency(P)
    sets = p2.gs_sets(P, adj)
    allidx = np.concatenate(sets)
    assert np.array_equal(np.sort(allidx), np.nonzero(P.free)[0])
    for S in sets:
        r, c = adj[S][:, S].nonzero()
        assert np.all(r == c)          # no two unknowns of a set share a micro-triangle


@pytest.mark.parametrize("name,L", [("square", 2), ("random", 1)])
def test_colour_gs_equals_sequential_gs(name, L):
    PH = p2.P2Hierarchy(mesh_of(name), L)
    rng = np.random.default_rng(4)
    x0, b = rng.standard_normal(PH.p2.n), rng.standard_normal(PH.p2.n)
    for forward in (True, False):
        order = np.concatenate([s for s, _ in PH.sets()])
        if not forward:
            order = np.concatenate([s for s, _ in PH.sets()[::-1]])
        want = mg.sequential_gs(PH.A, order, x0.copy(), b)
        got = p2.gs_sweep(PH, x0.copy(), b, forward)
        np.testing.assert_allclose(got, want, atol=1e-13)


def test_pmg_factor_level_independent():
    """p-multigrid with V(2,2) P2 smoothing and a P1 V(3,3) coarse correction
    (annulus): the asymptotic factor (last ratio after 12 cycles) stays below
    0.36 and varies by less than 0.05 over levels 3..5 (it settles at about
    0.336 from level 5 on; levels 1-2 converge faster)."""
    M = mesh_of("annulus")
    rhos = []
    for L in (3, 4, 5):
        PH = p2.P2Hierarchy(M, L)
        b = inputs.uniform_pm1(PH.p2.n, 1234)
        b[~PH.p2.free] = 0.0
        x, hist = p2.solve(PH, np.zeros(PH.p2.n), b, 2, 2, tol=0.0, max_iter=12)
        rhos.append(hist[-1] / hist[-2])
    rhos = np.array(rhos)
    print("p-multigrid factors", rhos)
    assert rhos.max() < 0.36 and rhos.max() - rhos.min() < 0.05, rhos
