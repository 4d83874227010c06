"""Pins of the Stokes oracle (P1-P1 with PSPG stabilisation, the inexact
Uzawa smoother and the all-at-once V-cycle; Sec. 5.2 and Sec. 4.3) against
closed forms, invariants and brute force:

- B applied to the coordinate fields gives minus the lumped mass (the
  divergence of (x, 0) is 1), B^T applied to a linear pressure gives the
  lumped mass at interior points (integration by parts);
- C annihilates constants everywhere and linear fields at face-interior
  points, and its diagonal there is delta h^2 times the 5-point Laplacian's
  4 on the right-isosceles unit-square lattice;
- the smoother's pressure scaling s equals a brute-force double loop over
  the entries of C + B D_A^-1 B^T;
- the exact solution is a fixed point of both Uzawa step orders;
- a manufactured smooth solution converges at second order in the velocity
  (a dropped term or a wrong sign stops convergence);
- the variable V-cycle's factor is bounded and level independent, and the
  solve reaches the direct solution."""
import numpy as np
import pytest

from oracle import fem
from oracle import mesh as om
from oracle import stokes
from paper_1805_10167_gb300 import inputs


def hierarchy(name="square", L=3, **kw):
    xy, tri = {"square": inputs.unit_square_mesh(), "annulus": inputs.annulus_mesh(32, 2)}[name]
    return stokes.StokesHierarchy(om.MacroMesh(xy, tri), L, **kw)


def lumped_mass(lv):
    area, _ = fem.element_geometry(lv)
    return np.bincount(lv.elements.ravel(), weights=np.repeat(area / 3.0, 3), minlength=lv.n)


@pytest.mark.parametrize("name,L", [("square", 2), ("annulus", 2)])
def test_divergence_of_coordinate_fields(name, L):
    S = hierarchy(name, L)
    lv = S.levels[L]
    B1, B2 = S.B[L]
    x, y = lv.coords[:, 0], lv.coords[:, 1]
    ml = lumped_mass(lv)
    np.testing.assert_allclose(B1 @ x, -ml, atol=1e-14)
    np.testing.assert_allclose(B2 @ y, -ml, atol=1e-14)
    np.testing.assert_allclose(B1 @ y, 0.0, atol=1e-14)
    np.testing.assert_allclose(B2 @ x, 0.0, atol=1e-14)


@pytest.mark.parametrize("name,L", [("square", 3), ("annulus", 2)])
def test_gradient_of_linear_pressure(name, L):
    S = hierarchy(name, L)
    lv = S.levels[L]
    ml = lumped_mass(lv)
    x, y = lv.coords[:, 0], lv.coords[:, 1]
    g1, g2 = S.grad_rows(L, 2.0 * x - 3.0 * y + 1.0)
    fr = lv.free
    np.testing.assert_allclose(g1[fr], 2.0 * ml[fr], rtol=1e-12)
    np.testing.assert_allclose(g2[fr], -3.0 * ml[fr], rtol=1e-12)
    assert np.all(g1[~fr] == 0.0) and np.all(g2[~fr] == 0.0)


def test_stabilisation_invariants_and_scale():
    L, delta = 3, 0.3
    S = hierarchy("square", L, delta=delta)
    lv = S.levels[L]
    C = S.C[L]
    np.testing.assert_allclose(C @ np.ones(lv.n), 0.0, atol=1e-15)
    lin = 0.7 * lv.coords[:, 0] - 1.3 * lv.coords[:, 1]
    inner = lv.kind == 2
    np.testing.assert_allclose((C @ lin)[inner], 0.0, atol=1e-15)
    # unit square of 8 right-isosceles faces with legs 1/2: micro hypotenuse^2 = 0.5 / N^2
    h2 = 0.5 / lv.N ** 2
    np.testing.assert_allclose(C.diagonal()[inner], delta * h2 * 4.0, rtol=1e-13)


def test_pressure_scaling_brute_force():
    L = 2
    S = hierarchy("annulus", L)
    lv = S.levels[L]
    A = S.H.A[L].toarray()
    B1, B2 = (B.toarray() for B in S.B[L])
    C = S.C[L].toarray()
    want = np.zeros(lv.n)
    for q in range(lv.n):
        acc = C[q, q]
        for j in range(lv.n):
            if lv.free[j]:
                acc += (B1[q, j] ** 2 + B2[q, j] ** 2) / A[j, j]
        want[q] = acc
    np.testing.assert_allclose(S.s[L], want, rtol=1e-13)


def random_rhs(S, L, seed=0):
    lv = S.levels[L]
    rng = np.random.default_rng(seed)
    f1, f2, g = rng.uniform(-1, 1, lv.n), rng.uniform(-1, 1, lv.n), rng.uniform(-1, 1, lv.n)
    f1[~lv.free] = 0.0
    f2[~lv.free] = 0.0
    g -= g.mean()
    return f1, f2, g


@pytest.mark.parametrize("name", ["square", "annulus"])
def test_direct_solution_is_smoother_fixed_point(name):
    L = 2
    S = hierarchy(name, L)
    f1, f2, g = random_rhs(S, L)
    u1, u2, p = S.direct_solve(f1, f2, g)
    assert S.norm(L, *S.residual(L, u1, u2, p, f1, f2, g)) < 1e-12 * np.sqrt(f1 @ f1 + f2 @ f2 + g @ g)
    assert abs(p.sum()) < 1e-10
    for forward in (True, False):
        v1, v2, q = u1.copy(), u2.copy(), p.copy()
        S.uzawa_step(L, v1, v2, q, f1, f2, g, forward)
        scale = np.abs(np.concatenate([u1, u2, p])).max()
        assert np.abs(np.concatenate([v1 - u1, v2 - u2, q - p])).max() < 1e-12 * scale


def manufactured():
    """u = curl psi, psi = x^2 (1-x)^2 y^2 (1-y)^2 (zero on the boundary of the
    unit square, divergence free), p = x^2 - 1/3 (zero mean); f = -lap u +
    grad p, derived by hand."""
    def a(t):  # t^2 (1-t)^2 and derivatives
        return t ** 2 * (1 - t) ** 2

    def a1(t):
        return 2 * t * (1 - t) * (1 - 2 * t)

    def a2(t):
        return 2 - 12 * t + 12 * t ** 2

    def a3(t):
        return -12 + 24 * t

    def u1(x, y):
        return a(x) * a1(y)

    def u2(x, y):
        return -a1(x) * a(y)

    def f1(x, y):   # -lap u1 + dp/dx, u1 = a(x) a'(y)
        return -(a2(x) * a1(y) + a(x) * a3(y)) + 2 * x

    def f2(x, y):   # -lap u2 + dp/dy, u2 = -a'(x) a(y)
        return (a3(x) * a(y) + a1(x) * a2(y))

    def p(x, y):
        return x ** 2 - 1.0 / 3.0
    return u1, u2, p, f1, f2


def test_manufactured_solution_converges():
    u1e, u2e, pe, f1f, f2f = manufactured()
    errs, perrs = [], []
    for L in (3, 4, 5):
        S = hierarchy("square", L)
        lv = S.levels[L]
        f1, f2 = fem.load_vector(lv, f1f), fem.load_vector(lv, f2f)
        # PSPG right-hand side: -delta sum_T h_T^2 integral_T f . grad(phi_q), one-point rule
        area, G = fem.element_geometry(lv)
        cen = lv.coords[lv.elements].mean(axis=1)
        h2 = stokes.longest_edge_sq(lv)
        fc = np.stack([f1f(cen[:, 0], cen[:, 1]), f2f(cen[:, 0], cen[:, 1])], axis=1)
        loc = -S.delta * (h2 * area)[:, None] * np.einsum("ed,edk->ek", fc, G)
        g = np.bincount(lv.elements.ravel(), weights=loc.ravel(), minlength=lv.n)
        g -= g.mean()
        u1, u2, p = S.direct_solve(f1, f2, g)
        errs.append(np.hypot(fem.l2_error(lv, u1, u1e), fem.l2_error(lv, u2, u2e)))
        pm = p - (fem.mass_matrix(lv) @ p).sum() / fem.mass_matrix(lv).sum()
        perrs.append(fem.l2_error(lv, pm, pe))
    ratios = [errs[k] / errs[k + 1] for k in range(2)]
    assert min(ratios) > 3.2 and ratios[1] > ratios[0] - 0.1, (errs, ratios)   # -> 4 (second order)
    assert perrs[2] < perrs[0] / 2.0, perrs


@pytest.mark.parametrize("name,levels,bound", [("square", (3, 4, 5, 6), 0.5), ("annulus", (3, 4), 0.6)])
def test_vcycle_factor_bounded_and_level_independent(name, levels, bound):
    rates = []
    for L in levels:
        S = hierarchy(name, L)
        f1, f2, g = random_rhs(S, L)
        lv = S.levels[L]
        u1, u2, p = np.zeros(lv.n), np.zeros(lv.n), np.zeros(lv.n)
        h = np.array(S.solve(u1, u2, p, f1, f2, g, tol=1e-8, max_iter=60))
        rates.append((h[-1] / h[0]) ** (1.0 / (len(h) - 1)))
    assert max(rates) < bound, rates
    assert max(rates) - min(rates) < 0.05, rates


@pytest.mark.parametrize("coarse", [0, 1])
def test_solve_reaches_direct_solution(coarse):
    L = 3
    S = hierarchy("square", L, coarse=coarse)
    f1, f2, g = random_rhs(S, L, seed=3)
    lv = S.levels[L]
    u1, u2, p = np.zeros(lv.n), np.zeros(lv.n), np.zeros(lv.n)
    h = S.solve(u1, u2, p, f1, f2, g, tol=1e-11, max_iter=80)
    assert h[-1] <= 1e-11 * h[0]
    e1, e2, ep = S.direct_solve(f1, f2, g)
    scale = np.abs(np.concatenate([e1, e2])).max()
    assert np.abs(np.concatenate([u1 - e1, u2 - e2])).max() < 1e-8 * scale
    assert np.abs((p - p.mean()) - (ep - ep.mean())).max() < 1e-8 * np.abs(ep).max()
