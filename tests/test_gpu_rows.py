"""Operator row kernels (apply, residual + norm, Jacobi) and the fused
refinement step (x_new = x + d, then the FP64 residual) on faces wide and
tall enough for several 96-column strips and row blocks (levels 7 and 8),
against the FP64 oracle; FP64 results to 1e-12."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import fem
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu

CASES = [("square", 8), ("random5", 7), ("annulus", 7)]


@pytest.fixture(scope="module")
def pairs():
    cache = {}

    def get(name, L, vark):
        key = (name, L, vark)
        if key not in cache:
            cache[key] = Pair(name, L, vark=vark)
        return cache[key]
    yield get
    for p in cache.values():
        p.close()


@pytest.mark.parametrize("name,L", CASES)
@pytest.mark.parametrize("vark", [False, True])
def test_apply_residual_jacobi_on_multi_strip_faces(pairs, name, L, vark):
    torch = pytest.importorskip("torch")
    P = pairs(name, L, vark)
    hhg = P.hhg
    rng = np.random.default_rng(11)
    for l in (L - 1, L):
        x, b = rng.standard_normal(P.H.levels[l].n), rng.standard_normal(P.H.levels[l].n)
        dx, db = P.to_dev(l, x), P.to_dev(l, b)
        y = P.new(l)
        P.g.apply(l, dx, y)
        assert rel_err(P.from_dev(l, y), fem.apply_element_loop(P.H.levels[l], x, P.H.k[l])) <= FP64_TOL
        r = P.new(l)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        P.g.residual(l, dx, db, r, nrm)
        want = P.H.residual(l, x, b)
        assert rel_err(P.from_dev(l, r), want) <= FP64_TOL
        nw = mg.norm_free(P.H, l, want)
        assert abs(nrm.item() - nw) <= FP64_TOL * nw
        xj = P.to_dev(l, x)
        P.g.smooth(l, xj, db, hhg.JACOBI, sweeps=2, omega=0.6)
        wj = x.copy()
        for _ in range(2):
            mg.jacobi_sweep(P.H, l, wj, b, omega=0.6)
        assert rel_err(P.from_dev(l, xj), wj) <= FP64_TOL
        # FP32 apply against the FP64 oracle: FP32 rounding of inputs and of
        # a 7-term sum, relative to the max norm
        y32 = P.new(l, prec=hhg.F32)
        P.g.apply(l, P.to_dev(l, x, prec=hhg.F32), y32, prec=hhg.F32)
        want = fem.apply_element_loop(P.H.levels[l], x, P.H.k[l])
        assert rel_err(P.from_dev(l, y32, prec=hhg.F32), want) <= 64 * 2.0 ** -24


@pytest.mark.parametrize("vark", [False, True])
def test_refinement_solve_on_multi_strip_faces(vark):
    """The FP32-in-FP64 refinement (fused update + residual, iterate
    ping-ponging through the level's workspace) reaches the FP64 tolerance
    and matches the oracle's FP64 multigrid solution."""
    P = Pair("square", 7, vark=vark)
    lv = P.H.levels[7]
    from paper_1805_10167_gb300 import inputs
    b = inputs.uniform_pm1(lv.n, 1234)
    for max_iter in (100, 3, 4):   # odd and even iteration counts end in either buffer
        x = P.to_dev(7, np.zeros(lv.n))
        st, rep = P.g.solve(7, x, P.to_dev(7, b), mode=P.hhg.SOLVE_IR, nu1=3, nu2=3, tol=1e-10,
                            max_iter=max_iter, raise_on_error=False)
        got = P.from_dev(7, x)
        rn = mg.norm_free(P.H, 7, P.H.residual(7, got, b))
        # the iterate handed back is the one whose residual was reported
        assert abs(rn - rep["r_final"]) <= 1e-6 * rep["r_final"] + 1e-12 * rep["r0"], max_iter
        if max_iter == 100:
            assert st == P.hhg.OK and rep["r_final"] <= 1e-10 * rep["r0"]
            want, _ = mg.solve(P.H, np.zeros(lv.n), b.copy(), 3, 3, tol=1e-12)
            assert rel_err(got, want) < 1e-8
        else:
            assert st == P.hhg.ERR_NOT_CONVERGED and rep["iterations"] == max_iter
    P.close()
