"""Multigrid-preconditioned conjugate gradients (hhg_solve mode
HHG_SOLVE_PCG) against the oracle's PCG on the same seeded problems: the
same iterates step by step, the same step count to 1e-10, and the FP64
tolerance reached on faces with several strips."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import krylov
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu


def _oracle_pcg(P, L, b, nu, max_iter, tol):
    lv = P.H.levels[L]
    pre = lambda v: mg.vcycle(P.H, L, np.zeros(lv.n), v, *nu)
    return krylov.pcg(lambda v: P.H.apply(L, v), pre, b, np.zeros(lv.n), lv.free, tol=tol, max_iter=max_iter)


@pytest.mark.parametrize("name,L,vark", [("square", 5, False), ("annulus", 5, False), ("annulus", 4, True),
                                         ("random5", 4, False)])
def test_pcg_iterates_match_oracle(name, L, vark):
    P = Pair(name, L, vark=vark)
    hhg = P.hhg
    lv = P.H.levels[L]
    from paper_1805_10167_gb300 import inputs
    b = inputs.uniform_pm1(lv.n, 1234)
    b[~lv.free] = 0.0
    for k in (1, 2, 4):   # after k steps: same iterate (no stop, tolerance 0)
        want, hist, steps = _oracle_pcg(P, L, b, (2, 2), k, 0.0)
        x = P.to_dev(L, np.zeros(lv.n))
        st, rep = P.g.solve(L, x, P.to_dev(L, b), mode=hhg.SOLVE_PCG, nu1=2, nu2=2, tol=0.0, max_iter=k,
                            raise_on_error=False)
        assert st == hhg.ERR_NOT_CONVERGED and rep["iterations"] == k
        # the preconditioned system is well conditioned (V-cycle contraction
        # about 0.1): rounding differences grow at most linearly in k
        assert rel_err(P.from_dev(L, x), want) <= 4 * k * FP64_TOL, k
    want, hist, steps = _oracle_pcg(P, L, b, (3, 3), 100, 1e-10)
    x = P.to_dev(L, np.zeros(lv.n))
    st, rep = P.g.solve(L, x, P.to_dev(L, b), mode=hhg.SOLVE_PCG, nu1=3, nu2=3, tol=1e-10)
    assert rep["iterations"] == steps
    assert rep["r_final"] <= 1e-10 * rep["r0"]
    got = P.from_dev(L, x)
    assert mg.norm_free(P.H, L, P.H.residual(L, got, b)) <= 1.01e-10 * rep["r0"]
    np.testing.assert_allclose(rep["history"][:3], hist[:3], rtol=1e-9)
    P.close()


def test_pcg_reaches_tolerance_on_multi_strip_faces_in_fewer_cycles_than_mg():
    P = Pair("square", 8)
    hhg = P.hhg
    L = 8
    lv = P.H.levels[L]
    from paper_1805_10167_gb300 import inputs
    b = inputs.uniform_pm1(lv.n, 99)
    x = P.to_dev(L, np.zeros(lv.n))
    st, rep = P.g.solve(L, x, P.to_dev(L, b), mode=hhg.SOLVE_PCG, nu1=3, nu2=3, tol=1e-10)
    assert rep["r_final"] <= 1e-10 * rep["r0"]
    got = P.from_dev(L, x)
    assert mg.norm_free(P.H, L, P.H.residual(L, got, b)) <= 1.01e-10 * rep["r0"]
    xm = P.to_dev(L, np.zeros(lv.n))
    st, rep_mg = P.g.solve(L, xm, P.to_dev(L, b), mode=hhg.SOLVE_MG, nu1=3, nu2=3, tol=1e-10)
    assert rep["iterations"] <= rep_mg["iterations"]
    assert rel_err(got, P.from_dev(L, xm)) < 1e-8
    P.close()


@pytest.mark.parametrize("name,L,vark", [("square", 7, False), ("annulus", 6, True)])
def test_flexible_cg_with_fp32_vcycle_reaches_fp64_tolerance(name, L, vark):
    """Flexible CG (FP64 vectors, operator and dots) preconditioned by one
    FP32 V(3,3) cycle reaches the 1e-10 FP64 residual, checked by the
    oracle, in at most two steps more than FP64-preconditioned CG."""
    P = Pair(name, L, vark=vark)
    hhg = P.hhg
    lv = P.H.levels[L]
    from paper_1805_10167_gb300 import inputs
    b = inputs.uniform_pm1(lv.n, 4321)
    b[~lv.free] = 0.0
    x = P.to_dev(L, np.zeros(lv.n))
    st, rep = P.g.solve(L, x, P.to_dev(L, b), mode=hhg.SOLVE_FPCG, nu1=3, nu2=3, tol=1e-10)
    got = P.from_dev(L, x)
    assert mg.norm_free(P.H, L, P.H.residual(L, got, b)) <= 1.01e-10 * rep["r0"]
    want, hist, steps = _oracle_pcg(P, L, b, (3, 3), 100, 1e-12)
    assert rel_err(got, want) < 1e-8
    x64 = P.to_dev(L, np.zeros(lv.n))
    st, rep64 = P.g.solve(L, x64, P.to_dev(L, b), mode=hhg.SOLVE_PCG, nu1=3, nu2=3, tol=1e-10)
    assert rep["iterations"] <= rep64["iterations"] + 2
    P.close()
