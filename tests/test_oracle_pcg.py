"""Pins of the oracle's preconditioned conjugate gradients (oracle/krylov.pcg)
and of the symmetric V-cycle as its preconditioner (Sec. 4.3: multigrid as a
preconditioner inside a Krylov solver).  Each pin rests on something other
than the oracle itself: SciPy's CG, a dense solve, the CG minimisation
property, the symmetry of the V-cycle as a linear map."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import krylov
from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs


def _problem(L, name="annulus"):
    xy, tri = inputs.annulus_mesh(32, 2) if name == "annulus" else inputs.unit_square_mesh()
    H = mg.Hierarchy(om.MacroMesh(xy, tri), L)
    lv = H.levels[L]
    b = inputs.uniform_pm1(lv.n, 7)
    b[~lv.free] = 0
    return H, lv, b


def _embed(v, fr):
    out = np.zeros(fr.size)
    out[fr] = v
    return out


def test_identity_preconditioner_matches_scipy_cg():
    """With M = I the iterates are plain CG's: after k steps they equal
    SciPy's conjugate gradients after k steps on the assembled free block."""
    H, lv, b = _problem(2)
    fr = lv.free
    Af = H.A[2][fr][:, fr].tocsr()
    for k in (1, 4, 9):
        x, hist, steps = krylov.pcg(lambda v: H.apply(2, v), lambda v: v.copy(), b, np.zeros(lv.n), fr,
                                    tol=0.0, max_iter=k)
        assert steps == k
        want, _ = spla.cg(Af, b[fr], x0=np.zeros(fr.sum()), rtol=0.0, atol=0.0, maxiter=k)
        np.testing.assert_allclose(x[fr], want, rtol=1e-9, atol=1e-12)


def test_exact_preconditioner_converges_in_one_step():
    H, lv, b = _problem(2)
    fr = lv.free
    Af = H.A[2][fr][:, fr].toarray()
    exact = lambda v: _embed(np.linalg.solve(Af, v[fr]), fr)
    x, hist, steps = krylov.pcg(lambda v: H.apply(2, v), exact, b, np.zeros(lv.n), fr, tol=1e-10)
    assert steps == 1
    np.testing.assert_allclose(x[fr], np.linalg.solve(Af, b[fr]), rtol=1e-10, atol=1e-13)


def test_energy_norm_error_decreases_with_vcycle_preconditioner():
    """CG minimises the A-norm of the error over the Krylov space, so it
    never grows from one step to the next; the exact solution is a dense solve."""
    H, lv, b = _problem(3)
    fr = lv.free
    Af = H.A[3][fr][:, fr].toarray()
    xs = np.linalg.solve(Af, b[fr])
    pre = lambda v: mg.vcycle(H, 3, np.zeros(lv.n), v, 1, 1)
    errs = []
    for k in range(1, 7):
        x, _, _ = krylov.pcg(lambda v: H.apply(3, v), pre, b, np.zeros(lv.n), fr, tol=0.0, max_iter=k)
        e = x[fr] - xs
        errs.append(float(e @ Af @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))
    assert errs[-1] < 1e-5 * errs[0]   # V(1,1)-PCG: about 0.1 per step in energy


def test_symmetric_vcycle_is_a_symmetric_preconditioner():
    """V(nu, nu) with forward Gauss-Seidel before and backward after and an
    exact coarse solve is a symmetric linear map of its right-hand side:
    <M u, v> = <u, M v> over the free DoFs (what makes it a CG preconditioner)."""
    H, lv, b = _problem(3, "square")
    fr = lv.free
    rng = np.random.default_rng(2)
    for nu in ((1, 1), (2, 2)):
        u, v = _embed(rng.standard_normal(fr.sum()), fr), _embed(rng.standard_normal(fr.sum()), fr)
        Mu = mg.vcycle(H, 3, np.zeros(lv.n), u, *nu)
        Mv = mg.vcycle(H, 3, np.zeros(lv.n), v, *nu)
        a, c = float(Mu[fr] @ v[fr]), float(u[fr] @ Mv[fr])
        assert abs(a - c) <= 1e-10 * max(abs(a), abs(c))


def test_pcg_beats_plain_multigrid_in_cycles():
    """On the annulus at level 5 the V(3,3)-preconditioned CG reaches 1e-10
    in no more preconditioner applications than V(3,3) multigrid needs cycles."""
    H, lv, b = _problem(5)
    fr = lv.free
    pre = lambda v: mg.vcycle(H, 5, np.zeros(lv.n), v, 3, 3)
    x, hist, steps = krylov.pcg(lambda v: H.apply(5, v), pre, b, np.zeros(lv.n), fr, tol=1e-10)
    assert hist[-1] <= 1e-10 * hist[0]
    _, mg_hist = mg.solve(H, np.zeros(lv.n), b.copy(), 3, 3, tol=1e-10)
    assert steps <= len(mg_hist) - 1


def test_flexible_beta_equals_standard_beta_for_a_fixed_preconditioner():
    """For a fixed symmetric preconditioner z_{k+1}.r_k = 0 in exact
    arithmetic, so the flexible (Polak-Ribiere) and the standard
    (Fletcher-Reeves) beta give the same iterates up to rounding."""
    H, lv, b = _problem(4)
    fr = lv.free
    pre = lambda v: mg.vcycle(H, 4, np.zeros(lv.n), v, 2, 2)
    for k in (2, 5):
        xs, _, _ = krylov.pcg(lambda v: H.apply(4, v), pre, b, np.zeros(lv.n), fr, tol=0.0, max_iter=k)
        xf, _, _ = krylov.pcg(lambda v: H.apply(4, v), pre, b, np.zeros(lv.n), fr, tol=0.0, max_iter=k,
                              flexible=True)
        np.testing.assert_allclose(xf[fr], xs[fr], rtol=1e-9, atol=1e-12)


def test_flexible_cg_with_a_single_precision_preconditioner_reaches_fp64_tolerance():
    """A V-cycle whose result is rounded to FP32 (a preconditioner that
    varies with its input's rounding, as the FP32 V-cycle does) inside
    flexible CG still reaches 1e-10 in FP64, within a step or two of the
    exact-arithmetic step count."""
    H, lv, b = _problem(5)
    fr = lv.free

    def pre32(v):
        s = np.abs(v).max()
        z = mg.vcycle(H, 5, np.zeros(lv.n), (v / s).astype(np.float32).astype(np.float64), 3, 3)
        return z.astype(np.float32).astype(np.float64) * s
    x, hist, steps = krylov.pcg(lambda v: H.apply(5, v), pre32, b, np.zeros(lv.n), fr, tol=1e-10,
                                flexible=True)
    assert hist[-1] <= 1e-10 * hist[0]
    r = b - H.apply(5, x)
    assert np.linalg.norm(r[fr]) <= 1.01e-10 * hist[0]
    pre = lambda v: mg.vcycle(H, 5, np.zeros(lv.n), v, 3, 3)
    _, _, steps64 = krylov.pcg(lambda v: H.apply(5, v), pre, b, np.zeros(lv.n), fr, tol=1e-10)
    assert steps <= steps64 + 2
