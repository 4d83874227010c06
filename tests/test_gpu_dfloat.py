"""FP64 face kernels in double-float arithmetic (hhg_fp64_arith): the
Gauss-Seidel sweeps, apply and residual rows, V-cycles and solves meet the
FP64 parity bound of 1e-12 against the FP64 oracle on levels where the mode
applies (N > 64); ghost copies stay bit-identical to their owners; the
multigrid and refinement solves reach the FP64 tolerance."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import fem
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pairs():
    cache = {}

    def get(name, L, vark):
        key = (name, L, vark)
        if key not in cache:
            cache[key] = Pair(name, L, vark=vark)
            cache[key].g.fp64_arith(cache[key].hhg.ARITH_DFLOAT)
        return cache[key]
    yield get
    for p in cache.values():
        p.close()


@pytest.mark.parametrize("name,L", [("square", 8), ("random5", 7)])
@pytest.mark.parametrize("vark", [False, True])
def test_dfloat_sweeps_and_rows_match_oracle(pairs, name, L, vark):
    torch = pytest.importorskip("torch")
    P = pairs(name, L, vark)
    hhg = P.hhg
    assert P.g.fp64_arith() == hhg.ARITH_DFLOAT
    rng = np.random.default_rng(5)
    for l in (L - 1, L):
        x0, b = rng.standard_normal(P.H.levels[l].n), rng.standard_normal(P.H.levels[l].n)
        for fwd in (True, False):
            want = x0.copy()
            for _ in range(2):
                mg.gs_sweep(P.H, l, want, b, forward=fwd)
            x = P.to_dev(l, x0)
            P.g.smooth(l, x, P.to_dev(l, b), hhg.GS_FWD if fwd else hhg.GS_BWD, sweeps=2)
            assert rel_err(P.from_dev(l, x), want) <= FP64_TOL, (l, fwd)
        y = P.new(l)
        P.g.apply(l, P.to_dev(l, x0), y)
        assert rel_err(P.from_dev(l, y), fem.apply_element_loop(P.H.levels[l], x0, P.H.k[l])) <= FP64_TOL
        r = P.new(l)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        P.g.residual(l, P.to_dev(l, x0), P.to_dev(l, b), r, nrm)
        want = P.H.residual(l, x0, b)
        assert rel_err(P.from_dev(l, r), want) <= FP64_TOL
        nw = mg.norm_free(P.H, l, want)
        assert abs(nrm.item() - nw) <= FP64_TOL * nw


def test_dfloat_sweep_keeps_ghost_copies_exact(pairs):
    """After double-float sweeps every face boundary slot still holds its
    owner's value bit for bit (Dirichlet values included)."""
    P = pairs("square", 8, False)
    hhg = P.hhg
    l = 8
    rng = np.random.default_rng(9)
    x0, b = rng.standard_normal(P.H.levels[l].n), rng.standard_normal(P.H.levels[l].n)
    x = P.to_dev(l, x0)
    P.g.smooth(l, x, P.to_dev(l, b), hhg.GS_FWD, sweeps=3)
    P.torch.cuda.synchronize()
    c = P.from_dev(l, x)
    I = P.info(l)
    h = x.cpu().numpy()
    N, S = I.N, I.row_stride
    G = P.H.levels[l].face_ids
    for f in range(I.n_faces):
        base = I.f_off + f * I.face_stride
        for t in range(0, N + 1, 7):
            for (i, j) in ((t, 0), (0, t), (N - t, t)):
                assert h[base + j * S + i] == c[G[f][j, i]], (f, i, j)
    fr = P.H.levels[l].free
    assert np.array_equal(c[~fr], x0[~fr])   # Dirichlet values untouched


@pytest.mark.parametrize("vark", [False, True])
def test_dfloat_vcycle_and_solves(pairs, vark):
    P = pairs("square", 8, vark)
    hhg = P.hhg
    L = 8
    rng = np.random.default_rng(3)
    x0, b = rng.standard_normal(P.H.levels[L].n), rng.standard_normal(P.H.levels[L].n)
    x = P.to_dev(L, x0)
    P.g.vcycle(L, x, P.to_dev(L, b), nu1=3, nu2=3)
    assert rel_err(P.from_dev(L, x), mg.vcycle(P.H, L, x0.copy(), b, 3, 3)) <= FP64_TOL
    from paper_1805_10167_gb300 import inputs
    bb = inputs.uniform_pm1(P.H.levels[L].n, 1234)
    want, hist = mg.solve(P.H, np.zeros(P.H.levels[L].n), bb.copy(), 3, 3, tol=1e-12)
    for mode in (hhg.SOLVE_MG, hhg.SOLVE_IR):
        x = P.to_dev(L, np.zeros(P.H.levels[L].n))
        st, rep = P.g.solve(L, x, P.to_dev(L, bb), mode=mode, nu1=3, nu2=3, tol=1e-10)
        assert rep["r_final"] <= 1e-10 * rep["r0"]
        got = P.from_dev(L, x)
        assert mg.norm_free(P.H, L, P.H.residual(L, got, bb)) <= 1.01e-10 * rep["r0"]
        assert rel_err(got, want) < 1e-8
        assert rep["iterations"] <= len(hist) + 1


def test_arith_mode_rejects_bad_values(pairs):
    P = pairs("square", 4, False)
    with pytest.raises(P.hhg.HHGError) as e:
        P.g.fp64_arith(7)
    assert e.value.status == P.hhg.ERR_ARG
