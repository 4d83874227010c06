"""Stokes flow on the GPU (P1-P1 with PSPG stabilisation, inexact Uzawa
smoother, all-at-once V-cycle; Sec. 5.2, Sec. 4.3) through the C-ABI against
the Stokes oracle: operator, residual and norm, the smoother's pressure
scaling, Uzawa steps in both orders, one V-cycle (every result at the FP64
bound 1e-12), and solves with the oracle's cycle count."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, macro_mesh, rel_err
from oracle import mesh as om
from oracle import stokes

pytestmark = pytest.mark.gpu

CASES = [("square", 1), ("square", 4), ("annulus", 3), ("annulus16", 2), ("random5", 3), ("random11", 2)]


class StokesPair:
    def __init__(self, name, L, coarse=0, delta=0.3, omega=0.4, nvel=2):
        import torch
        from paper_1805_10167_gb300 import hhg
        self.torch, self.hhg, self.L = torch, hhg, L
        xy, tri = macro_mesh(name)
        self.S = stokes.StokesHierarchy(om.MacroMesh(xy, tri), L, delta, omega, nvel, coarse)
        self.g = hhg.Mesh(xy, tri, L)
        self.g.stokes_setup(delta, omega, nvel, coarse)
        self.rng = np.random.default_rng(7 + L)

    def n(self, l):
        return self.S.levels[l].n

    def new(self, l):
        return self.torch.zeros(self.g.info(l).vec_len, dtype=self.torch.float64, device="cuda")

    def to_dev(self, l, c):
        out = self.new(l)
        self.g.from_canonical(l, self.torch.tensor(c, dtype=self.torch.float64, device="cuda"), out)
        return out

    def from_dev(self, l, v):
        out = self.torch.zeros(self.n(l), dtype=self.torch.float64, device="cuda")
        self.g.to_canonical(l, v, out)
        self.torch.cuda.synchronize()
        return out.cpu().numpy()

    def rhs(self, l):
        lv = self.S.levels[l]
        f1, f2, g = (self.rng.standard_normal(lv.n) for _ in range(3))
        f1[~lv.free] = 0.0
        f2[~lv.free] = 0.0
        g -= g.mean()
        return f1, f2, g


@pytest.fixture(scope="module")
def pairs():
    cache = {}

    def get(name, L, coarse=0, nvel=2):
        if (name, L, coarse, nvel) not in cache:
            cache[(name, L, coarse, nvel)] = StokesPair(name, L, coarse, nvel=nvel)
        return cache[(name, L, coarse, nvel)]
    yield get
    for p in cache.values():
        p.g.close()


@pytest.mark.parametrize("name,L", CASES)
def test_stokes_apply_and_residual_parity(pairs, name, L):
    torch = pytest.importorskip("torch")
    P = pairs(name, L)
    for l in range(L + 1):
        u1, u2, p = (P.rng.standard_normal(P.n(l)) for _ in range(3))
        d = [P.to_dev(l, v) for v in (u1, u2, p)]
        y = [P.new(l) for _ in range(3)]
        P.g.stokes_apply(l, *d, *y)
        want = P.S.apply(l, u1, u2, p)
        for got, w in zip(y, want):
            assert rel_err(P.from_dev(l, got), w) <= FP64_TOL, l
        f1, f2, g = P.rhs(l)
        r = [P.new(l) for _ in range(3)]
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        P.g.stokes_residual(l, *d, *(P.to_dev(l, v) for v in (f1, f2, g)), *r, nrm)
        want = P.S.residual(l, u1, u2, p, f1, f2, g)
        for got, w in zip(r, want):
            assert rel_err(P.from_dev(l, got), w) <= FP64_TOL, l
        wn = P.S.norm(l, *want)
        assert abs(nrm.item() - wn) <= FP64_TOL * wn


@pytest.mark.parametrize("name,L", CASES)
def test_stokes_pressure_scaling_parity(pairs, name, L):
    P = pairs(name, L)
    for l in range(1, L + 1):
        s = P.new(l)
        P.g.stokes_diag(l, s)
        assert rel_err(P.from_dev(l, s), 1.0 / P.S.s[l]) <= FP64_TOL, l


@pytest.mark.parametrize("name,L,nvel", [c + (2,) for c in CASES] + [("annulus", 3, 1), ("random5", 3, 3)])
def test_stokes_uzawa_steps_parity(pairs, name, L, nvel):
    P = pairs(name, L, nvel=nvel)
    f1, f2, g = P.rhs(L)
    fd = [P.to_dev(L, v) for v in (f1, f2, g)]
    for forward in (True, False):
        u1, u2, p = (P.rng.standard_normal(P.n(L)) for _ in range(3))
        lv = P.S.levels[L]
        u1[~lv.free] = 0.0
        u2[~lv.free] = 0.0
        d = [P.to_dev(L, v) for v in (u1, u2, p)]
        P.g.stokes_smooth(L, *d, *fd, forward=forward, steps=2)
        w = [u1.copy(), u2.copy(), p.copy()]
        for _ in range(2):
            P.S.uzawa_step(L, *w, f1, f2, g, forward)
        for got, want in zip(d, w):
            assert rel_err(P.from_dev(L, got), want) <= FP64_TOL, forward


@pytest.mark.parametrize("name,L,nvel", [c + (2,) for c in CASES] + [("square", 4, 1)])
def test_stokes_vcycle_parity(pairs, name, L, nvel):
    P = pairs(name, L, nvel=nvel)
    f1, f2, g = P.rhs(L)
    lv = P.S.levels[L]
    u1, u2, p = (P.rng.standard_normal(lv.n) for _ in range(3))
    u1[~lv.free] = 0.0
    u2[~lv.free] = 0.0
    d = [P.to_dev(L, v) for v in (u1, u2, p)]
    P.g.stokes_vcycle(L, *d, *(P.to_dev(L, v) for v in (f1, f2, g)), 2, 2)
    w = [u1.copy(), u2.copy(), p.copy()]
    P.S.vcycle(L, *w, f1, f2, g, 2, 2)
    for got, want in zip(d, w):
        assert rel_err(P.from_dev(L, got), want) <= FP64_TOL


@pytest.mark.parametrize("name,L,coarse", [("square", 4, 0), ("annulus", 3, 0), ("annulus16", 3, 1),
                                           ("random5", 3, 1)])
def test_stokes_solve_matches_oracle(pairs, name, L, coarse):
    P = pairs(name, L, coarse)
    f1, f2, g = P.rhs(L)
    z = np.zeros(P.n(L))
    d = [P.to_dev(L, z) for _ in range(3)]
    fd = [P.to_dev(L, v) for v in (f1, f2, g)]
    st, rep = P.g.stokes_solve(L, *d, *fd, tol=1e-8, max_iter=80)
    w = [z.copy(), z.copy(), z.copy()]
    hist = P.S.solve(*w, f1, f2, g, tol=1e-8, max_iter=80)
    assert rep["iterations"] == len(hist) - 1
    assert rep["r_final"] <= 1e-8 * rep["r0"]
    # rounding differences stay at the FP64 bound relative to the initial residual
    np.testing.assert_allclose(rep["history"], hist, rtol=0, atol=FP64_TOL * hist[0])
    got = [P.from_dev(L, v) for v in d]
    assert P.S.norm(L, *P.S.residual(L, *got, f1, f2, g)) <= 1.01e-8 * hist[0]
    # replays of the captured cycle give the same iterate
    d2 = [P.to_dev(L, z) for _ in range(3)]
    P.g.stokes_solve(L, *d2, *fd, tol=1e-8, max_iter=80)
    for a, b in zip(d, d2):
        assert P.torch.equal(a, b)


def test_stokes_argument_errors():
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.unit_square_mesh()
    g = hhg.Mesh(xy, tri, 3)
    v = [torch.zeros(g.info(3).vec_len, dtype=torch.float64, device="cuda") for _ in range(6)]
    with pytest.raises(hhg.HHGError) as e:          # not set up
        g.stokes_vcycle(3, *v)
    assert e.value.status == hhg.ERR_ARG
    for bad in ({"delta": 0.0}, {"omega": -1.0}, {"nvel": 0}, {"coarse_level": 3}):
        with pytest.raises(hhg.HHGError) as e:
            g.stokes_setup(**bad)
        assert e.value.status == hhg.ERR_ARG
    g.stokes_setup(coarse_level=1)
    w = [torch.zeros(g.info(1).vec_len, dtype=torch.float64, device="cuda") for _ in range(6)]
    with pytest.raises(hhg.HHGError) as e:          # below the coarse level
        g.stokes_vcycle(0, *[torch.zeros(g.info(0).vec_len, dtype=torch.float64, device="cuda") for _ in range(6)])
    assert e.value.status == hhg.ERR_ARG
    with pytest.raises(hhg.HHGError) as e:          # no smoothing on the coarse level
        g.stokes_smooth(1, *w)
    assert e.value.status == hhg.ERR_ARG
    with pytest.raises(hhg.HHGError) as e:
        g.stokes_solve(1, *w)
    assert e.value.status == hhg.ERR_ARG
    k = torch.ones(8 * 64, dtype=torch.float64, device="cuda")   # 8 faces x 8^2 elements
    g.set_coefficient(k)
    with pytest.raises(hhg.HHGError) as e:          # k = 1 only
        g.stokes_vcycle(3, *v)
    assert e.value.status == hhg.ERR_ARG
    g.close()


FP32_CYCLE_TOL = 1e-5   # one FP32 cycle against the FP64 one: FP32 roundoff (6e-8) times the cycle's growth


@pytest.mark.parametrize("name,L,coarse", [("square", 4, 0), ("annulus", 3, 0), ("random5", 3, 1)])
def test_stokes_mixed_precision_step_and_solve(pairs, name, L, coarse):
    """One refinement step (FP64 residual, FP32 variable V-cycle from zero,
    FP64 update) against the oracle's FP64 cycle from the same iterate, at the
    stated FP32 bound; then the mixed solve reaches the FP64 tolerance 1e-10
    with at most two steps more than the oracle's FP64 cycles."""
    P = pairs(name, L, coarse)
    f1, f2, g = P.rhs(L)
    fd = [P.to_dev(L, v) for v in (f1, f2, g)]
    lv = P.S.levels[L]
    u1, u2, p = (P.rng.standard_normal(lv.n) for _ in range(3))
    u1[~lv.free] = 0.0
    u2[~lv.free] = 0.0
    d = [P.to_dev(L, v) for v in (u1, u2, p)]
    st, rep = P.g.stokes_solve_ir(L, *d, *fd, tol=0.0, max_iter=1, raise_on_error=False)
    assert rep["iterations"] == 1
    w = [u1.copy(), u2.copy(), p.copy()]
    P.S.vcycle(L, *w, f1, f2, g, 2, 2)
    errs = [rel_err(P.from_dev(L, got), want) for got, want in zip(d, w)]
    print(f"{name} level {L}: one mixed-precision step against the FP64 cycle, max relative error {max(errs):.1e}")
    assert max(errs) <= FP32_CYCLE_TOL
    z = np.zeros(P.n(L))
    d = [P.to_dev(L, z) for _ in range(3)]
    st, rep = P.g.stokes_solve_ir(L, *d, *fd, tol=1e-10, max_iter=80)
    hist = P.S.solve(*[z.copy() for _ in range(3)], f1, f2, g, tol=1e-10, max_iter=80)
    assert rep["r_final"] <= 1e-10 * rep["r0"]
    assert rep["iterations"] <= len(hist) - 1 + 2
    got = [P.from_dev(L, v) for v in d]
    assert P.S.norm(L, *P.S.residual(L, *got, f1, f2, g)) <= 1.01e-10 * hist[0]
