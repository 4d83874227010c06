"""P2 elements and p-multigrid on the GPU (through the C-ABI) against the
P2 oracle: operator, residual and norm, colour Gauss-Seidel sweeps, one
p-multigrid cycle (all at the FP64 bound 1e-12), and solves to 1e-10 with
the oracle's cycle count.  A P2 vector of level L is a level-(L+1) vector."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, macro_mesh, rel_err
from oracle import mesh as om
from oracle import p2

pytestmark = pytest.mark.gpu

CASES = [("square", 1), ("square", 3), ("annulus", 2), ("annulus16", 3), ("random5", 2), ("random11", 3)]


class P2Pair:
    def __init__(self, name, L):
        import torch
        from paper_1805_10167_gb300 import hhg
        self.torch, self.hhg, self.L = torch, hhg, L
        xy, tri = macro_mesh(name)
        self.PH = p2.P2Hierarchy(om.MacroMesh(xy, tri), L)
        self.g = hhg.Mesh(xy, tri, L + 1)
        self.info = self.g.info(L + 1)
        self.rng = np.random.default_rng(17 + L)

    def to_dev(self, c):
        t = self.torch
        out = t.zeros(self.info.vec_len, dtype=t.float64, device="cuda")
        self.g.from_canonical(self.L + 1, t.tensor(c, dtype=t.float64, device="cuda"), out)
        return out

    def from_dev(self, v):
        t = self.torch
        out = t.zeros(self.info.n_nodes, dtype=t.float64, device="cuda")
        self.g.to_canonical(self.L + 1, v, out)
        t.cuda.synchronize()
        return out.cpu().numpy()

    def random(self):
        return self.rng.standard_normal(self.PH.p2.n)


@pytest.fixture(scope="module")
def pairs():
    cache = {}

    def get(name, L):
        if (name, L) not in cache:
            cache[(name, L)] = P2Pair(name, L)
        return cache[(name, L)]
    yield get
    for p in cache.values():
        p.g.close()


@pytest.mark.parametrize("name,L", CASES)
def test_p2_apply_and_residual_parity(pairs, name, L):
    torch = pytest.importorskip("torch")
    P = pairs(name, L)
    assert P.info.n_nodes == P.PH.p2.n
    x, b = P.random(), P.random()
    xd = P.to_dev(x)
    y = torch.zeros_like(xd)
    P.g.p2_apply(L, xd, y)
    want = p2.apply_element_loop(P.PH.p2, x)
    assert rel_err(P.from_dev(y), want) <= FP64_TOL
    r = torch.zeros_like(xd)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.g.p2_residual(L, xd, P.to_dev(b), r, nrm)
    want = P.PH.residual(x, b)
    assert rel_err(P.from_dev(r), want) <= FP64_TOL
    assert abs(nrm.item() - P.PH.norm(want)) <= FP64_TOL * P.PH.norm(want)


@pytest.mark.parametrize("name,L", CASES)
def test_p2_gauss_seidel_parity(pairs, name, L):
    P = pairs(name, L)
    x, b = P.random(), P.random()
    for smoother, forward in ((P.hhg.GS_FWD, True), (P.hhg.GS_BWD, False)):
        xd = P.to_dev(x)
        P.g.p2_smooth(L, xd, P.to_dev(b), smoother=smoother, sweeps=2)
        want = x.copy()
        for _ in range(2):
            p2.gs_sweep(P.PH, want, b, forward)
        assert rel_err(P.from_dev(xd), want) <= FP64_TOL, forward


@pytest.mark.parametrize("name,L", CASES)
def test_p2_cycle_parity(pairs, name, L):
    P = pairs(name, L)
    x, b = P.random(), P.random()
    xd = P.to_dev(x)
    P.g.p2_cycle(L, xd, P.to_dev(b), nu1=2, nu2=2, nu1c=3, nu2c=3)
    want = p2.pmg_cycle(P.PH, x.copy(), b, 2, 2, 3, 3)
    assert rel_err(P.from_dev(xd), want) <= FP64_TOL


@pytest.mark.parametrize("name,L", [("square", 3), ("annulus", 3), ("random11", 3)])
def test_p2_solve_matches_oracle(pairs, name, L):
    P = pairs(name, L)
    b = P.random()
    b[~P.PH.p2.free] = 0.0
    xd = P.to_dev(np.zeros(P.PH.p2.n))
    st, rep = P.g.p2_solve(L, xd, P.to_dev(b))
    _, hist = p2.solve(P.PH, np.zeros(P.PH.p2.n), b.copy(), 2, 2, tol=1e-10)
    assert rep["iterations"] == len(hist) - 1
    got = P.from_dev(xd)
    assert P.PH.norm(P.PH.residual(got, b)) <= 1.01e-10 * P.PH.norm(b)
    exact = p2.direct_solve(P.PH, b)
    assert rel_err(got, exact) < 1e-8
    # replays of the captured cycle give the same iterate
    xd2 = P.to_dev(np.zeros(P.PH.p2.n))
    P.g.p2_solve(L, xd2, P.to_dev(b))
    assert P.torch.equal(xd, xd2)


def test_p2_argument_errors(pairs):
    torch = pytest.importorskip("torch")
    P = pairs("square", 1)
    x = P.to_dev(P.random())
    for bad in (0, 2):       # level 0 has no P2 space here; level 2 needs a level-3 lattice
        with pytest.raises(P.hhg.HHGError) as e:
            P.g.p2_apply(bad, x, x)
        assert e.value.status == P.hhg.ERR_ARG
    with pytest.raises(P.hhg.HHGError) as e:
        P.g.p2_smooth(1, x, x, smoother=P.hhg.JACOBI)
    assert e.value.status == P.hhg.ERR_ARG
    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.unit_square_mesh()
    g = hhg.Mesh(xy, tri, 2)
    k = torch.ones(8 * 16, dtype=torch.float64, device="cuda")   # 8 faces x 4^2 elements
    g.set_coefficient(k)
    v = torch.zeros(g.info(2).vec_len, dtype=torch.float64, device="cuda")
    with pytest.raises(hhg.HHGError) as e:
        g.p2_apply(1, v, v)
    assert e.value.status == hhg.ERR_ARG
    g.close()
