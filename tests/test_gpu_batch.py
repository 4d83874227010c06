"""Batched solves of independent problems (one launch per phase across all
problems of a level group, CUDA-graph replayed iterations, autotuned face
sweeps) against per-problem FP64 oracle solves."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs

pytestmark = pytest.mark.gpu


def problems(n=6, seed0=1000):
    out = []
    for k in range(n):
        seed = seed0 + k
        nf = 2 + (seed * 7919) % 15
        xy, tri = inputs.random_square_mesh(seed, nf)
        L = 2 + (seed % 3)
        out.append((xy, tri, L))
    return out


def oracle_solution(xy, tri, L, b, tol=1e-12):
    H = mg.Hierarchy(om.MacroMesh(xy, tri), L)
    x, hist = mg.solve(H, np.zeros(H.levels[L].n), b.copy(), 3, 3, tol=tol)
    return H, x


@pytest.mark.parametrize("mode", ["ir", "mg", "fpcg"])
def test_batch_solve_matches_oracle(mode):
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    probs = problems()
    B = hhg.Batch([(xy, tri) for xy, tri, L in probs], [L for xy, tri, L in probs])
    xs, bs, bh = [], [], []
    for p, (xy, tri, L) in enumerate(probs):
        n = B.info(p).n_nodes
        b = inputs.uniform_pm1(n, 1000 + p)
        bh.append(b)
        bs.append(torch.tensor(b, dtype=torch.float64, device="cuda"))
        xs.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
    st, reps = B.solve(xs, bs, mode={"ir": hhg.SOLVE_IR, "mg": hhg.SOLVE_MG, "fpcg": hhg.SOLVE_FPCG}[mode])
    for p, (xy, tri, L) in enumerate(probs):
        H, want = oracle_solution(xy, tri, L, bh[p])
        got = xs[p].cpu().numpy()
        lv = H.levels[L]
        r = H.residual(L, got, bh[p])
        r0 = mg.norm_free(H, L, H.residual(L, np.zeros(lv.n), bh[p]))
        assert mg.norm_free(H, L, r) <= 1.01e-10 * r0, p
        assert reps[p]["r_final"] <= 1e-10 * reps[p]["r0"]
        assert rel_err(got, want) < 1e-8, p
    B.close()


def test_batch_mg_cycle_count_matches_single_problem_solves():
    """FP64 batch iterations: each problem's recorded cycle count equals the
    count of the single-mesh solver on the same problem."""
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    probs = problems(4, 2000)
    B = hhg.Batch([(xy, tri) for xy, tri, L in probs], [L for xy, tri, L in probs])
    xs, bs = [], []
    for p, (xy, tri, L) in enumerate(probs):
        n = B.info(p).n_nodes
        bs.append(torch.tensor(inputs.uniform_pm1(n, 7 + p), dtype=torch.float64, device="cuda"))
        xs.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
    st, reps = B.solve(xs, bs, mode=hhg.SOLVE_MG)
    for p, (xy, tri, L) in enumerate(probs):
        g = hhg.Mesh(xy, tri, L)
        I = g.info(L)
        bi = torch.zeros(I.vec_len, dtype=torch.float64, device="cuda")
        xi = torch.zeros_like(bi)
        g.from_canonical(L, bs[p], bi)
        _, rep = g.solve(L, xi, bi, mode=hhg.SOLVE_MG)
        assert rep["iterations"] == reps[p]["iterations"], p
        g.close()
    B.close()


def test_autotuned_split_gives_identical_results():
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    probs = problems(3, 3000)
    probs = [(xy, tri, 5) for xy, tri, _ in probs]
    B = hhg.Batch([(xy, tri) for xy, tri, L in probs], [L for xy, tri, L in probs])
    bs = [torch.tensor(inputs.uniform_pm1(B.info(p).n_nodes, p), dtype=torch.float64, device="cuda")
          for p in range(3)]
    x1 = [torch.zeros_like(b) for b in bs]
    B.solve(x1, bs)
    B.tune()
    x2 = [torch.zeros_like(b) for b in bs]
    B.solve(x2, bs)
    for a, b in zip(x1, x2):
        assert torch.equal(a, b)
    B.close()
    # plain mesh: tuning keeps the V-cycle bitwise unchanged
    P = Pair("annulus", 5)
    x0, b = P.random(5), P.random(5)
    xa = P.to_dev(5, x0)
    P.g.vcycle(5, xa, P.to_dev(5, b))
    P.g.tune(prec=0)
    xb = P.to_dev(5, x0)
    P.g.vcycle(5, xb, P.to_dev(5, b))
    assert torch.equal(xa, xb)
    want = mg.vcycle(P.H, 5, x0.copy(), b, 3, 3)
    assert rel_err(P.from_dev(5, xb), want) <= FP64_TOL
    P.close()


def test_batch_flexible_cg_matches_single_problem_solves_and_needs_fewer_steps():
    """Batched flexible CG: every problem reaches the FP64 tolerance in the
    step count of the single-mesh flexible CG (within one step: FP32 rounding
    differs between the merged and the single mesh), and never more steps
    than FP32-in-FP64 refinement needs on the same problem."""
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    probs = problems(5, 2000)
    B = hhg.Batch([(xy, tri) for xy, tri, L in probs], [L for xy, tri, L in probs])
    bs, xs = [], []
    for p in range(len(probs)):
        n = B.info(p).n_nodes
        bs.append(torch.tensor(inputs.uniform_pm1(n, 2000 + p), dtype=torch.float64, device="cuda"))
        xs.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
    st, reps = B.solve(xs, bs, mode=hhg.SOLVE_FPCG)
    for _ in range(2):   # replays of the captured iteration give the same answer
        xs2 = [torch.zeros_like(x) for x in xs]
        st, reps2 = B.solve(xs2, bs, mode=hhg.SOLVE_FPCG)
        for a, c in zip(xs, xs2):
            assert torch.equal(a, c)
    for p, (xy, tri, L) in enumerate(probs):
        g = hhg.Mesh(xy, tri, L)
        I = g.info(L)
        bi = torch.zeros(I.vec_len, dtype=torch.float64, device="cuda")
        g.from_canonical(L, bs[p], bi)
        its = {}
        for mode in (hhg.SOLVE_FPCG, hhg.SOLVE_IR):
            xi = torch.zeros_like(bi)
            _, rep = g.solve(L, xi, bi, mode=mode)
            its[mode] = rep["iterations"]
        assert abs(reps[p]["iterations"] - its[hhg.SOLVE_FPCG]) <= 1, (p, reps[p]["iterations"], its)
        assert reps[p]["iterations"] <= its[hhg.SOLVE_IR], (p, reps[p]["iterations"], its)
        assert reps[p]["r_final"] <= 1e-10 * reps[p]["r0"]
        g.close()
    B.close()
