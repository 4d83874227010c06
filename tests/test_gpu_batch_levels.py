"""Batched solves at the batch workload's levels (6-9): problems of equal
level merged into one mesh, the register-strip face sweeps with autotuned
splits across problem boundaries, FP32 refinement and batched flexible CG,
each problem's iterate against its own FP64 oracle solve."""
import numpy as np
import pytest

from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs

pytestmark = pytest.mark.gpu

# (seed, macro-faces, level): two problems per level group, the finest
# levels with the fewest faces (as the oracle has to hold each of them)
PROBLEMS = [(1001, 2, 9), (1002, 3, 9), (1003, 4, 8), (1004, 6, 8),
            (1005, 9, 7), (1006, 12, 7), (1007, 17, 6), (1008, 30, 6)]


@pytest.fixture(scope="module")
def oracle_solutions():
    out = []
    for seed, nf, L in PROBLEMS:
        xy, tri = inputs.random_square_mesh(seed, nf)
        H = mg.Hierarchy(om.MacroMesh(xy, tri), L)
        b = inputs.uniform_pm1(H.levels[L].n, seed)
        x, _ = mg.solve(H, np.zeros(H.levels[L].n), b.copy(), 3, 3, tol=1e-12)
        out.append((xy, tri, L, H, b, x))
    return out


@pytest.mark.parametrize("mode", ["ir", "fpcg"])
def test_batch_levels_6_to_9_match_oracle(oracle_solutions, mode):
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    B = hhg.Batch([(xy, tri) for xy, tri, *_ in oracle_solutions], [L for _, _, L, *_ in oracle_solutions])
    B.tune()
    xs, bs = [], []
    for p, (xy, tri, L, H, b, x) in enumerate(oracle_solutions):
        assert B.info(p).n_nodes == H.levels[L].n
        bs.append(torch.tensor(b, dtype=torch.float64, device="cuda"))
        xs.append(torch.zeros_like(bs[-1]))
    st, reps = B.solve(xs, bs, mode={"ir": hhg.SOLVE_IR, "fpcg": hhg.SOLVE_FPCG}[mode])
    assert st == hhg.OK
    for p, (xy, tri, L, H, b, want) in enumerate(oracle_solutions):
        got = xs[p].cpu().numpy()
        lv = H.levels[L]
        r0 = mg.norm_free(H, L, H.residual(L, np.zeros(lv.n), b))
        assert mg.norm_free(H, L, H.residual(L, got, b)) <= 1.01e-10 * r0, p
        assert reps[p]["r_final"] <= 1e-10 * reps[p]["r0"], p
        err = np.abs(got - want).max() / np.abs(want).max()
        print(f"problem {p} (level {L}, {len(tri)} faces): {reps[p]['iterations']} iterations, "
              f"rel. error vs oracle {err:.2e}")
        assert err < 1e-8, p
    B.close()
