"""P2 at the benchmark's full size: P2 on level 9 of the 128-face annulus
(its unknowns are the level-10 lattice, 67 M free), the configuration the
benchmark times.  The oracle cannot hold it, so the operator is checked on
sampled face-interior rows of all four point types built one by one from
the oracle's P2 element matrices (tests/fullsize_rows.py, pinned on the CPU),
and the p-multigrid solve by the property the oracle pins at small levels:
a level-independent factor per cycle (about 0.336 for V(2,2) with a P1
V(3,3) coarse correction), here below 0.36, reaching 1e-10."""
import numpy as np
import pytest

import fullsize_rows as fr
from paper_1805_10167_gb300 import inputs

pytestmark = pytest.mark.gpu

LP = 9              # P2 level
L1 = LP + 1         # its lattice
N1 = 1 << L1


@pytest.fixture(scope="module")
def big():
    torch = pytest.importorskip("torch")
    from paper_1805_10167_gb300 import hhg
    xy, tri = inputs.annulus_mesh(32, 2)
    g = hhg.Mesh(xy, tri, L1)
    ns = {"torch": torch, "hhg": hhg, "xy": xy, "tri": inputs._ccw(xy, tri), "g": g, "info": g.info(L1)}
    yield ns
    g.close()


def _samples(nf, n, seed):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        f = int(rng.integers(nf))
        J = int(rng.integers(1, N1 - 1))
        I = int(rng.integers(1, N1 - J))
        pts.append((f, I, J))
    for f in (0, nf - 1):       # every point type next to each side of the face
        for J in (1, 2, 3, 4, N1 // 2, N1 // 2 + 1, N1 - 3, N1 - 2):
            for I in (1, 2, 3, 4, N1 - 2 - J, N1 - 1 - J):
                if I >= 1 and I + J <= N1 - 1:
                    pts.append((f, I, J))
    return pts


def test_p2_apply_rows_full_size(big):
    B = big
    t, g, info = B["torch"], B["g"], B["info"]
    gen = t.Generator(device="cuda").manual_seed(21)
    c = t.rand(info.n_nodes, dtype=t.float64, device="cuda", generator=gen) * 2 - 1
    x = t.zeros(info.vec_len, dtype=t.float64, device="cuda")
    g.from_canonical(L1, c, x)
    y = t.zeros_like(x)
    g.p2_apply(LP, x, y)
    h_x, h_y = x.cpu().numpy(), y.cpu().numpy()
    S, FS, off = info.row_stride, info.face_stride, info.f_off
    pts = _samples(info.n_faces, 2000, 7)
    got, want = [], []
    for f, I, J in pts:
        base = off + f * FS
        w = fr.p2_row(B["xy"], B["tri"], N1, f, I, J)
        want.append(sum(v * h_x[base + (J + dJ) * S + I + dI] for (dI, dJ), v in w.items()))
        got.append(h_y[base + J * S + I])
    got, want = np.array(got), np.array(want)
    err = np.abs(got - want).max() / np.abs(want).max()
    print(f"P2 level {LP} apply: {len(pts)} sampled rows, max-norm relative error {err:.2e}")
    assert err <= 1e-12


def test_p2_pmg_solve_full_size(big):
    B = big
    t, g, info = B["torch"], B["g"], B["info"]
    bc = t.tensor(inputs.uniform_pm1(info.n_nodes, 1234), dtype=t.float64, device="cuda")
    b = t.zeros(info.vec_len, dtype=t.float64, device="cuda")
    g.from_canonical(L1, bc, b)
    x = t.zeros_like(b)
    st, rep = g.p2_solve(LP, x, b)
    h = np.array(rep["history"])
    rho = h[-1] / h[-2]
    print(f"P2 level {LP} p-multigrid: {rep['iterations']} cycles, last factor {rho:.3f}")
    assert st == B["hhg"].OK
    assert rep["r_final"] <= 1e-10 * rep["r0"]
    assert rho < 0.36 and rep["iterations"] <= 25
