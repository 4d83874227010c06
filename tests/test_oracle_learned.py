"""Pins of the learned-smoother network and of FGMRES (CPU, FP64)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import krylov, learned
from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs


def small_case(seed=0, N=8, H=None, W=None):
    rng = np.random.default_rng(seed)
    M, Mi = learned.masks(N, H=H, W=W)
    X = rng.standard_normal((3,) + M.shape) * M
    e = rng.standard_normal(M.shape) * Mi
    return X, M, Mi, e


def test_parameter_count():
    assert learned.n_params() == 16 * (27 + 1) + 16 * (144 + 1) + (144 + 1)


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 5, 6))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    out = learned.conv(x, W, b)
    for o in range(2):
        for j in range(5):
            for i in range(6):
                s = b[o]
                for c in range(3):
                    for dj in (-1, 0, 1):
                        for di in (-1, 0, 1):
                            if 0 <= j + dj < 5 and 0 <= i + di < 6:
                                s += W[o, c, dj + 1, di + 1] * x[c, j + dj, i + di]
                assert out[o, j, i] == pytest.approx(s, abs=1e-12)


def test_backward_equals_central_differences():
    X, M, Mi, e = small_case(2, N=7)
    p = learned.init_params(3)
    for k in learned.ORDER:
        p[k] = p[k] + 0.05 * np.random.default_rng(4).standard_normal(p[k].shape)
    L, g = learned.loss_and_grad(p, X, M, Mi, e, Mi)
    v0 = learned.flatten(p)
    gv = learned.flatten(g)
    rng = np.random.default_rng(5)
    idx = rng.choice(v0.size, 40, replace=False)
    h = 1e-6
    for t in idx:
        vp, vm = v0.copy(), v0.copy()
        vp[t] += h
        vm[t] -= h
        Lp = learned.loss_and_grad(learned.unflatten(vp), X, M, Mi, e, Mi)[0]
        Lm = learned.loss_and_grad(learned.unflatten(vm), X, M, Mi, e, Mi)[0]
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(gv[t], rel=1e-5, abs=1e-8), (t, fd, gv[t])


def test_output_vanishes_off_the_interior_and_is_local():
    X, M, Mi, e = small_case(6, N=12)
    p = learned.init_params(7)
    d, _ = learned.forward(p, X, M, Mi)
    assert np.all(d[Mi == 0] == 0)
    # receptive field 7 x 7: a change at (6, 6) leaves points 4 away untouched
    X2 = X.copy()
    X2[:, 6, 3] += 1.0
    d2, _ = learned.forward(p, X2, M, Mi)
    changed = np.argwhere(np.abs(d2 - d) > 0)
    assert np.all(np.abs(changed - np.array([6, 3])).max(axis=1) <= 3)


def test_adam_matches_its_definition_on_a_quadratic():
    v = np.array([1.0, -2.0])
    m = s = np.zeros(2)
    for t in range(1, 4):
        g = 2 * v
        v_new, m, s = learned.adam_step(v, g, m, s, t, lr=0.1)
        # first step of Adam moves every coordinate by lr (bias-corrected)
        if t == 1:
            np.testing.assert_allclose(np.abs(v_new - v), 0.1, rtol=1e-6)
        v = v_new


# ------------------------------------------------------------------ FGMRES
def _problem(L=2):
    xy, tri = inputs.annulus_mesh(32, 2)
    H = mg.Hierarchy(om.MacroMesh(xy, tri), L)
    lv = H.levels[L]
    b = inputs.uniform_pm1(lv.n, 3)
    b[~lv.free] = 0
    return H, lv, b


def test_fgmres_identity_preconditioner_is_minimal_residual():
    """With M = I, after k steps the iterate minimises ||b - A x|| over
    x0 + K_k(A, r0) (least squares over an explicit Krylov basis)."""
    H, lv, b = _problem(1)
    fr = lv.free
    A = lambda v: H.apply(1, v)
    for k in (1, 3, 6):
        x, hist, steps = krylov.fgmres(A, lambda v, j: v.copy(), b, np.zeros(lv.n), fr, m=20, tol=0.0, max_iter=k)
        Af = H.A[1][fr][:, fr].toarray()
        r0 = b[fr]
        K = [r0]
        for _ in range(k - 1):
            K.append(Af @ K[-1])
        K = np.array(K).T
        y = np.linalg.lstsq(Af @ K, r0, rcond=None)[0]
        np.testing.assert_allclose(x[fr], K @ y, rtol=1e-8, atol=1e-10)


def test_fgmres_exact_preconditioner_one_step():
    H, lv, b = _problem(2)
    fr = lv.free
    Af = H.A[2][fr][:, fr].toarray()
    exact = lambda v, j: np.where(fr, 0.0, 0.0) + _embed(np.linalg.solve(Af, v[fr]), fr)
    x, hist, steps = krylov.fgmres(lambda v: H.apply(2, v), exact, b, np.zeros(lv.n), fr, tol=1e-10)
    assert steps == 1
    assert hist[-1] <= 1e-10 * hist[0]


def _embed(v, fr):
    out = np.zeros(fr.size)
    out[fr] = v
    return out


def test_fgmres_with_vcycle_preconditioner_converges_monotonically():
    H, lv, b = _problem(4)
    fr = lv.free

    def pre(v, j):
        z = np.zeros(lv.n)
        return mg.vcycle(H, 4, z, v, 1, 1)
    x, hist, steps = krylov.fgmres(lambda v: H.apply(4, v), pre, b, np.zeros(lv.n), fr, tol=1e-10)
    assert hist[-1] <= 1e-10 * hist[0]
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    assert steps < 20


def test_residual_loss_gradient_equals_central_differences():
    X, M, Mi, e = small_case(8, N=9)
    rng = np.random.default_rng(9)
    ku = rng.uniform(0.5, 2.0, M.shape) * M
    kd = rng.uniform(0.5, 2.0, M.shape) * M
    wts = learned.edge_weights((0.4, 0.9, 0.6), ku, kd)
    shat = rng.standard_normal(M.shape) * Mi
    p = learned.init_params(11)
    p["W3"] = p["W3"] * 10
    L, g = learned.residual_loss_and_grad(p, X, M, Mi, shat, Mi, wts)
    v0, gv = learned.flatten(p), learned.flatten(g)
    for t in np.random.default_rng(12).choice(v0.size, 40, replace=False):
        vp, vm = v0.copy(), v0.copy()
        vp[t] += 1e-6
        vm[t] -= 1e-6
        fd = (learned.residual_loss_and_grad(learned.unflatten(vp), X, M, Mi, shat, Mi, wts)[0]
              - learned.residual_loss_and_grad(learned.unflatten(vm), X, M, Mi, shat, Mi, wts)[0]) / 2e-6
        assert fd == pytest.approx(gv[t], rel=1e-5, abs=1e-8)


def test_scaled_operator_matches_assembled_rows():
    """D^-1 A on a face lattice built from the cotangent weights equals the
    brute-force assembled matrix rows (divided by the diagonal) at interior
    points, for a random coefficient."""
    xy, tri = inputs.annulus_mesh(32, 2)
    M_ = om.MacroMesh(xy, tri)
    L = 3
    lv = om.Level(M_, L)
    N = lv.N
    rng = np.random.default_rng(13)
    k = rng.uniform(0.5, 2.0, M_.nf * N * N)
    from oracle import fem
    A = fem.assemble(lv, k).tocsr()
    dvec = rng.standard_normal(lv.n)
    import math
    f = 5
    v0, v1, v2 = xy[M_.tri[f]]

    def cot(a, b, c):
        u, w = b - a, c - a
        return (u @ w) / abs(u[0] * w[1] - u[1] * w[0])
    cots = (cot(v0, v1, v2), cot(v1, v2, v0), cot(v2, v0, v1))
    Mc, Mi = learned.masks(N)
    ku = np.zeros((N + 1, N + 1))
    kd = np.zeros((N + 1, N + 1))
    kf = k[f * N * N:(f + 1) * N * N]
    r = 0
    for j in range(N):
        for i in range(N - j):
            ku[j, i] = kf[r]
            r += 1
    for j in range(N - 1):
        for i in range(N - 1 - j):
            kd[j, i] = kf[r]
            r += 1
    G = lv.face_ids[f]
    img = np.zeros((N + 1, N + 1))
    img[G >= 0] = dvec[G[G >= 0]]
    out = learned.scaled_operator(img, learned.edge_weights(cots, ku, kd))
    want = (A @ dvec) / A.diagonal()
    for j in range(1, N - 1):
        for i in range(1, N - j):
            assert out[j, i] == pytest.approx(want[G[j, i]], rel=1e-12, abs=1e-12)


def test_bf16_rounding_matches_torch_bfloat16():
    """The oracle's BF16 rounding (round to nearest, ties to even, at bit 16 of
    the binary32 pattern) against torch's own float32 -> bfloat16 conversion,
    element by element over about 10^6 values: random finite bit patterns
    (normal and subnormal), exact ties with even and odd kept parts, the
    neighbours of each tie, +-0, the largest finite values (which round to
    infinity) and plain normal samples."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2024)
    bits = rng.integers(0, 2 ** 32, 600_000, dtype=np.uint64).astype(np.uint32)
    bits = bits[(bits & 0x7F800000) != 0x7F800000]          # finite patterns only
    hi = rng.integers(0, 2 ** 16, 100_000, dtype=np.uint64).astype(np.uint32) << 16
    hi = hi[(hi & 0x7F800000) != 0x7F800000]
    ties = hi | 0x8000                                         # exactly half-way
    below, above = hi | 0x7FFF, hi | 0x8001
    special = np.array([0x00000000, 0x80000000, 0x7F7FFFFF, 0xFF7FFFFF, 0x7F7F8000,
                        0x00000001, 0x00008000, 0x00018000, 0x3F808000, 0x3F818000],
                       dtype=np.uint32)
    x = np.concatenate([bits, ties, below, above, special]).view(np.float32)
    x = np.concatenate([x, rng.standard_normal(200_000).astype(np.float32)])
    assert x.size > 900_000
    got = learned.bf16(x)
    want = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, want)
    # +-0 keep their sign
    z = learned.bf16(np.array([0.0, -0.0], dtype=np.float32))
    assert np.signbit(z).tolist() == [False, True]
