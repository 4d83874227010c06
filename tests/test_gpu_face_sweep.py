"""The two face Gauss-Seidel kernels (shared-memory ring of row blocks,
register strips) and their work splits against the FP64 oracle's
colour-ordered sweep.  Levels 7 and 8 (N = 128, 256) give several 90-column
strips per face, so the strip halos are exercised; small row blocks (7 rows,
16 rows) exercise the row-block halos and the alignment of the register ring.
Every split must give the oracle's sweep to 1e-12 in FP64; FP32 sweeps are
held to a bound derived from FP32 rounding."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu

SPLITS = [(0, 1), (0, 3), (1, 7), (1, 16), (1, 64), (1, 128)]
# FP32: inputs rounded to FP32 (2^-24 relative) and two sweeps of 4-term
# updates of O(1) data; 512 unit roundoffs of the max norm bound the result
FP32_TOL = 512 * 2.0 ** -24


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


@pytest.mark.parametrize("name,L", [("square", 8), ("random5", 7)])
@pytest.mark.parametrize("vark", [False, True])
@pytest.mark.parametrize("split", SPLITS)
def test_face_sweep_kernels_match_oracle(pairs, name, L, vark, split):
    P = pairs(name, L, vark)
    hhg = P.hhg
    rng = np.random.default_rng(7)
    for l in (L - 1, L):
        for prec in (hhg.F64, hhg.F32):
            assert P.g.sweep_config(l, prec, *split) == split
            assert P.g.sweep_config(l, prec) == split
        x0 = rng.standard_normal(P.H.levels[l].n)
        b = rng.standard_normal(P.H.levels[l].n)
        for fwd in (True, False):
            # one FP64 sweep reads b, two or more read b / A_pp (one scaling pass)
            want1 = mg.gs_sweep(P.H, l, x0.copy(), b, forward=fwd)
            want = mg.gs_sweep(P.H, l, want1.copy(), b, forward=fwd)
            mode = hhg.GS_FWD if fwd else hhg.GS_BWD
            x = P.to_dev(l, x0)
            P.g.smooth(l, x, P.to_dev(l, b), mode, sweeps=1)
            assert rel_err(P.from_dev(l, x), want1) <= FP64_TOL, (l, fwd, "f64, 1 sweep")
            x = P.to_dev(l, x0)
            P.g.smooth(l, x, P.to_dev(l, b), mode, sweeps=2)
            assert rel_err(P.from_dev(l, x), want) <= FP64_TOL, (l, fwd, "f64")
            x32 = P.to_dev(l, x0, prec=hhg.F32)
            P.g.smooth(l, x32, P.to_dev(l, b, prec=hhg.F32), mode, sweeps=2, prec=hhg.F32)
            assert rel_err(P.from_dev(l, x32, prec=hhg.F32), want) <= FP32_TOL, (l, fwd, "f32")


def test_sweep_config_rejects_bad_arguments(pairs):
    P = pairs("square", 4, False)
    hhg = P.hhg
    for variant, param in [(2, 4), (-1, 4), (1, 0), (0, -3)]:
        with pytest.raises(hhg.HHGError) as e:
            P.g.sweep_config(4, hhg.F64, variant, param)
        assert e.value.status == hhg.ERR_ARG
    with pytest.raises(hhg.HHGError):
        P.g.sweep_config(9, hhg.F64)   # level above max_level


def test_tuner_choice_is_a_valid_config(pairs):
    P = pairs("square", 8, False)
    hhg = P.hhg
    P.g.tune(prec=hhg.F32)
    for l in range(4, 9):
        v, p = P.g.sweep_config(l, hhg.F32)
        assert v in (hhg.SWEEP_RING, hhg.SWEEP_STRIP) and p >= 1


@pytest.mark.parametrize("name,L", [("square", 8), ("random5", 7)])
@pytest.mark.parametrize("vark", [False, True])
@pytest.mark.parametrize("split", [(1, 16), (1, 64), (0, 3)])
def test_vcycle_with_scaled_right_hand_sides_matches_oracle(pairs, name, L, vark, split):
    """Inside a V-cycle the FP64 strip sweeps of levels with N > 64 and k = 1
    read b / A_pp computed once per right-hand side (from the caller's b on
    the top level, by the restriction below it); the cycle must still give
    the oracle's to 1e-12, with every split on levels L - 1 and L."""
    P = pairs(name, L, vark)
    hhg = P.hhg
    old = [P.g.sweep_config(l) for l in (L - 1, L)]
    try:
        for l in (L - 1, L):
            P.g.sweep_config(l, hhg.F64, *split)
        rng = np.random.default_rng(11)
        x0, b = rng.standard_normal(P.H.levels[L].n), rng.standard_normal(P.H.levels[L].n)
        x = P.to_dev(L, x0)
        bd = P.to_dev(L, b)
        want = x0.copy()
        for call in range(3):   # the third call replays a captured graph
            P.g.vcycle(L, x, bd, nu1=2, nu2=1)
            want = mg.vcycle(P.H, L, want, b, 2, 1)
            assert rel_err(P.from_dev(L, x), want) <= FP64_TOL, call
    finally:
        for l, c in zip((L - 1, L), old):
            P.g.sweep_config(l, hhg.F64, *c)
