"""Repeated calls replay captured CUDA graphs (the first call with a given
level, cycle shape and vector pair runs directly, the second is captured,
later ones replay): the results must equal the oracle's after every call, on
the caller's default stream and on a side stream, and a change of the sweep
split, the FP64 arithmetic mode or the coefficient between calls must be
picked up (the captured sequences are dropped)."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    P = Pair("annulus", 6)
    yield P
    P.close()


@pytest.mark.parametrize("side_stream", [False, True])
def test_repeated_vcycles_match_oracle_after_every_call(pair, side_stream):
    P = pair
    torch, hhg = P.torch, P.hhg
    L = 6
    x0, b = P.random(L), P.random(L)
    x = P.to_dev(L, x0)
    bd = P.to_dev(L, b)
    want = x0.copy()
    st = torch.cuda.Stream() if side_stream else None
    for call in range(5):
        if st is not None:
            st.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(st):
                P.g.vcycle(L, x, bd, nu1=2, nu2=1, stream=st)
            torch.cuda.current_stream().wait_stream(st)
        else:
            P.g.vcycle(L, x, bd, nu1=2, nu2=1)
        want = mg.vcycle(P.H, L, want, b, 2, 1)
        assert rel_err(P.from_dev(L, x), want) <= FP64_TOL, call


def test_configuration_changes_between_replays_are_seen(pair):
    P = pair
    hhg = P.hhg
    L = 6
    x0, b = P.random(L), P.random(L)
    x = P.to_dev(L, x0)
    bd = P.to_dev(L, b)
    want = x0.copy()
    old = P.g.sweep_config(L)
    try:
        for call in range(7):
            if call == 3:   # a different split of the face sweep
                P.g.sweep_config(L, variant=hhg.SWEEP_STRIP, param=8)
            if call == 5:
                P.g.fp64_arith(hhg.ARITH_DFLOAT)
            P.g.vcycle(L, x, bd, nu1=1, nu2=1)
            want = mg.vcycle(P.H, L, want, b, 1, 1)
            assert rel_err(P.from_dev(L, x), want) <= FP64_TOL, call
    finally:
        P.g.sweep_config(L, variant=old[0], param=old[1])
        P.g.fp64_arith(hhg.ARITH_IEEE)


def test_coefficient_change_between_replays_is_seen():
    torch = pytest.importorskip("torch")
    P = Pair("square", 5)
    V = Pair("square", 5, vark=True)
    try:
        L = 5
        x0, b = P.random(L), P.random(L)
        x = P.to_dev(L, x0)
        bd = P.to_dev(L, b)
        for _ in range(3):   # captured with k = 1
            P.g.vcycle(L, x, bd, nu1=1, nu2=1)
        P.g.set_coefficient(V.k_dev)
        x2 = P.to_dev(L, x0)
        for _ in range(3):
            P.g.vcycle(L, x2, bd, nu1=1, nu2=1)
        want = x0.copy()
        for _ in range(3):
            want = mg.vcycle(V.H, L, want, b, 1, 1)
        assert rel_err(P.from_dev(L, x2), want) <= FP64_TOL
        P.g.set_coefficient(None)
        x3 = P.to_dev(L, x0)
        for _ in range(3):
            P.g.vcycle(L, x3, bd, nu1=1, nu2=1)
        want = x0.copy()
        for _ in range(3):
            want = mg.vcycle(P.H, L, want, b, 1, 1)
        assert rel_err(P.from_dev(L, x3), want) <= FP64_TOL
    finally:
        P.close()
        V.close()
