"""The one-CTA coarse tail of the V-cycle (levels <= 3 in a single launch,
shared-memory vectors, host-assembled rows) against the level-by-level
kernels and the oracle: FP64 cycles to 1e-12 with the tail on and off
(k = 1 and the random field), FP32 cycles within FP32 rounding of each
other, and the cut-off control."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,L,vark", [("square", 4, False), ("annulus", 5, False), ("annulus", 5, True),
                                         ("random7", 4, False), ("random11", 3, True), ("annulus16", 2, False)])
def test_tail_cycle_matches_oracle_and_kernels(name, L, vark):
    P = Pair(name, L, vark=vark)
    assert P.g.coarse_tail() == min(3, L)
    x0, b = P.random(L), P.random(L)
    want = mg.vcycle(P.H, L, x0.copy(), b, 3, 3)
    xa = P.to_dev(L, x0)
    P.g.vcycle(L, xa, P.to_dev(L, b))
    got_tail = P.from_dev(L, xa)
    assert rel_err(got_tail, want) <= FP64_TOL
    assert P.g.coarse_tail(0) == 0
    xb = P.to_dev(L, x0)
    P.g.vcycle(L, xb, P.to_dev(L, b))
    got_plain = P.from_dev(L, xb)
    assert rel_err(got_plain, want) <= FP64_TOL
    assert rel_err(got_tail, got_plain) <= FP64_TOL
    # FP32 cycles: the two paths within FP32 rounding
    P.g.coarse_tail(3)
    x32 = [P.to_dev(L, x0, prec=1), P.to_dev(L, x0, prec=1)]
    b32 = P.to_dev(L, b, prec=1)
    P.g.vcycle(L, x32[0], b32, prec=1)
    P.g.coarse_tail(0)
    P.g.vcycle(L, x32[1], b32, prec=1)
    assert rel_err(P.from_dev(L, x32[0], prec=1), P.from_dev(L, x32[1], prec=1)) <= 1e-5
    P.close()


def test_tail_solve_cycle_count_and_cutoff_control():
    P = Pair("annulus", 6)
    L = 6
    b = P.random(L, zero_dirichlet=True)
    its = []
    for cut in (3, 1, 0):
        assert P.g.coarse_tail(cut) == cut
        x = P.to_dev(L, np.zeros(P.H.levels[L].n))
        st, rep = P.g.solve(L, x, P.to_dev(L, b))
        its.append(rep["iterations"])
        assert rep["r_final"] <= 1e-10 * rep["r0"]
    assert its[0] == its[1] == its[2]
    with pytest.raises(P.hhg.HHGError) as e:
        P.g.coarse_tail(-1)
    assert e.value.status == P.hhg.ERR_ARG
    P.close()
