"""The bounded device-side waits report a timeout and leave the context usable.

A host-side test hook (hhg_debug_wait_limit) makes every grid barrier of the
whole-sweep Gauss-Seidel kernel await one arrival more than its launch has
-- an arrival that never comes -- with a short poll limit.  Nothing faults,
traps or hangs: each wait gives up, sets the mesh's device error word, and
the launch runs to its end with every access in bounds.  The test checks
that hhg_sync and hhg_solve report HHG_ERR_TIMEOUT, that the report clears
the error word, and that calls made after the hook is lifted succeed and
match the oracle."""
import numpy as np
import pytest

from gpu_support import FP64_TOL, Pair, rel_err
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [3, 7])      # small-face (shared memory) and strip face phases
def test_grid_barrier_timeout_is_reported_and_recovered(L):
    P = Pair("annulus", L)
    hhg = P.hhg
    x0, b = P.random(L), P.random(L)
    xd, bd = P.to_dev(L, x0), P.to_dev(L, b)
    P.g.coarse_tail(0)                           # every level through the whole-sweep kernel
    P.g.sync()                                   # nothing pending

    P.g.debug_wait_limit(1, 2000)
    P.g.smooth(L, xd, bd, smoother=hhg.GS_FWD, sweeps=2)   # asynchronous: returns OK
    with pytest.raises(hhg.HHGError) as e:
        P.g.sync()
    assert e.value.status == hhg.ERR_TIMEOUT
    P.g.sync()                                   # the report cleared the error word
    st, rep = P.g.solve(L, P.to_dev(L, np.zeros(P.H.levels[L].n)), bd, max_iter=2,
                        raise_on_error=False)
    assert st == hhg.ERR_TIMEOUT and rep["status"] == hhg.ERR_TIMEOUT

    P.g.debug_wait_limit(0)                      # normal operation again
    P.g.sync()
    xd = P.to_dev(L, x0)
    P.g.smooth(L, xd, bd, smoother=hhg.GS_FWD, sweeps=1)
    P.g.sync()
    want = mg.gs_sweep(P.H, L, x0.copy(), b, forward=True)
    assert rel_err(P.from_dev(L, xd), want) <= FP64_TOL
    x = P.to_dev(L, np.zeros(P.H.levels[L].n))
    st, rep = P.g.solve(L, x, bd)
    assert st == hhg.OK and rep["r_final"] <= 1e-10 * rep["r0"]
    P.close()


def test_debug_wait_limit_rejects_negative_count():
    P = Pair("square", 2)
    with pytest.raises(P.hhg.HHGError) as e:
        P.g.debug_wait_limit(-1)
    assert e.value.status == P.hhg.ERR_ARG
    P.close()
