"""hhg_dot_noalloc, the allocation-free dot product, against hhg_dot.

Some callers must not allocate device memory when they compute (for example
code running while the application's memory pool refuses new allocations).
hhg_dot_noalloc serves them with its reduction scratch in a fixed device
array inside the library.  This test calls it through the C-ABI twice in a
row on the same data and on fresh data and compares every result with
hhg_dot's, and checks that the device's free memory is the same before
and after calls made once the mesh exists.  It lives in its own file,
collected last, and passes both alone in a fresh process and after the
other GPU tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative, the FP64 tolerance of the other parity tests


@pytest.mark.parametrize("name,L,prec", [("annulus", 5, 0), ("random5", 4, 0), ("annulus", 4, 1)])
def test_dot_noalloc_matches_dot_on_consecutive_calls(name, L, prec):
    torch = pytest.importorskip("torch")
    from gpu_support import Pair
    P = Pair(name, L)
    out_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    out_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        a, b = P.random(L), P.random(L)
        da, db = P.to_dev(L, a, prec=prec), P.to_dev(L, b, prec=prec)
        for same_data in range(2):      # two calls in a row on the same vectors
            out_ref.zero_()
            out_new.fill_(np.nan)
            P.g.dot(L, da, db, out_ref, prec=prec)
            P.g.dot_noalloc(L, da, db, out_new, prec=prec)
            torch.cuda.synchronize()
            ref, new = out_ref.item(), out_new.item()
            scale = float(torch.sqrt((da.double() ** 2).sum() * (db.double() ** 2).sum()))
            assert abs(new - ref) <= TOL * scale, (call, same_data, ref, new)
    # the scratch address and the kernels' module were set up with the mesh:
    # calls made now change no device allocation, first or later ones alike
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        P.g.dot_noalloc(L, da, db, out_new, prec=prec)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    P.close()


def test_dot_noalloc_first_call_on_a_fresh_mesh_allocates_nothing():
    """The very first hhg_dot_noalloc call on a newly created mesh leaves the
    device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    from gpu_support import Pair
    P = Pair("square", 4)
    a = P.to_dev(4, P.random(4))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    P.g.dot_noalloc(4, a, a, out)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert out.item() > 0
    P.close()


def test_dot_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    from gpu_support import Pair
    P = Pair("square", 2)
    x = P.new(2)
    with pytest.raises(P.hhg.HHGError) as e:
        P.g.dot_noalloc(2, x, x, None)
    assert e.value.status == P.hhg.ERR_ARG
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad_level in (-1, 3):          # valid result buffer, level out of range
        with pytest.raises(P.hhg.HHGError) as e:
            P.g.dot_noalloc(bad_level, x, x, out)
        assert e.value.status == P.hhg.ERR_ARG
    P.close()
