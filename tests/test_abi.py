"""The C-ABI library loads and exports every entry point declared in
include/hhg.h; host-side validation rejects invalid meshes before touching
the GPU (CPU only: no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_path():
    p = os.path.join(ROOT, "paper_1805_10167_gb300", "libhhg.so")
    if not os.path.exists(p):
        from paper_1805_10167_gb300 import build
        build.build()
    return p


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hhg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hhg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(_lib_path())
    names = declared_symbols()
    assert "hhg_vcycle" in names and "hhg_solve" in names and "hhg_mesh_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_checked_build_exports_the_same_and_is_selected():
    """libhhg_checked.so (device-side index checks) exports every declared
    entry point, recompiles the kernels with table-driven indexing, and is
    the library the binding loads under HHG_LIBRARY=checked."""
    import subprocess
    import sys
    from paper_1805_10167_gb300 import build
    p = os.path.join(ROOT, "paper_1805_10167_gb300", "libhhg_checked.so")
    normal = _lib_path()
    if not os.path.exists(p) or os.path.getmtime(p) < os.path.getmtime(normal):
        build.build(checked=True)
    lib = ctypes.CDLL(p)
    for n in declared_symbols():
        assert hasattr(lib, n), n
    redo = {os.path.basename(s) for s in build.sources() if build.uses_checks(s)}
    assert {"kernels.cu", "face_gs_strip.cu", "face_rows.cu", "face_gs.cu", "p2.cu"} <= redo
    code = "from paper_1805_10167_gb300 import hhg; import os; print(os.path.basename(hhg.LIB_PATH), hhg.ERR_BOUNDS)"
    for var, want in (("checked", "libhhg_checked.so"), ("", "libhhg.so")):
        env = dict(os.environ, HHG_LIBRARY=var)
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr
        assert r.stdout.split() == [want, "9"]


def test_status_codes_match_header():
    src = open(os.path.join(ROOT, "include", "hhg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(HHG_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", src))
    _lib_path()
    from paper_1805_10167_gb300 import hhg
    for k, v in codes.items():
        assert getattr(hhg, k[4:]) == v, k
    assert codes["HHG_ERR_BOUNDS"] == 9


def test_binding_covers_header():
    _lib_path()
    from paper_1805_10167_gb300 import hhg
    assert sorted(hhg.EXPORTED) == declared_symbols()


def test_invalid_meshes_rejected_on_host():
    _lib_path()
    from paper_1805_10167_gb300 import hhg
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    with pytest.raises(hhg.HHGError) as e:
        hhg.Mesh(xy, np.array([[0, 1, 7]]), 2)
    assert e.value.status == hhg.ERR_MESH
    with pytest.raises(hhg.HHGError) as e:
        hhg.Mesh(xy, np.array([[0, 1, 1]]), 2)
    assert e.value.status == hhg.ERR_MESH
    with pytest.raises(hhg.HHGError) as e:          # collinear
        hhg.Mesh(np.array([[0, 0], [1, 0], [2, 0]], dtype=np.float64), np.array([[0, 1, 2]]), 2)
    assert e.value.status == hhg.ERR_MESH
    with pytest.raises(hhg.HHGError) as e:          # an edge in three faces
        hhg.Mesh(np.array([[0, 0], [1, 0], [0, 1], [0, -1], [1, 1]], dtype=np.float64),
                 np.array([[0, 1, 2], [0, 3, 1], [0, 1, 4]]), 2)
    assert e.value.status == hhg.ERR_MESH
    with pytest.raises(hhg.HHGError) as e:
        hhg.Mesh(xy, np.array([[0, 1, 2]]), 0)
    assert e.value.status == hhg.ERR_ARG
    assert "max_level" in hhg.last_error()


def test_invalid_batch_rejected_on_host():
    _lib_path()
    from paper_1805_10167_gb300 import hhg, inputs
    good = inputs.unit_square_mesh()
    bad = (good[0], np.array([[0, 1, 42]]))
    with pytest.raises(hhg.HHGError) as e:
        hhg.Batch([good, bad], [2, 3])
    assert e.value.status == hhg.ERR_MESH
    assert "problem 1" in hhg.last_error()
    with pytest.raises(hhg.HHGError) as e:
        hhg.Batch([good], [11])
    assert e.value.status == hhg.ERR_ARG


NOALLOC_PROG = r"""
#include <cstdio>
#include "noalloc.h"
using namespace hhg;
static int rejects(int64_t len) {
  try { noalloc_ctas(len); } catch (const std::invalid_argument&) { return 1; }
  return 0;
}
int main() {
  const int64_t lim = kNoallocMaxSlots;
  std::printf("%lld %d %d %d %d %d %d %d\n", (long long)lim, noalloc_ctas(0), noalloc_ctas(1),
              noalloc_ctas(kNoallocSlotsPerCta), noalloc_ctas(kNoallocSlotsPerCta + 1),
              noalloc_ctas(lim), rejects(lim), rejects(lim + 1));
  return 0;
}
"""


def test_noalloc_scratch_limit_boundary(tmp_path):
    """hhg_dot_noalloc's static array holds 2^14 partial sums of 2^14 slots
    each: a level vector of exactly 2^28 slots fits (2^14 CTAs), one slot
    more is rejected (host logic of csrc/noalloc.h, compiled with g++)."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "noalloc_limit.cpp"
    src.write_text(NOALLOC_PROG)
    exe = tmp_path / "noalloc_limit"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1805_10167_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [2 ** 28, 0, 1, 1, 2, 2 ** 14, 0, 1]
