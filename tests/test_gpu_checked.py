"""The bounds-checking build libhhg_checked.so (device-side checks of every
table-driven index: ids read from the face, edge, vertex, corner and
vertex-edge records, their rotated face frames, positions along edges, face
tasks) runs the parity suites of the operator, the smoothers, the
transfers, the V-cycle and solves, P2, Stokes and the row kernels with no
failed check and the same results as the normal build.

The suites run in a child pytest with HHG_LIBRARY=checked; a failed check
shows as a wrong result, as HHG_ERR_BOUNDS from hhg_sync / hhg_solve, or as
HHG_ERR_BOUNDS when a mesh is closed (the session then fails)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_p2.py", "tests/test_gpu_face_sweep.py",
          "tests/test_gpu_rows.py", "tests/test_gpu_tail.py", "tests/test_gpu_stokes.py"]


def test_checked_build_runs_parity_suites_clean():
    lib = os.path.join(ROOT, "paper_1805_10167_gb300", "libhhg_checked.so")
    if not os.path.exists(lib):
        from paper_1805_10167_gb300 import build
        build.build(checked=True)
    env = dict(os.environ, HHG_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "index checks failed" not in r.stderr, tail

