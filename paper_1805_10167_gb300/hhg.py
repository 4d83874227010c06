"""Thin ctypes binding of libhhg (include/hhg.h).

Argument marshalling only: every step of the multigrid path runs in the
library's CUDA kernels.  Vectors are passed as device pointers -- torch CUDA
tensors (their ``data_ptr()``) or plain integers -- and streams as raw
``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).
There is no CPU fallback: if ``libhhg.so`` has not been built, importing this
module raises ImportError.  ``HHG_LIBRARY=checked`` in the environment loads
the bounds-checking build ``libhhg_checked.so`` instead (device-side index
checks; a failed check is reported as ERR_BOUNDS).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_VARIANT = os.environ.get("HHG_LIBRARY", "")
if _VARIANT not in ("", "checked"):
    raise ImportError(f"HHG_LIBRARY={_VARIANT!r}: expected 'checked' or unset")
LIB_PATH = os.path.join(_HERE, "libhhg_checked.so" if _VARIANT == "checked" else "libhhg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} not built: run `python -m paper_1805_10167_gb300.build"
                      f"{' --checked' if _VARIANT else ''}` (or __graft_entry__.build())")
lib = C.CDLL(LIB_PATH)

(OK, ERR_ARG, ERR_MESH, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_NAN, ERR_TIMEOUT, ERR_BREAKDOWN,
 ERR_BOUNDS) = range(10)
F64, F32 = 0, 1
SWEEP_RING, SWEEP_STRIP = 0, 1
ARITH_IEEE, ARITH_DFLOAT = 0, 1
GS_FWD, GS_BWD, JACOBI = 0, 1, 2
SOLVE_MG, SOLVE_IR, SOLVE_FGMRES, SOLVE_PCG, SOLVE_FPCG = 0, 1, 2, 3, 4
SMOOTH_GS, SMOOTH_LEARNED, SMOOTH_LEARNED_GS = 0, 1, 2
TC_MMA_SYNC, TC_TCGEN05 = 0, 1
LEARNED_NPARAMS = 2913


class Info(C.Structure):
    _fields_ = [("N", C.c_int32), ("n_edge_colours", C.c_int32), ("n_nodes", C.c_int64),
                ("n_free", C.c_int64), ("vec_len", C.c_int64), ("n_elems", C.c_int64),
                ("row_stride", C.c_int64), ("v_off", C.c_int64), ("e_off", C.c_int64),
                ("f_off", C.c_int64), ("edge_stride", C.c_int64), ("face_stride", C.c_int64),
                ("n_vertices", C.c_int32), ("n_edges", C.c_int32), ("n_faces", C.c_int32),
                ("max_level", C.c_int32)]


class VcycleOpts(C.Structure):
    _fields_ = [("nu1", C.c_int32), ("nu2", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("max_iter", C.c_int32), ("tol", C.c_double), ("smoother", C.c_int32),
                ("restart", C.c_int32)]


class SolveReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("r0", C.c_double),
                ("r_final", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_cap", C.c_int32), ("smoother_used", C.c_int32),
                ("judge_learned", C.c_double), ("judge_gs", C.c_double)]


class P2Opts(C.Structure):
    _fields_ = [("nu1", C.c_int32), ("nu2", C.c_int32), ("nu1c", C.c_int32), ("nu2c", C.c_int32),
                ("max_iter", C.c_int32), ("tol", C.c_double)]


class StokesOpts(C.Structure):
    _fields_ = [("delta", C.c_double), ("omega", C.c_double), ("nvel", C.c_int32), ("coarse_level", C.c_int32),
                ("nu_growth", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "hhg_mesh_create": [C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32), C.c_int64,
                        C.POINTER(C.c_uint8), C.c_int32, C.POINTER(_P)],
    "hhg_mesh_destroy": [_P],
    "hhg_mesh_info": [_P, C.c_int32, C.POINTER(Info)],
    "hhg_set_coefficient": [_P, _P, _P],
    "hhg_from_canonical": [_P, C.c_int32, C.c_int32, _P, _P, _P],
    "hhg_to_canonical": [_P, C.c_int32, C.c_int32, _P, _P, _P],
    "hhg_dof_coords": [_P, C.c_int32, _P, _P],
    "hhg_sync": [_P, _P],
    "hhg_coarse_tail": [_P, C.c_int32, C.POINTER(C.c_int32)],
    "hhg_p2_apply": [_P, C.c_int32, _P, _P, _P],
    "hhg_p2_residual": [_P, C.c_int32, _P, _P, _P, _P, _P],
    "hhg_p2_smooth": [_P, C.c_int32, _P, _P, C.c_int32, C.c_int32, _P],
    "hhg_p2_cycle": [_P, C.c_int32, _P, _P, C.POINTER(P2Opts), _P],
    "hhg_p2_solve": [_P, C.c_int32, _P, _P, C.POINTER(P2Opts), C.POINTER(SolveReport), _P],
    "hhg_stokes_setup": [_P, C.POINTER(StokesOpts)],
    "hhg_stokes_apply": [_P, C.c_int32] + [_P] * 7,
    "hhg_stokes_residual": [_P, C.c_int32] + [_P] * 11,
    "hhg_stokes_smooth": [_P, C.c_int32] + [_P] * 6 + [C.c_int32, C.c_int32, _P],
    "hhg_stokes_vcycle": [_P, C.c_int32] + [_P] * 6 + [C.c_int32, C.c_int32, _P],
    "hhg_stokes_solve": [_P, C.c_int32] + [_P] * 6 + [C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                                       C.POINTER(SolveReport), _P],
    "hhg_stokes_solve_ir": [_P, C.c_int32] + [_P] * 6 + [C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                                          C.POINTER(SolveReport), _P],
    "hhg_stokes_diag": [_P, C.c_int32, _P, _P],
    "hhg_debug_wait_limit": [_P, C.c_int32, C.c_int64],
    "hhg_apply": [_P, C.c_int32, C.c_int32, _P, _P, _P],
    "hhg_residual": [_P, C.c_int32, C.c_int32, _P, _P, _P, _P, _P],
    "hhg_assign": [_P, C.c_int32, C.c_int32, C.c_double, _P, C.c_double, _P, _P, _P],
    "hhg_dot": [_P, C.c_int32, C.c_int32, _P, _P, _P, _P],
    "hhg_dot_noalloc": [_P, C.c_int32, C.c_int32, _P, _P, _P, _P],
    "hhg_restrict": [_P, C.c_int32, C.c_int32, _P, _P, _P],
    "hhg_prolongate_add": [_P, C.c_int32, C.c_int32, _P, _P, _P],
    "hhg_smooth": [_P, C.c_int32, C.c_int32, _P, _P, C.c_int32, C.c_int32, C.c_double, _P],
    "hhg_vcycle": [_P, C.c_int32, C.c_int32, _P, _P, C.POINTER(VcycleOpts), _P],
    "hhg_solve": [_P, C.c_int32, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveReport), _P],
    "hhg_tune": [_P, C.c_int32, _P],
    "hhg_fp64_arith": [_P, C.c_int32, C.POINTER(C.c_int32)],
    "hhg_sweep_config": [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "hhg_batch_create": [C.c_int32, C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int64),
                         C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                         C.POINTER(_P)],
    "hhg_batch_destroy": [_P],
    "hhg_batch_info": [_P, C.c_int32, C.POINTER(Info)],
    "hhg_batch_tune": [_P, _P],
    "hhg_batch_solve": [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(SolveOpts), C.POINTER(SolveReport), _P],
    "hhg_learned_set_weights": [_P, C.POINTER(C.c_float), C.c_int64],
    "hhg_learned_get_weights": [_P, C.POINTER(C.c_float), C.c_int64],
    "hhg_learned_apply": [_P, C.c_int32, C.c_int32, _P, _P, _P, _P],
    "hhg_learned_tensor_path": [_P, C.c_int32, C.POINTER(C.c_int32)],
    "hhg_learned_grad": [_P, C.c_int32, _P, _P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_float),
                         C.POINTER(C.c_float), _P],
    "hhg_learned_train": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_uint64,
                          C.POINTER(C.c_float), _P],
    "hhg_profile_begin": [C.c_uint32, C.c_int32],
    "hhg_profile_end": [C.POINTER(C.c_int64), C.POINTER(C.c_double)],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.hhg_last_error.argtypes = [C.c_char_p, C.c_size_t]
lib.hhg_last_error.restype = C.c_size_t

EXPORTED = sorted(list(_SIGS) + ["hhg_last_error"])


K_FACE_GS, K_FACE_ROWS, K_EDGE_VERTEX, K_TRANSFER, K_GHOST, K_OTHER, K_COUNT = range(7)
K_NAMES = ["face_gs", "face_rows", "edge_vertex", "transfer", "ghost", "other"]


# index-check failures reported when a mesh was closed (bounds-checking build;
# kept here too because a mesh closed by the garbage collector cannot raise)
BOUNDS_FAILURES: list = []


class HHGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hhg status {status}: {msg}")
        self.status = status


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib.hhg_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(status):
    if status != OK:
        raise HHGError(status, last_error())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def profile_begin(mask, level):
    """Start counting launches (all classes) and timing classes in `mask` on `level`."""
    _check(lib.hhg_profile_begin(int(mask), int(level)))


def profile_end():
    """Returns (launches per class, milliseconds per class) since profile_begin."""
    n = (C.c_int64 * K_COUNT)()
    ms = (C.c_double * K_COUNT)()
    _check(lib.hhg_profile_end(n, ms))
    return list(n), list(ms)


class Mesh:
    """A macro mesh with its level hierarchy and device workspaces."""

    def __init__(self, xy, tri, max_level, dirichlet_vertex=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        dv = None
        if dirichlet_vertex is not None:
            dv = np.ascontiguousarray(dirichlet_vertex, dtype=np.uint8)
        h = _P()
        st = lib.hhg_mesh_create(
            xy.ctypes.data_as(C.POINTER(C.c_double)), xy.shape[0],
            tri.ctypes.data_as(C.POINTER(C.c_int32)), tri.shape[0],
            dv.ctypes.data_as(C.POINTER(C.c_uint8)) if dv is not None else None,
            int(max_level), C.byref(h))
        _check(st)
        self.h = h
        self.max_level = int(max_level)

    def close(self):
        if getattr(self, "h", None):
            h, self.h = self.h, None
            st = lib.hhg_mesh_destroy(h)
            if st == ERR_BOUNDS:     # bounds-checking build: a failure not reported before
                msg = last_error()
                BOUNDS_FAILURES.append(msg)
                raise HHGError(st, msg)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, level) -> Info:
        out = Info()
        _check(lib.hhg_mesh_info(self.h, int(level), C.byref(out)))
        return out

    def set_coefficient(self, k_dev, stream=None):
        _check(lib.hhg_set_coefficient(self.h, _ptr(k_dev), _stream(stream)))

    def from_canonical(self, level, src, dst, prec=F64, stream=None):
        _check(lib.hhg_from_canonical(self.h, level, prec, _ptr(src), _ptr(dst), _stream(stream)))

    def to_canonical(self, level, src, dst, prec=F64, stream=None):
        _check(lib.hhg_to_canonical(self.h, level, prec, _ptr(src), _ptr(dst), _stream(stream)))

    # ---- P2 elements and p-multigrid (vectors: level + 1 layout)
    def p2_apply(self, level, x, y, stream=None):
        _check(lib.hhg_p2_apply(self.h, level, _ptr(x), _ptr(y), _stream(stream)))

    def p2_residual(self, level, x, b, r, norm_dev=None, stream=None):
        _check(lib.hhg_p2_residual(self.h, level, _ptr(x), _ptr(b), _ptr(r), _ptr(norm_dev), _stream(stream)))

    def p2_smooth(self, level, x, b, smoother=GS_FWD, sweeps=1, stream=None):
        _check(lib.hhg_p2_smooth(self.h, level, _ptr(x), _ptr(b), smoother, sweeps, _stream(stream)))

    def p2_cycle(self, level, x, b, nu1=2, nu2=2, nu1c=3, nu2c=3, stream=None):
        o = P2Opts(nu1, nu2, nu1c, nu2c, 100, 1e-10)
        _check(lib.hhg_p2_cycle(self.h, level, _ptr(x), _ptr(b), C.byref(o), _stream(stream)))

    def p2_solve(self, level, x, b, nu1=2, nu2=2, nu1c=3, nu2c=3, tol=1e-10, max_iter=100, stream=None,
                 raise_on_error=True):
        """Returns (status, report dict)."""
        o = P2Opts(nu1, nu2, nu1c, nu2c, max_iter, tol)
        hist = (C.c_double * (max_iter + 1))()
        rep = SolveReport(0, 0, 0.0, 0.0, hist, max_iter + 1, 0, 0.0, 0.0)
        st = lib.hhg_p2_solve(self.h, level, _ptr(x), _ptr(b), C.byref(o), C.byref(rep), _stream(stream))
        out = {"iterations": rep.iterations, "status": rep.status, "r0": rep.r0, "r_final": rep.r_final,
               "history": [hist[i] for i in range(min(rep.iterations + 1, max_iter + 1))]}
        if raise_on_error and st != OK:
            raise HHGError(st, last_error())
        return st, out

    # -------------------------------------------------------------- Stokes
    def stokes_setup(self, delta=0.3, omega=0.4, nvel=2, coarse_level=0, nu_growth=2):
        o = StokesOpts(delta, omega, nvel, coarse_level, nu_growth)
        _check(lib.hhg_stokes_setup(self.h, C.byref(o)))

    def stokes_apply(self, level, u1, u2, p, y1, y2, yp, stream=None):
        _check(lib.hhg_stokes_apply(self.h, level, *(_ptr(v) for v in (u1, u2, p, y1, y2, yp)), _stream(stream)))

    def stokes_residual(self, level, u1, u2, p, f1, f2, g, r1, r2, rp, norm_dev=None, stream=None):
        _check(lib.hhg_stokes_residual(self.h, level, *(_ptr(v) for v in (u1, u2, p, f1, f2, g, r1, r2, rp)),
                                       _ptr(norm_dev), _stream(stream)))

    def stokes_smooth(self, level, u1, u2, p, f1, f2, g, forward=True, steps=1, stream=None):
        _check(lib.hhg_stokes_smooth(self.h, level, *(_ptr(v) for v in (u1, u2, p, f1, f2, g)), int(bool(forward)),
                                     steps, _stream(stream)))

    def stokes_vcycle(self, level, u1, u2, p, f1, f2, g, nu1=2, nu2=2, stream=None):
        _check(lib.hhg_stokes_vcycle(self.h, level, *(_ptr(v) for v in (u1, u2, p, f1, f2, g)), nu1, nu2,
                                     _stream(stream)))

    def stokes_solve(self, level, u1, u2, p, f1, f2, g, nu1=2, nu2=2, tol=1e-8, max_iter=100, stream=None,
                     raise_on_error=True):
        """Returns (status, report dict)."""
        hist = (C.c_double * (max_iter + 1))()
        rep = SolveReport(0, 0, 0.0, 0.0, hist, max_iter + 1, 0, 0.0, 0.0)
        st = lib.hhg_stokes_solve(self.h, level, *(_ptr(v) for v in (u1, u2, p, f1, f2, g)), nu1, nu2, tol,
                                  max_iter, C.byref(rep), _stream(stream))
        out = {"iterations": rep.iterations, "status": rep.status, "r0": rep.r0, "r_final": rep.r_final,
               "history": [hist[i] for i in range(min(rep.iterations + 1, max_iter + 1))]}
        if raise_on_error and st != OK:
            raise HHGError(st, last_error())
        return st, out

    def stokes_solve_ir(self, level, u1, u2, p, f1, f2, g, nu1=2, nu2=2, tol=1e-8, max_iter=100, stream=None,
                        raise_on_error=True):
        """FP32 variable V-cycles inside FP64 iterative refinement.  Returns
        (status, report dict)."""
        hist = (C.c_double * (max_iter + 1))()
        rep = SolveReport(0, 0, 0.0, 0.0, hist, max_iter + 1, 0, 0.0, 0.0)
        st = lib.hhg_stokes_solve_ir(self.h, level, *(_ptr(v) for v in (u1, u2, p, f1, f2, g)), nu1, nu2, tol,
                                     max_iter, C.byref(rep), _stream(stream))
        out = {"iterations": rep.iterations, "status": rep.status, "r0": rep.r0, "r_final": rep.r_final,
               "history": [hist[i] for i in range(min(rep.iterations + 1, max_iter + 1))]}
        if raise_on_error and st != OK:
            raise HHGError(st, last_error())
        return st, out

    def stokes_diag(self, level, s_out, stream=None):
        _check(lib.hhg_stokes_diag(self.h, level, _ptr(s_out), _stream(stream)))

    def coarse_tail(self, level=None):
        """Reads, or sets when level is given, the coarse-tail cut-off (0 = off);
        returns the cut-off in effect for FP64 cycles."""
        v = C.c_int32(level or 0)
        _check(lib.hhg_coarse_tail(self.h, 0 if level is None else 1, C.byref(v)))
        return v.value

    def sync(self, stream=None):
        _check(lib.hhg_sync(self.h, _stream(stream)))

    def debug_wait_limit(self, extra_arrivals, max_polls=0):
        _check(lib.hhg_debug_wait_limit(self.h, extra_arrivals, max_polls))

    def dof_coords(self, level, xy_dev, stream=None):
        _check(lib.hhg_dof_coords(self.h, level, _ptr(xy_dev), _stream(stream)))

    def apply(self, level, x, y, prec=F64, stream=None):
        _check(lib.hhg_apply(self.h, level, prec, _ptr(x), _ptr(y), _stream(stream)))

    def residual(self, level, x, b, r, norm_dev=None, prec=F64, stream=None):
        _check(lib.hhg_residual(self.h, level, prec, _ptr(x), _ptr(b), _ptr(r), _ptr(norm_dev),
                                _stream(stream)))

    def assign(self, level, alpha, x1, beta, x2, dst, prec=F64, stream=None):
        _check(lib.hhg_assign(self.h, level, prec, float(alpha), _ptr(x1), float(beta), _ptr(x2),
                              _ptr(dst), _stream(stream)))

    def dot(self, level, x1, x2, out_dev, prec=F64, stream=None):
        _check(lib.hhg_dot(self.h, level, prec, _ptr(x1), _ptr(x2), _ptr(out_dev), _stream(stream)))

    def dot_noalloc(self, level, x1, x2, out_dev, prec=F64, stream=None):
        """hhg_dot without any device allocation (static scratch; see include/hhg.h)."""
        _check(lib.hhg_dot_noalloc(self.h, level, prec, _ptr(x1), _ptr(x2), _ptr(out_dev),
                                   _stream(stream)))

    def restrict(self, fine_level, r_fine, b_coarse, prec=F64, stream=None):
        _check(lib.hhg_restrict(self.h, fine_level, prec, _ptr(r_fine), _ptr(b_coarse), _stream(stream)))

    def prolongate_add(self, fine_level, x_coarse, x_fine, prec=F64, stream=None):
        _check(lib.hhg_prolongate_add(self.h, fine_level, prec, _ptr(x_coarse), _ptr(x_fine),
                                      _stream(stream)))

    def smooth(self, level, x, b, smoother=GS_FWD, sweeps=1, omega=2.0 / 3.0, prec=F64, stream=None):
        _check(lib.hhg_smooth(self.h, level, prec, _ptr(x), _ptr(b), smoother, sweeps, omega,
                              _stream(stream)))

    # ---- learned smoother
    def learned_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib.hhg_learned_set_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size))

    def learned_get_weights(self):
        w = np.zeros(LEARNED_NPARAMS, dtype=np.float32)
        _check(lib.hhg_learned_get_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size))
        return w

    def learned_apply(self, level, s, x=None, d=None, prec=F64, stream=None):
        _check(lib.hhg_learned_apply(self.h, level, prec, _ptr(s), _ptr(x), _ptr(d), _stream(stream)))

    def learned_tensor_path(self, path=None):
        """Reads, or sets when path is given, the network kernel's tensor-core
        path (TC_MMA_SYNC / TC_TCGEN05)."""
        v = C.c_int32(path or 0)
        _check(lib.hhg_learned_tensor_path(self.h, 0 if path is None else 1, C.byref(v)))
        return v.value

    def learned_grad(self, X, S, crops, K=None, stream=None):
        crops = np.ascontiguousarray(crops, dtype=np.int32).reshape(-1, 4)
        g = np.zeros(LEARNED_NPARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(lib.hhg_learned_grad(self.h, crops.shape[0], _ptr(X), _ptr(S), _ptr(K),
                                    crops.ctypes.data_as(C.POINTER(C.c_int32)),
                                    g.ctypes.data_as(C.POINTER(C.c_float)),
                                    loss.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)))
        return float(loss[0]), g

    def learned_train(self, level, n_pairs=10000, epochs=20, batch=128, lr=1e-3, seed=0, stream=None):
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(lib.hhg_learned_train(self.h, level, n_pairs, epochs, batch, lr, seed,
                                     hist.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)))
        return hist[:epochs]

    def tune(self, prec=F64, stream=None):
        _check(lib.hhg_tune(self.h, prec, _stream(stream)))

    def fp64_arith(self, mode=None):
        """Reads, or sets when mode is given, the arithmetic of the FP64 face
        kernels (ARITH_IEEE / ARITH_DFLOAT)."""
        v = C.c_int32(mode or 0)
        _check(lib.hhg_fp64_arith(self.h, 0 if mode is None else 1, C.byref(v)))
        return v.value

    def sweep_config(self, level, prec=F64, variant=None, param=None):
        """Reads the face-sweep kernel (SWEEP_RING / SWEEP_STRIP) and its split
        of one level, or sets them when variant and param are given."""
        v, p = C.c_int32(variant or 0), C.c_int32(param or 0)
        set_ = variant is not None
        _check(lib.hhg_sweep_config(self.h, level, prec, 1 if set_ else 0, C.byref(v), C.byref(p)))
        return v.value, p.value

    def vcycle(self, level, x, b, nu1=3, nu2=3, prec=F64, stream=None):
        o = VcycleOpts(nu1, nu2)
        _check(lib.hhg_vcycle(self.h, level, prec, _ptr(x), _ptr(b), C.byref(o), _stream(stream)))

    def solve(self, level, x, b, mode=SOLVE_MG, nu1=3, nu2=3, tol=1e-10, max_iter=100,
              stream=None, history=True, raise_on_error=True, smoother=SMOOTH_GS, restart=20):
        """Returns (status, report dict)."""
        o = SolveOpts(mode, nu1, nu2, max_iter, tol, smoother, restart)
        hist = (C.c_double * (max_iter + 1))()
        rep = SolveReport(0, 0, 0.0, 0.0, hist if history else None, max_iter + 1 if history else 0, 0, 0.0, 0.0)
        st = lib.hhg_solve(self.h, level, _ptr(x), _ptr(b), C.byref(o), C.byref(rep), _stream(stream))
        out = {"iterations": rep.iterations, "status": rep.status, "r0": rep.r0,
               "r_final": rep.r_final, "smoother_used": rep.smoother_used,
               "judge_learned": rep.judge_learned, "judge_gs": rep.judge_gs,
               "history": [hist[i] for i in range(min(rep.iterations + 1, max_iter + 1))]}
        if raise_on_error and st != OK:
            raise HHGError(st, last_error())
        return st, out


class Batch:
    """Independent problems solved together (see hhg_batch_create)."""

    def __init__(self, meshes, levels):
        n = len(meshes)
        self._xy = [np.ascontiguousarray(m[0], dtype=np.float64) for m in meshes]
        self._tri = [np.ascontiguousarray(m[1], dtype=np.int32) for m in meshes]
        xy_p = (C.POINTER(C.c_double) * n)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in self._xy])
        tri_p = (C.POINTER(C.c_int32) * n)(*[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in self._tri])
        nv = (C.c_int64 * n)(*[a.shape[0] for a in self._xy])
        nt = (C.c_int64 * n)(*[a.shape[0] for a in self._tri])
        lv = (C.c_int32 * n)(*[int(v) for v in levels])
        h = _P()
        _check(lib.hhg_batch_create(n, xy_p, nv, tri_p, nt, lv, C.byref(h)))
        self.h, self.n = h, n

    def close(self):
        if getattr(self, "h", None):
            lib.hhg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, p) -> Info:
        out = Info()
        _check(lib.hhg_batch_info(self.h, int(p), C.byref(out)))
        return out

    def tune(self, stream=None):
        _check(lib.hhg_batch_tune(self.h, _stream(stream)))

    def solve(self, xs, bs, mode=SOLVE_FPCG, nu1=3, nu2=3, tol=1e-10, max_iter=100, stream=None,
              raise_on_error=True):
        """xs, bs: per-problem device vectors in canonical order.  Returns
        (status, list of per-problem report dicts)."""
        n = self.n
        xp = (_P * n)(*[_ptr(v) for v in xs])
        bp = (_P * n)(*[_ptr(v) for v in bs])
        o = SolveOpts(mode, nu1, nu2, max_iter, tol)
        reps = (SolveReport * n)()
        st = lib.hhg_batch_solve(self.h, xp, bp, C.byref(o), reps, _stream(stream))
        out = [{"iterations": r.iterations, "status": r.status, "r0": r.r0, "r_final": r.r_final} for r in reps]
        if raise_on_error and st != OK:
            raise HHGError(st, last_error())
        return st, out
