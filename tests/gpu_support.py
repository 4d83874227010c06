"""Shared set-up of the GPU parity tests: one macro mesh seen by the CUDA
library (through the C-ABI) and by the oracle, with vectors moved between the
two in canonical order.  Imports of torch / the binding happen lazily so that
CPU-only collection never needs the GPU."""
import numpy as np

from oracle import mesh as om
from oracle import multigrid as mg
from paper_1805_10167_gb300 import inputs

FP64_TOL = 1e-12      # relative (max-norm) parity bound of every FP64 result


def macro_mesh(name):
    if name == "square":
        return inputs.unit_square_mesh()
    if name == "annulus":
        return inputs.annulus_mesh(32, 2)
    if name == "annulus16":
        return inputs.annulus_mesh(16, 4)
    if name.startswith("random"):
        seed = int(name[6:] or 5)
        return inputs.random_square_mesh(seed, 9 + seed % 7)
    raise KeyError(name)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


class Pair:
    """GPU mesh + oracle hierarchy on the same macro mesh up to level L."""

    def __init__(self, name, L, vark=False, seed=0, dirichlet=None):
        import torch
        from paper_1805_10167_gb300 import hhg
        self.torch, self.hhg = torch, hhg
        self.xy, self.tri = macro_mesh(name)
        self.L = L
        self.k = None
        if vark:
            c = inputs.element_centroids(self.xy, self.tri, L)
            self.k = inputs.grf_coefficient(c, seed=42 + seed)
        self.M = om.MacroMesh(self.xy, self.tri, dirichlet_vertex=dirichlet)
        self.H = mg.Hierarchy(self.M, L, self.k)
        self.g = hhg.Mesh(self.xy, self.tri, L, dirichlet_vertex=dirichlet)
        if vark:
            self.k_dev = torch.tensor(self.k, dtype=torch.float64, device="cuda")
            self.g.set_coefficient(self.k_dev)
        self.rng = np.random.default_rng(1000 + seed)

    def info(self, l):
        return self.g.info(l)

    def dtype(self, prec):
        return self.torch.float64 if prec == self.hhg.F64 else self.torch.float32

    def new(self, l, prec=0):
        return self.torch.zeros(self.info(l).vec_len, dtype=self.dtype(prec), device="cuda")

    def to_dev(self, l, canon, prec=0):
        t = self.torch
        src = t.tensor(np.asarray(canon), dtype=self.dtype(prec), device="cuda")
        out = self.new(l, prec)
        self.g.from_canonical(l, src, out, prec=prec)
        return out

    def from_dev(self, l, v, prec=0):
        t = self.torch
        dst = t.zeros(self.info(l).n_nodes, dtype=self.dtype(prec), device="cuda")
        self.g.to_canonical(l, v, dst, prec=prec)
        t.cuda.synchronize()
        return dst.double().cpu().numpy()

    def random(self, l, zero_dirichlet=False):
        v = self.rng.standard_normal(self.H.levels[l].n)
        if zero_dirichlet:
            v[~self.H.levels[l].free] = 0.0
        return v

    def close(self):
        self.g.close()
