"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
CUDA library (through its C ABI) and to the CPU oracle."""

import numpy as np

from fem_inputs import hex_lattice, lognormal, submesh
from oracle import assemble


def cuda(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make_mesh(N, perturb=0.15, seed=10, shuffle=False, drop=0):
    c, h = hex_lattice(N, perturb, seed=seed, shuffle=shuffle)
    if drop:
        c, h = submesh(c, h, np.arange(h.shape[0] - drop))
    return c, h


class Case:
    """A (mesh, p, q, coefficient) problem on both sides."""

    def __init__(self, c, h, p, q=None, kind="diffusion", coef_seed=20, oracle=True):
        import paper_1911_09220_gb300 as F
        self.c, self.h, self.p = c, h, p
        self.q = p + 2 if q is None else q
        self.kind = kind
        E = h.shape[0]
        self.coef = lognormal(coef_seed, E) if coef_seed is not None else np.ones(E)
        self.mesh = F.Mesh(c, h)
        self.space = F.Space(self.mesh, p)
        self.form = F.Form(self.space, kind, self.q, coef=cuda(self.coef))
        self.prob = assemble.Problem(c, h, p, self.q, kappa=self.coef, rho=self.coef) if oracle else None
        self.n = self.space.ndof
