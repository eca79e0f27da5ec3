"""Global sparse assembly, SpMV and diagonal (oracle; test infrastructure
only).

A = sum_e G_e^T A_e G_e: the element restriction G scatters each element
matrix into global rows/columns through the element's DOF list; duplicate
entries are summed (Sec. 4.3, A = P^T G^T B^T D B G P with P = I on one
device, stored here at the T-vector level as a global sparse matrix).
"""

import numpy as np
import scipy.sparse as sp

from . import element, numbering


def csr_from_elements(Ae, e2l, ndof):
    E, nd, _ = Ae.shape
    rows = np.repeat(e2l, nd, axis=1).ravel()
    cols = np.tile(e2l, (1, nd)).ravel()
    A = sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(ndof, ndof)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


class Problem:
    """Everything the oracle knows about one (mesh, p, q) discretisation."""

    def __init__(self, coords, hexes, p, q, kappa=None, rho=None, chunk=512):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.hexes = np.asarray(hexes, dtype=np.int64)
        self.p, self.q = p, q
        self.E = self.hexes.shape[0]
        self.ref = element.Reference(p, q)
        self.num = numbering.build(self.hexes, p, nv=self.coords.shape[0])
        self.e2l = self.num["e2l"]
        self.ndof = self.num["ndof"]
        self.kappa = np.ones(self.E) if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.rho = np.ones(self.E) if rho is None else np.asarray(rho, dtype=np.float64)
        self.chunk = chunk
        self._K = None
        self._M = None

    def X(self, sl=slice(None)):
        return self.coords[self.hexes[sl]]

    def _assemble(self, which):
        blocks = []
        for s in range(0, self.E, self.chunk):
            sl = slice(s, min(s + self.chunk, self.E))
            if which == "diffusion":
                Ae = element.stiffness(self.ref, self.X(sl), self.kappa[sl])
            else:
                Ae = element.mass(self.ref, self.X(sl), self.rho[sl])
            blocks.append(csr_from_elements(Ae, self.e2l[sl], self.ndof))
        A = blocks[0]
        for b in blocks[1:]:
            A = A + b
        A.sort_indices()
        return A

    @property
    def K(self):
        if self._K is None:
            self._K = self._assemble("diffusion")
        return self._K

    @property
    def M(self):
        if self._M is None:
            self._M = self._assemble("mass")
        return self._M

    def matrix(self, kind):
        return self.K if kind == "diffusion" else self.M

    def apply(self, kind, x):
        """y = A x by CSR SpMV."""
        return self.matrix(kind) @ np.asarray(x, dtype=np.float64)

    def diagonal(self, kind):
        return self.matrix(kind).diagonal()

    def dof_coords(self):
        return numbering.dof_coords(self.coords, self.hexes, self.p, self.e2l, self.ref.nodes)

    def load(self, f):
        b = np.zeros(self.ndof)
        for s in range(0, self.E, self.chunk):
            sl = slice(s, min(s + self.chunk, self.E))
            be = element.load(self.ref, self.X(sl), f)
            np.add.at(b, self.e2l[sl].ravel(), be.ravel())
        return b

    def load_from_qvalues(self, fq):
        b = np.zeros(self.ndof)
        for s in range(0, self.E, self.chunk):
            sl = slice(s, min(s + self.chunk, self.E))
            be = element.load_from_qvalues(self.ref, self.X(sl), fq[sl])
            np.add.at(b, self.e2l[sl].ravel(), be.ravel())
        return b

    def qpoint_coords(self):
        out = []
        for s in range(0, self.E, self.chunk):
            sl = slice(s, min(s + self.chunk, self.E))
            out.append(element.qpoint_coords(self.ref, self.X(sl)))
        return np.concatenate(out, axis=0)


def sampled_apply(coords, hexes, e2l, p, q, kind, coef, x, rows, ref=None):
    """(A x)_i for the global DOFs in `rows` only, each from the rows of the
    (at most 8) element matrices whose element holds DOF i. Needs only the
    element DOF lists, so it works at sizes where no global matrix fits."""
    coords = np.asarray(coords, dtype=np.float64)
    hexes = np.asarray(hexes, dtype=np.int64)
    ref = element.Reference(p, q) if ref is None else ref
    rows = np.asarray(rows, dtype=np.int64)
    flat = e2l.ravel()
    order = np.argsort(flat, kind="stable")
    sorted_dofs = flat[order]
    out = np.zeros(rows.size)
    nd = e2l.shape[1]
    for r, i in enumerate(rows):
        lo = np.searchsorted(sorted_dofs, i, side="left")
        hi = np.searchsorted(sorted_dofs, i, side="right")
        hits = order[lo:hi]
        els, locs = hits // nd, hits % nd
        X = coords[hexes[els]]
        acc = 0.0
        for k in range(els.size):
            Xk = X[k:k + 1]
            if kind == "diffusion":
                row = element.stiffness_row(ref, Xk, coef[els[k]:els[k] + 1], locs[k])
            else:
                row = element.mass_row(ref, Xk, coef[els[k]:els[k] + 1], locs[k])
            acc += row[0] @ x[e2l[els[k]]]
        out[r] = acc
    return out
