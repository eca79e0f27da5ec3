"""Two-dimensional (quadrilateral) H1 operators (oracle; test infrastructure
only).

The same plain definitions as the 3D oracle, on the reference square [0,1]^2:
bilinear geometry x(xhat) = sum_v x_v N_v(xhat) (Sec. 3.1), nodal GLL basis
(Sec. 3.3), q^2 Gauss points, dense element matrices by direct quadrature
  K_e[i,j] = sum_q kappa_e w_q detJ (J^-T ghat_i).(J^-T ghat_j),
  M_e[i,j] = sum_q rho_e w_q detJ phi_i phi_j,
and global assembly with the numbering of Sec. 3.4 (vertices, then edges by
first appearance in element order with local edges (0,1), (1,2), (3,2),
(0,3), DOFs from the lower to the higher global vertex, then element
interiors, lexicographic). Local vertex order: 0:(0,0) 1:(1,0) 2:(1,1)
3:(0,1) (counter-clockwise); local DOFs lexicographic, first index fastest.
The paper's 2D diffusion setup listing (Sec. 5.3) stores the same D:
alpha W adj(J) adj(J)^T / det J.
"""

import numpy as np
import scipy.sparse as sp

from . import rules, lagrange
from .assemble import csr_from_elements

CORNERS2 = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.int64)
EDGES2 = np.array([[0, 1], [1, 2], [3, 2], [0, 3]], dtype=np.int64)


def lattice2(p):
    r = np.arange(p + 1)
    i2, i1 = np.meshgrid(r, r, indexing="ij")
    return np.stack([i1.ravel(), i2.ravel()], axis=1)


def numbering2(quads, p, nv=None):
    """Global numbering and element DOF lists for quadrilaterals."""
    quads = np.asarray(quads, dtype=np.int64)
    E = quads.shape[0]
    nv = int(quads.max()) + 1 if nv is None else nv
    D = p + 1
    L = lattice2(p)
    W = np.ones((L.shape[0], 4), dtype=np.int64)       # bilinear corner weights x p^2
    for v in range(4):
        for d in range(2):
            W[:, v] *= np.where(CORNERS2[v, d] == 1, L[:, d], p - L[:, d])
    ge = quads[:, EDGES2]
    keys = np.sort(ge, axis=2).reshape(-1, 2)
    _, first, inverse = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    edge_id = rank[inverse.ravel()].reshape(E, 4)
    n_edges = order.size
    pm1 = p - 1
    off_e, off_i = nv, nv + n_edges * pm1
    ndof = off_i + E * pm1 * pm1
    e2l = np.full((E, D * D), -1, dtype=np.int64)
    for k in range(D * D):
        nz = np.nonzero(W[k])[0]
        if nz.size == 1:
            e2l[:, k] = quads[:, nz[0]]
        elif nz.size == 2:
            a, b = nz
            le = [i for i in range(4) if set(EDGES2[i]) == {a, b}][0]
            pos = np.where(quads[:, a] < quads[:, b], W[k, b], W[k, a]) // p
            e2l[:, k] = off_e + edge_id[:, le] * pm1 + (pos - 1)
        else:
            i1, i2 = L[k]
            e2l[:, k] = off_i + np.arange(E) * pm1 * pm1 + (i1 - 1) + pm1 * (i2 - 1)
    counts = np.bincount(edge_id.ravel(), minlength=n_edges)
    bnd = counts[edge_id] == 1
    mask = np.zeros(ndof, dtype=bool)
    for le in range(4):
        pts = [k for k in range(D * D) if set(np.nonzero(W[k])[0]) <= set(EDGES2[le])]
        rows = np.nonzero(bnd[:, le])[0]
        if rows.size:
            mask[e2l[np.ix_(rows, pts)].ravel()] = True
    return {"e2l": e2l, "ndof": ndof, "boundary_mask": mask, "boundary_dofs": np.nonzero(mask)[0]}


class Reference2:
    def __init__(self, p, q):
        self.p, self.q = p, q
        self.nodes = rules.gll_nodes(p)
        self.qpts, self.qwts = rules.gauss_legendre(q)
        self.B, self.G = lagrange.basis_1d(self.nodes, self.qpts)
        Q, D = self.B.shape
        # point k = k1 + Q k2, DOF i = i1 + D i2
        phi = np.zeros((Q, Q, D, D))
        dphi = np.zeros((2, Q, Q, D, D))
        for k2 in range(Q):
            for k1 in range(Q):
                phi[k2, k1] = np.outer(self.B[k2], self.B[k1])
                dphi[0, k2, k1] = np.outer(self.B[k2], self.G[k1])
                dphi[1, k2, k1] = np.outer(self.G[k2], self.B[k1])
        self.phi = phi.reshape(Q * Q, D * D)
        self.dphi = dphi.reshape(2, Q * Q, D * D).transpose(1, 0, 2).copy()
        g2 = np.stack(np.meshgrid(self.qpts, self.qpts, indexing="ij"), -1)
        self.xi = g2.reshape(-1, 2)[:, ::-1].copy()
        self.w = np.outer(self.qwts, self.qwts).ravel()
        self.N = np.ones((Q * Q, 4))
        self.dN = np.ones((Q * Q, 4, 2))
        for v in range(4):
            for d in range(2):
                f = np.where(CORNERS2[v, d] == 1, self.xi[:, d], 1.0 - self.xi[:, d])
                df = 1.0 if CORNERS2[v, d] == 1 else -1.0
                self.N[:, v] *= f
                for c in range(2):
                    self.dN[:, v, c] *= df if c == d else f


def geometry2(ref, X):
    """Points [E,Q2,2], J [E,Q2,2,2], detJ [E,Q2], J^-1 [E,Q2,2,2]."""
    x = np.einsum("qv,evr->eqr", ref.N, X)
    J = np.einsum("evr,qvc->eqrc", X, ref.dN)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    Jinv = np.empty_like(J)
    Jinv[..., 0, 0] = J[..., 1, 1] / det
    Jinv[..., 0, 1] = -J[..., 0, 1] / det
    Jinv[..., 1, 0] = -J[..., 1, 0] / det
    Jinv[..., 1, 1] = J[..., 0, 0] / det
    return x, J, det, Jinv


def stiffness2(ref, X, kappa):
    _, _, det, Jinv = geometry2(ref, X)
    g = np.einsum("eqcr,qcd->eqrd", Jinv, ref.dphi)
    wq = ref.w[None, :] * det * np.asarray(kappa, dtype=np.float64)[:, None]
    return np.einsum("eqrd,eq,eqrf->edf", g, wq, g, optimize=True)


def mass2(ref, X, rho):
    _, _, det, _ = geometry2(ref, X)
    wq = ref.w[None, :] * det * np.asarray(rho, dtype=np.float64)[:, None]
    return np.einsum("qd,eq,qf->edf", ref.phi, wq, ref.phi, optimize=True)


class Problem2:
    """Everything the oracle knows about one 2D (mesh, p, q) discretisation."""

    def __init__(self, coords, quads, p, q, kappa=None, rho=None):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int64)
        self.p, self.q, self.E = p, q, self.quads.shape[0]
        self.ref = Reference2(p, q)
        self.num = numbering2(self.quads, p, nv=self.coords.shape[0])
        self.e2l, self.ndof = self.num["e2l"], self.num["ndof"]
        self.kappa = np.ones(self.E) if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.rho = np.ones(self.E) if rho is None else np.asarray(rho, dtype=np.float64)
        X = self.coords[self.quads]
        self.K = csr_from_elements(stiffness2(self.ref, X, self.kappa), self.e2l, self.ndof)
        self.M = csr_from_elements(mass2(self.ref, X, self.rho), self.e2l, self.ndof)

    def matrix(self, kind):
        return self.K if kind == "diffusion" else self.M

    def apply(self, kind, x):
        return self.matrix(kind) @ np.asarray(x, dtype=np.float64)

    def dof_coords(self):
        L = lattice2(self.p)
        xi = self.ref.nodes[L]
        N = np.ones((L.shape[0], 4))
        for v in range(4):
            for d in range(2):
                N[:, v] *= np.where(CORNERS2[v, d] == 1, xi[:, d], 1.0 - xi[:, d])
        pts = np.einsum("kv,evr->ekr", N, self.coords[self.quads])
        out = np.zeros((self.ndof, 2))
        out[self.e2l.ravel()] = pts.reshape(-1, 2)
        return out

    def qpoint_coords(self):
        x, _, _, _ = geometry2(self.ref, self.coords[self.quads])
        return x

    def load_from_qvalues(self, fq):
        _, _, det, _ = geometry2(self.ref, self.coords[self.quads])
        be = np.einsum("eq,qd->ed", self.ref.w[None, :] * det * fq, self.ref.phi)
        b = np.zeros(self.ndof)
        np.add.at(b, self.e2l.ravel(), be.ravel())
        return b
