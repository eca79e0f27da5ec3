"""High-order (curved) element geometry (oracle; test infrastructure only).

Sec. 3.1 describes mesh geometry either by vertex coordinates (the
trilinear map of `element.geometry`) or by a nodal grid function: element
K maps the reference cell through x(xhat) = sum_i x_{K,i} w_i(xhat), where
w_i are the order-k GLL Lagrange basis functions and x_{K,i} the element's
nodal coordinates. Here every element carries its own nodes at its order-k
GLL lattice (lexicographic, first index fastest, in the element's local
frame). J = dx/dxhat = sum_i x_{K,i} (grad w_i)^T; the element matrices,
the load vector and the DOF coordinates use the same plain definitions as
the trilinear oracle with this map. The quadrilateral case (CurvedProblem2)
follows the same definitions with the 2D oracle's numbering and reference
element.
"""

import numpy as np
import scipy.sparse as sp

from . import assemble, element, lagrange, numbering, rules, twod


def lattice_nodes(k):
    """Reference coordinates of the order-k GLL lattice [(k+1)^3, 3]."""
    return rules.gll_nodes(k)[numbering.lattice(k)]


def nodes_from_corners(X, k):
    """Nodal coordinates [E, (k+1)^3, 3] of the trilinear map of corner
    coordinates X [E, 8, 3] at the order-k GLL lattice (the same geometry,
    written as a grid function)."""
    xi = lattice_nodes(k)
    N = np.ones((xi.shape[0], 8))
    for v in range(8):
        for d in range(3):
            N[:, v] *= np.where(numbering.CORNERS[v, d] == 1, xi[:, d], 1.0 - xi[:, d])
    return np.einsum("kv,evr->ekr", N, X)


class NodalReference:
    """Order-k geometry basis tabulated at the quadrature points of `ref`."""

    def __init__(self, ref, k):
        self.k = k
        Bk, Gk = lagrange.basis_1d(rules.gll_nodes(k), ref.qpts)
        self.phi, self.dphi = lagrange.basis_3d(Bk, Gk)      # [Q3, K3], [Q3, 3, K3]


def _det_inv(J):
    a, b, c = J[..., 0, 0], J[..., 0, 1], J[..., 0, 2]
    d, e, f = J[..., 1, 0], J[..., 1, 1], J[..., 1, 2]
    g, h, i = J[..., 2, 0], J[..., 2, 1], J[..., 2, 2]
    cof = np.empty_like(J)
    cof[..., 0, 0] = e * i - f * h
    cof[..., 0, 1] = -(d * i - f * g)
    cof[..., 0, 2] = d * h - e * g
    cof[..., 1, 0] = -(b * i - c * h)
    cof[..., 1, 1] = a * i - c * g
    cof[..., 1, 2] = -(a * h - b * g)
    cof[..., 2, 0] = b * f - c * e
    cof[..., 2, 1] = -(a * f - c * d)
    cof[..., 2, 2] = a * e - b * d
    det = a * cof[..., 0, 0] + b * cof[..., 0, 1] + c * cof[..., 0, 2]
    return det, np.swapaxes(cof, -1, -2) / det[..., None, None]


def geometry(nref, Xn):
    """Points [E,Q3,3], J [E,Q3,3,3], detJ [E,Q3], J^-1 for nodes Xn [E,K3,3]."""
    x = np.einsum("qk,ekr->eqr", nref.phi, Xn)
    J = np.einsum("ekr,qck->eqrc", Xn, nref.dphi)
    det, Jinv = _det_inv(J)
    return x, J, det, Jinv


def stiffness(ref, nref, Xn, kappa):
    _, _, det, Jinv = geometry(nref, Xn)
    g = np.einsum("eqcr,qcd->eqrd", Jinv, ref.dphi)
    wq = ref.w[None, :] * det * np.asarray(kappa, dtype=np.float64)[:, None]
    return np.einsum("eqrd,eq,eqrf->edf", g, wq, g, optimize=True)


def mass(ref, nref, Xn, rho):
    _, _, det, _ = geometry(nref, Xn)
    wq = ref.w[None, :] * det * np.asarray(rho, dtype=np.float64)[:, None]
    return np.einsum("qd,eq,qf->edf", ref.phi, wq, ref.phi, optimize=True)


class CurvedProblem:
    """A (mesh, p, q) discretisation whose geometry is the order-k nodal
    field Xn [E, (k+1)^3, 3]; the hexes give the topology (numbering)."""

    def __init__(self, hexes, Xn, k, p, q, kappa=None, rho=None):
        self.hexes = np.asarray(hexes, dtype=np.int64)
        self.Xn = np.asarray(Xn, dtype=np.float64)
        self.k, self.p, self.q = k, p, q
        self.E = self.hexes.shape[0]
        self.ref = element.Reference(p, q)
        self.nref = NodalReference(self.ref, k)
        self.num = numbering.build(self.hexes, p)
        self.e2l, self.ndof = self.num["e2l"], self.num["ndof"]
        self.kappa = np.ones(self.E) if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.rho = np.ones(self.E) if rho is None else np.asarray(rho, dtype=np.float64)
        self.K = assemble.csr_from_elements(stiffness(self.ref, self.nref, self.Xn, self.kappa), self.e2l, self.ndof)
        self.M = assemble.csr_from_elements(mass(self.ref, self.nref, self.Xn, self.rho), self.e2l, self.ndof)

    def matrix(self, kind):
        return self.K if kind == "diffusion" else self.M

    def apply(self, kind, x):
        return self.matrix(kind) @ np.asarray(x, dtype=np.float64)

    def qpoint_coords(self):
        x, _, _, _ = geometry(self.nref, self.Xn)
        return x

    def dof_coords(self):
        """x at each DOF's GLL node, from the first element holding it."""
        Bk, _ = lagrange.basis_1d(rules.gll_nodes(self.k), rules.gll_nodes(self.p))
        phi, _ = lagrange.basis_3d(Bk, Bk)                  # [D3, K3]
        pts = np.einsum("dk,ekr->edr", phi, self.Xn)
        flat = self.e2l.ravel()
        _, first = np.unique(flat, return_index=True)
        out = np.zeros((self.ndof, 3))
        out[flat[first]] = pts.reshape(-1, 3)[first]
        return out

    def load_from_qvalues(self, fq):
        _, _, det, _ = geometry(self.nref, self.Xn)
        be = np.einsum("eq,qd->ed", self.ref.w[None, :] * det * fq, self.ref.phi)
        b = np.zeros(self.ndof)
        np.add.at(b, self.e2l.ravel(), be.ravel())
        return b


# ---------------------------------------------------------------- 2D ----
# The same definitions on quadrilaterals (the d = 2 case of Sec. 3.1): element
# K carries its nodal coordinates at the order-k GLL lattice of the reference
# square [(k+1)^2, 2] (first index fastest, in the element's local vertex
# frame 0:(0,0) 1:(1,0) 2:(1,1) 3:(0,1)), x(xhat) = sum_i x_{K,i} w_i(xhat)
# with the order-k GLL Lagrange products w_i, J = sum_i x_{K,i} (grad w_i)^T.

def basis_2d(B, G):
    """Values and reference gradients of the 2D tensor-product basis at the
    tensor-product points: point k = k1 + Q k2, function i = i1 + D i2.
    Returns (phi [Q^2, D^2], dphi [Q^2, 2, D^2])."""
    Q, D = B.shape
    phi = np.zeros((Q, Q, D, D))
    dphi = np.zeros((2, Q, Q, D, D))
    for k2 in range(Q):
        for k1 in range(Q):
            phi[k2, k1] = np.outer(B[k2], B[k1])
            dphi[0, k2, k1] = np.outer(B[k2], G[k1])
            dphi[1, k2, k1] = np.outer(G[k2], B[k1])
    return phi.reshape(Q * Q, D * D), dphi.reshape(2, Q * Q, D * D).transpose(1, 0, 2).copy()


def lattice_nodes2(k):
    """Reference coordinates of the order-k GLL lattice of the square [(k+1)^2, 2]."""
    return rules.gll_nodes(k)[twod.lattice2(k)]


def nodes_from_corners2(X, k):
    """Nodal coordinates [E, (k+1)^2, 2] of the bilinear map of corner
    coordinates X [E, 4, 2] at the order-k GLL lattice."""
    xi = lattice_nodes2(k)
    N = np.ones((xi.shape[0], 4))
    for v in range(4):
        for d in range(2):
            N[:, v] *= np.where(twod.CORNERS2[v, d] == 1, xi[:, d], 1.0 - xi[:, d])
    return np.einsum("kv,evr->ekr", N, X)


class NodalReference2:
    """Order-k geometry basis of the square tabulated at the Gauss points of `ref`."""

    def __init__(self, ref, k):
        self.k = k
        Bk, Gk = lagrange.basis_1d(rules.gll_nodes(k), ref.qpts)
        self.phi, self.dphi = basis_2d(Bk, Gk)      # [Q2, K2], [Q2, 2, K2]


def geometry2(nref, Xn):
    """Points [E,Q2,2], J [E,Q2,2,2], detJ [E,Q2], J^-1 for nodes Xn [E,K2,2]."""
    x = np.einsum("qk,ekr->eqr", nref.phi, Xn)
    J = np.einsum("ekr,qck->eqrc", Xn, nref.dphi)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    Jinv = np.empty_like(J)
    Jinv[..., 0, 0] = J[..., 1, 1] / det
    Jinv[..., 0, 1] = -J[..., 0, 1] / det
    Jinv[..., 1, 0] = -J[..., 1, 0] / det
    Jinv[..., 1, 1] = J[..., 0, 0] / det
    return x, J, det, Jinv


class CurvedProblem2:
    """A 2D (mesh, p, q) discretisation whose geometry is the order-k nodal
    field Xn [E, (k+1)^2, 2]; the quads give the topology (numbering). The
    element matrices are the plain direct-quadrature ones of the 2D oracle
    with this map."""

    def __init__(self, quads, Xn, k, p, q, kappa=None, rho=None, nv=None):
        self.quads = np.asarray(quads, dtype=np.int64)
        self.Xn = np.asarray(Xn, dtype=np.float64)
        self.k, self.p, self.q = k, p, q
        self.E = self.quads.shape[0]
        self.ref = twod.Reference2(p, q)
        self.nref = NodalReference2(self.ref, k)
        self.num = twod.numbering2(self.quads, p, nv=nv)
        self.e2l, self.ndof = self.num["e2l"], self.num["ndof"]
        self.kappa = np.ones(self.E) if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.rho = np.ones(self.E) if rho is None else np.asarray(rho, dtype=np.float64)
        _, _, det, Jinv = geometry2(self.nref, self.Xn)
        g = np.einsum("eqcr,qcd->eqrd", Jinv, self.ref.dphi)
        wk = self.ref.w[None, :] * det * self.kappa[:, None]
        Ke = np.einsum("eqrd,eq,eqrf->edf", g, wk, g, optimize=True)
        wr = self.ref.w[None, :] * det * self.rho[:, None]
        Me = np.einsum("qd,eq,qf->edf", self.ref.phi, wr, self.ref.phi, optimize=True)
        self.K = assemble.csr_from_elements(Ke, self.e2l, self.ndof)
        self.M = assemble.csr_from_elements(Me, self.e2l, self.ndof)

    def matrix(self, kind):
        return self.K if kind == "diffusion" else self.M

    def apply(self, kind, x):
        return self.matrix(kind) @ np.asarray(x, dtype=np.float64)

    def qpoint_coords(self):
        x, _, _, _ = geometry2(self.nref, self.Xn)
        return x

    def dof_coords(self):
        """x at each DOF's GLL node, from the first element holding it."""
        Bk, _ = lagrange.basis_1d(rules.gll_nodes(self.k), rules.gll_nodes(self.p))
        phi, _ = basis_2d(Bk, Bk)                       # [D2, K2]
        pts = np.einsum("dk,ekr->edr", phi, self.Xn)
        flat = self.e2l.ravel()
        _, first = np.unique(flat, return_index=True)
        out = np.zeros((self.ndof, 2))
        out[flat[first]] = pts.reshape(-1, 2)[first]
        return out

    def load_from_qvalues(self, fq):
        _, _, det, _ = geometry2(self.nref, self.Xn)
        be = np.einsum("eq,qd->ed", self.ref.w[None, :] * det * fq, self.ref.phi)
        b = np.zeros(self.ndof)
        np.add.at(b, self.e2l.ravel(), be.ravel())
        return b
