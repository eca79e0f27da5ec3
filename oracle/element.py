"""Dense element matrices by direct quadrature (oracle; test infrastructure
only).

Geometry (Sec. 3.1, Eq. mesh_eq_x): x(xhat) = sum_v x_v N_v(xhat) with the
trilinear corner functions N_v on the reference cube [0,1]^3; J = dx/dxhat
(rows: physical coordinate, columns: reference coordinate).

Diffusion (Sec. 2, A_ij = int grad phi_j . grad phi_i, with a per-element
coefficient kappa_e):
  K_e[i,j] = sum_q kappa_e w_q detJ_q (J_q^-T ghat_i(q)) . (J_q^-T ghat_j(q))
Mass (Sec. 4.4, (M_E)_ij = sum_k B_ki (D_E)_kk B_kj with
(D_E)_kk = alpha_k det J(xhat_k) rho(Phi(xhat_k))):
  M_e[i,j] = sum_q rho_e w_q detJ_q phi_i(q) phi_j(q)
Load (Sec. 2, b_i = int f phi_i):
  b_e[i] = sum_q w_q detJ_q f(x(xhat_q)) phi_i(q)

The sums run over all q^3 tensor Gauss points of the rule; nothing is
factorised. J^-1 is formed from cofactors.
"""

import numpy as np

from . import rules, lagrange
from .numbering import CORNERS


class Reference:
    """1D rules and 3D basis tables for order p with q Gauss points per
    direction."""

    def __init__(self, p, q):
        self.p, self.q = p, q
        self.nodes = rules.gll_nodes(p)
        self.qpts, self.qwts = rules.gauss_legendre(q)
        self.B, self.G = lagrange.basis_1d(self.nodes, self.qpts)
        self.phi, self.dphi = lagrange.basis_3d(self.B, self.G)   # [Q3,D3], [Q3,3,D3]
        q3 = np.stack(np.meshgrid(self.qpts, self.qpts, self.qpts, indexing="ij"), -1)
        # point k = (k1,k2,k3) with k1 fastest: coordinates (xi1, xi2, xi3)
        self.xi = q3.reshape(-1, 3)[:, ::-1].copy()                # [Q3,3]
        w3 = np.einsum("c,b,a->cba", self.qwts, self.qwts, self.qwts)
        self.w = w3.ravel()                                        # [Q3]
        # trilinear corner functions and their reference gradients at the points
        self.N = np.ones((self.xi.shape[0], 8))
        self.dN = np.ones((self.xi.shape[0], 8, 3))
        for v in range(8):
            for d in range(3):
                f = np.where(CORNERS[v, d] == 1, self.xi[:, d], 1.0 - self.xi[:, d])
                df = np.where(CORNERS[v, d] == 1, 1.0, -1.0)
                self.N[:, v] *= f
                for c in range(3):
                    self.dN[:, v, c] *= df if c == d else f


def geometry(ref, X):
    """For element corner coordinates X [E,8,3]: physical points [E,Q3,3],
    Jacobians J [E,Q3,3,3], detJ [E,Q3] and J^-1 [E,Q3,3,3] (cofactors)."""
    x = np.einsum("qv,evr->eqr", ref.N, X)
    J = np.einsum("evr,qvc->eqrc", X, ref.dN)
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
    Jinv = np.swapaxes(cof, -1, -2) / det[..., None, None]
    return x, J, det, Jinv


def stiffness(ref, X, kappa):
    """Element diffusion matrices [E, D3, D3]."""
    _, _, det, Jinv = geometry(ref, X)
    # physical gradients: grad phi = J^-T ghat, i.e. g[r] = sum_c Jinv[c, r] ghat[c]
    g = np.einsum("eqcr,qcd->eqrd", Jinv, ref.dphi)
    wq = ref.w[None, :] * det * np.asarray(kappa, dtype=np.float64)[:, None]
    return np.einsum("eqrd,eq,eqrf->edf", g, wq, g, optimize=True)


def mass(ref, X, rho):
    """Element mass matrices [E, D3, D3]."""
    _, _, det, _ = geometry(ref, X)
    wq = ref.w[None, :] * det * np.asarray(rho, dtype=np.float64)[:, None]
    return np.einsum("qd,eq,qf->edf", ref.phi, wq, ref.phi, optimize=True)


def load(ref, X, f):
    """Element load vectors [E, D3] for a source f(points [..,3]) -> values."""
    x, _, det, _ = geometry(ref, X)
    fq = f(x)
    return np.einsum("eq,qd->ed", ref.w[None, :] * det * fq, ref.phi)


def load_from_qvalues(ref, X, fq):
    """Element load vectors for source values given at the quadrature points
    fq [E, Q3]."""
    _, _, det, _ = geometry(ref, X)
    return np.einsum("eq,qd->ed", ref.w[None, :] * det * fq, ref.phi)


def stiffness_row(ref, X, kappa, i_loc):
    """Row i_loc of each element's diffusion matrix: [E, D3]. The same sum
    as `stiffness`, restricted to one test function per element."""
    _, _, det, Jinv = geometry(ref, X)
    g = np.einsum("eqcr,qcd->eqrd", Jinv, ref.dphi)               # [E,Q3,3,D3]
    gi = g[np.arange(g.shape[0]), :, :, i_loc]                    # [E,Q3,3]
    wq = ref.w[None, :] * det * np.asarray(kappa, dtype=np.float64)[:, None]
    return np.einsum("eqr,eq,eqrf->ef", gi, wq, g, optimize=True)


def mass_row(ref, X, rho, i_loc):
    _, _, det, _ = geometry(ref, X)
    wq = ref.w[None, :] * det * np.asarray(rho, dtype=np.float64)[:, None]
    pi = np.broadcast_to(ref.phi[:, i_loc].T, det.shape)          # [E,Q3]
    return np.einsum("eq,eq,qf->ef", pi, wq, ref.phi, optimize=True)


def qpoint_coords(ref, X):
    """Physical coordinates of the quadrature points [E, Q3, 3]."""
    x, _, _, _ = geometry(ref, X)
    return x
