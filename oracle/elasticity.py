"""Linear elasticity operator (oracle; test infrastructure only).

Vector H1 (three components) with per-element Lame coefficients:
  a(u, v) = sum_e int_e lambda_e (div u)(div v) + 2 mu_e eps(u):eps(v) dx,
eps(u) = (grad u + grad u^T) / 2. For the basis u = phi_j e_d, v = phi_i e_c
the element matrix is, by direct quadrature with physical gradients
g = J^-T ghat,
  K_e[(c,i),(d,j)] = sum_q w_q detJ_q [ lambda g_c(phi_i) g_d(phi_j)
                     + mu ( delta_cd g(phi_i).g(phi_j) + g_d(phi_i) g_c(phi_j) ) ].
Global vectors are component-major ("by nodes"): entry c * ndof + i.
Geometry: the trilinear map of `element.geometry`, or an order-k nodal
geometry of `curved`.
"""

import numpy as np
import scipy.sparse as sp

from . import curved, element, numbering


def stiffness(ref, X, lam, mu):
    """Element matrices [E, 3*D3, 3*D3] (rows/cols component-major) on the
    trilinear geometry of the corner coordinates X [E, 8, 3]."""
    _, _, det, Jinv = element.geometry(ref, X)
    return stiffness_from_geometry(ref, det, Jinv, lam, mu)


def stiffness_from_geometry(ref, det, Jinv, lam, mu):
    """Element matrices from det J [E, Q] and J^-1 [E, Q, 3, 3] at the points."""
    g = np.einsum("eqcr,qcd->eqrd", Jinv, ref.dphi)                # [E,Q,3,D] physical gradients
    w = ref.w[None, :] * det                                       # [E,Q]
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    E, _, _, D = g.shape
    K = np.zeros((E, 3, D, 3, D))
    lap = np.einsum("eq,eqri,eqrj->eij", w, g, g, optimize=True)   # g(phi_i).g(phi_j)
    for c in range(3):
        for d in range(3):
            gc_i_gd_j = np.einsum("eq,eqi,eqj->eij", w, g[:, :, c, :], g[:, :, d, :], optimize=True)
            gd_i_gc_j = np.einsum("eq,eqi,eqj->eij", w, g[:, :, d, :], g[:, :, c, :], optimize=True)
            blk = lam[:, None, None] * gc_i_gd_j + mu[:, None, None] * gd_i_gc_j
            if c == d:
                blk = blk + mu[:, None, None] * lap
            K[:, c, :, d, :] = blk
    return K.reshape(E, 3 * D, 3 * D)


class ElasticityProblem:
    """Assembled elasticity matrix [3 ndof, 3 ndof]. Xn, k: optional order-k
    nodal geometry (else the trilinear vertex map)."""

    def __init__(self, coords, hexes, p, q, lam, mu, Xn=None, k=0):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.hexes = np.asarray(hexes, dtype=np.int64)
        self.p, self.q = p, q
        self.E = self.hexes.shape[0]
        self.ref = element.Reference(p, q)
        self.num = numbering.build(self.hexes, p, nv=self.coords.shape[0])
        self.e2l, self.ndof = self.num["e2l"], self.num["ndof"]
        if k:
            _, _, det, Jinv = curved.geometry(curved.NodalReference(self.ref, k), Xn)
            Ke = stiffness_from_geometry(self.ref, det, Jinv, lam, mu)
        else:
            Ke = stiffness(self.ref, self.coords[self.hexes], lam, mu)
        # vector element DOF list: component c of local DOF i -> c * ndof + e2l[e, i]
        v2l = np.concatenate([self.e2l + c * self.ndof for c in range(3)], axis=1)
        rows = np.repeat(v2l, v2l.shape[1], axis=1).ravel()
        cols = np.tile(v2l, (1, v2l.shape[1])).ravel()
        self.K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(3 * self.ndof, 3 * self.ndof))
        self.K.sum_duplicates()

    def apply(self, x):
        return self.K @ np.asarray(x, dtype=np.float64)


def sampled_apply(coords, hexes, e2l, p, q, lam, mu, x, rows, ref=None):
    """(K x)_r for the vector rows r = c * ndof + i in `rows` only, each from
    the rows of the (at most 8) element matrices whose element holds DOF i
    (component-major vectors). Needs only the element DOF lists, so it works
    at sizes where no global matrix fits."""
    coords = np.asarray(coords, dtype=np.float64)
    hexes = np.asarray(hexes, dtype=np.int64)
    ref = element.Reference(p, q) if ref is None else ref
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    ndof = int(e2l.max()) + 1
    D = e2l.shape[1]
    flat = e2l.ravel()
    order = np.argsort(flat, kind="stable")
    sorted_dofs = flat[order]
    out = np.zeros(len(rows))
    for r, vi in enumerate(np.asarray(rows, dtype=np.int64)):
        c, i = divmod(int(vi), ndof)
        lo = np.searchsorted(sorted_dofs, i, side="left")
        hi = np.searchsorted(sorted_dofs, i, side="right")
        acc = 0.0
        for s in order[lo:hi]:
            e, k = divmod(int(s), D)
            Ke = stiffness(ref, coords[hexes[e:e + 1]], lam[e:e + 1], mu[e:e + 1])[0]
            xe = np.concatenate([x[d * ndof + e2l[e]] for d in range(3)])
            acc += Ke[c * D + k] @ xe
        out[r] = acc
    return out
