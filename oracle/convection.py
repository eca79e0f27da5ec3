"""Convection operator (oracle; test infrastructure only).

The paper lists convection among the partially assembled integrators
(Sec. 5.3, the fem directory: mass, diffusion, convection, ...). For a
velocity field beta given at the quadrature points, the element matrix of
(beta . grad u, v) (test function v = phi_i, trial u = phi_j) is

  C_e[i, j] = sum_q w_q detJ_q phi_i(q) beta_q . (J_q^-T ghat_j(q)),

the plain definition the partially assembled apply must reproduce (PA
stores D_q = w_q detJ_q J_q^-1 beta_q, so that the point value is
D_q . ghat). Geometry: the trilinear map of `element.geometry`, or an
order-k nodal geometry of `curved`.
"""

import numpy as np

from . import assemble, curved, element, numbering


def convection(ref, det, Jinv, beta):
    """Element matrices [E, D3, D3] from the geometry at the points and the
    velocity beta [E, Q3, 3] (physical components)."""
    # J^-T ghat_j: g[e, q, r, j] = sum_c Jinv[e, q, c, r] dphi[q, c, j]
    g = np.einsum("eqcr,qcj->eqrj", Jinv, ref.dphi)
    bg = np.einsum("eqr,eqrj->eqj", beta, g)               # beta . grad phi_j
    wq = ref.w[None, :] * det
    return np.einsum("qi,eq,eqj->eij", ref.phi, wq, bg, optimize=True)


class ConvectionProblem:
    """Assembled convection matrix on a (mesh, p, q) discretisation.
    beta: [E, Q3, 3] at the form's quadrature points. Xn, k: optional
    order-k nodal geometry (else the trilinear vertex map)."""

    def __init__(self, coords, hexes, p, q, beta, Xn=None, k=0):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.hexes = np.asarray(hexes, dtype=np.int64)
        self.p, self.q = p, q
        self.ref = element.Reference(p, q)
        self.num = numbering.build(self.hexes, p, nv=self.coords.shape[0])
        self.e2l, self.ndof = self.num["e2l"], self.num["ndof"]
        if k:
            self.x, _, det, Jinv = curved.geometry(curved.NodalReference(self.ref, k), Xn)
        else:
            self.x, _, det, Jinv = element.geometry(self.ref, self.coords[self.hexes])
        self.C = assemble.csr_from_elements(convection(self.ref, det, Jinv, np.asarray(beta, dtype=np.float64)),
                                            self.e2l, self.ndof)

    def apply(self, x):
        return self.C @ np.asarray(x, dtype=np.float64)
