"""Compliance gradient (oracle; test infrastructure only).

The paper has no gradient; its topology-optimisation application (LiDO,
Sec. 7) motivates it. For A(kappa) u = b with b independent of kappa and
A(kappa) = sum_e kappa_e Khat_e (Khat_e: element diffusion matrix with
kappa = 1, eliminated on essential DOFs where u = 0), the compliance
J = b^T u has dJ/dkappa_e = -u^T (dA/dkappa_e) u = -u_e^T Khat_e u_e,
and with kappa_e = 0.01 + rho_e^3, dJ/drho_e = 3 rho_e^2 dJ/dkappa_e.
"""

import numpy as np

from . import element


def dJ_dkappa(prob, u):
    """-u_e^T Khat_e u_e for every element of an oracle `Problem`."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros(prob.E)
    for s in range(0, prob.E, prob.chunk):
        sl = slice(s, min(s + prob.chunk, prob.E))
        Ke = element.stiffness(prob.ref, prob.X(sl), np.ones(sl.stop - sl.start))
        ue = u[prob.e2l[sl]]
        out[sl] = -np.einsum("ei,eij,ej->e", ue, Ke, ue)
    return out
