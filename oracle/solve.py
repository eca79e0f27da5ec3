"""Essential boundary conditions, Jacobi-PCG and dense Cholesky (oracle; test
infrastructure only).

Boundary conditions (Sec. 5.1 on FormLinearSystem: A = P^T Ahat P plus
"further modifications" for essential conditions, which the paper leaves
unstated). Reading: symmetric elimination. With E the diagonal 0/1 selector
of essential DOFs and g their prescribed values,
  A_c = (I - E) A (I - E) + E,   b_c = (I - E)(b - A g) + E g.

Solver (the CG call of Sec. 5.2 with a relative tolerance and an iteration
cap): textbook preconditioned conjugate gradients (Saad, Iterative Methods
for Sparse Linear Systems, Alg. 9.1) with the Jacobi preconditioner
M = diag(A_c), starting from x0, stopping when the recursively updated
residual satisfies ||r||_2 <= rtol ||b||_2; the true residual is then
recomputed and, if it is still above the tolerance, the iteration restarts
from the current iterate (up to the cap).
"""

import numpy as np
import scipy.sparse as sp


def constrain(A, ess):
    """A_c = (I-E) A (I-E) + E as a CSR matrix."""
    n = A.shape[0]
    keep = np.ones(n)
    keep[np.asarray(ess, dtype=np.int64)] = 0.0
    Dk = sp.diags(keep)
    Ac = (Dk @ A @ Dk + sp.diags(1.0 - keep)).tocsr()
    Ac.sort_indices()
    return Ac


def constrain_rhs(A, b, ess, g=None):
    """b_c = (I-E)(b - A g) + E g (g = 0 when not given)."""
    n = A.shape[0]
    ess = np.asarray(ess, dtype=np.int64)
    gfull = np.zeros(n)
    if g is not None:
        gfull[ess] = np.asarray(g, dtype=np.float64)
    bc = np.asarray(b, dtype=np.float64) - A @ gfull
    bc[ess] = gfull[ess]
    return bc


def pcg(A, b, diag=None, x0=None, rtol=1e-10, maxit=20000):
    """Jacobi-preconditioned CG on SPD A. Returns (x, info dict)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    d = A.diagonal() if diag is None else np.asarray(diag, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    it = 0
    restarts = 0
    history = []
    while True:
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * bnorm or it >= maxit:
            break
        z = r / d
        p = z.copy()
        rz = r @ z
        while it < maxit:
            q = A @ p
            pq = p @ q
            if not (pq > 0.0) or not np.isfinite(pq):
                return x, {"iterations": it, "converged": False, "breakdown": True,
                           "restarts": restarts, "history": history}
            alpha = rz / pq
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            rnorm = np.linalg.norm(r)
            history.append(rnorm)
            if rnorm <= rtol * bnorm:
                break
            z = r / d
            rz_new = r @ z
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
        restarts += 1
    true_res = np.linalg.norm(b - A @ x)
    return x, {"iterations": it, "converged": true_res <= rtol * bnorm, "breakdown": False,
               "restarts": restarts - 1, "true_relres": true_res / bnorm, "history": history}


def cholesky_solve(A, b):
    """Exact discrete solution of a small SPD system by dense Cholesky."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    L = np.linalg.cholesky(Ad)
    y = np.linalg.solve(L, b)
    return np.linalg.solve(L.T, y)
