"""1D Lagrange basis by the direct product formula (oracle; test
infrastructure only).

For nodes x_0..x_p the j-th basis function is
  l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)
and its derivative is
  l'_j(x) = sum_{k != j} 1/(x_j - x_k) prod_{m != j,k} (x - x_m) / (x_j - x_m).

B1d[k, j] = l_j(xq_k) and G1d[k, j] = l'_j(xq_k) are the 1D factors of the
basis evaluator B (Sec. 4.4, Eq. for B_ki as a product of 1D factors).
"""

import numpy as np


def basis_1d(nodes, pts):
    """(B, G) with B[k, j] = l_j(pts[k]) and G[k, j] = l'_j(pts[k])."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    n = nodes.size
    B = np.zeros((pts.size, n))
    G = np.zeros((pts.size, n))
    for j in range(n):
        for k, x in enumerate(pts):
            val = 1.0
            for m in range(n):
                if m != j:
                    val *= (x - nodes[m]) / (nodes[j] - nodes[m])
            B[k, j] = val
            der = 0.0
            for l in range(n):
                if l == j:
                    continue
                term = 1.0 / (nodes[j] - nodes[l])
                for m in range(n):
                    if m != j and m != l:
                        term *= (x - nodes[m]) / (nodes[j] - nodes[m])
                der += term
            G[k, j] = der
    return B, G


def basis_3d(B, G):
    """Values and reference gradients of the tensor-product basis at the
    tensor-product points, from the 1D factors (Sec. 4.4, B_ki as a product
    of 1D matrices). Local DOF i = (i1, i2, i3) and point k = (k1, k2, k3)
    are both lexicographic with the first index fastest.

    Returns (phi [Q^3, D^3], dphi [Q^3, 3, D^3])."""
    Q, D = B.shape
    # Explicit loops over the 1D point indices keep the definition visible.
    phi = np.zeros((Q, Q, Q, D, D, D))
    dphi = np.zeros((3, Q, Q, Q, D, D, D))
    for k3 in range(Q):
        for k2 in range(Q):
            for k1 in range(Q):
                phi[k3, k2, k1] = np.einsum("c,b,a->cba", B[k3], B[k2], B[k1])
                dphi[0, k3, k2, k1] = np.einsum("c,b,a->cba", B[k3], B[k2], G[k1])
                dphi[1, k3, k2, k1] = np.einsum("c,b,a->cba", B[k3], G[k2], B[k1])
                dphi[2, k3, k2, k1] = np.einsum("c,b,a->cba", G[k3], B[k2], B[k1])
    phi = phi.reshape(Q ** 3, D ** 3)
    dphi = dphi.reshape(3, Q ** 3, D ** 3).transpose(1, 0, 2).copy()
    return phi, dphi
