"""p-multigrid preconditioned flexible CG (oracle; test infrastructure only).

The paper names matrix-free p-multigrid as a preconditioner for partially
assembled high-order operators without fixing an algorithm (Sec. 5.2, the
paragraph on matrix-free preconditioners). The reading implemented here,
step by step in the order it is applied, is:

* levels: orders p_0 = p, p_{l+1} = floor(p_l / 2) down to 1, on the same
  mesh with the same per-element coefficient, each rediscretised with
  q_l = p_l + (q_0 - p_0) Gauss points (the fine form's offset);
* coarse essential DOFs: a coarse DOF is essential iff every fine DOF of the
  same mesh entity (vertex, edge, face or interior of one element) is;
* prolongation P_l (n_l x n_{l+1}): nodal interpolation of the coarse
  function at the fine GLL nodes; the row of fine DOF i is taken from the
  first element slot (e, k) that holds i (element-major order), with
  coefficients I[k1,j1] I[k2,j2] I[k3,j3], I[i,j] = l^c_j(xi^f_i);
  masked P~ = (I - E_f) P (I - E_c), restriction R = P~^T;
* level operator: the constrained operator A_c = (I-E) A (I-E) + E and its
  diagonal D (1 on essential DOFs);
* smoother: K steps of Chebyshev iteration with Jacobi preconditioning
  (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1) on
  [alpha * lam_hi, lam_hi], lam_hi = beta * lam, lam = the D-Rayleigh
  quotient v^T A v / v^T D v after m power iterations v <- D^-1 A v / norm,
  started from v_i = frac(i * 2654435761 / 2^32) - 1/2 masked to free DOFs;
* coarsest level (p = 1): a fixed number of Jacobi-PCG iterations from zero;
* V-cycle: pre-smoothing from zero, restriction of the residual, recursion,
  prolongation of the correction, post-smoothing; every step is written out
  below exactly as the library performs it;
* outer iteration: flexible CG (Notay 2000; beta = z_new . (r_new - r) /
  z . r), which stays correct when the preconditioner is not a fixed linear
  map (the coarsest-level CG is not).
* elasticity (three-component vectors, component-major): every level is the
  elasticity operator with the same Lame coefficients; the coarse essential
  rule is applied to each component's mask, and P is block-diagonal with the
  scalar P in each component's block.
"""

import numpy as np
import scipy.sparse as sp

from . import assemble, elasticity, lagrange, numbering, rules
from . import solve as osolve

HASH_MUL = 2654435761


def level_orders(p):
    out = [p]
    while out[-1] > 1:
        out.append(out[-1] // 2)
    return out


def start_vector(n):
    """v_i = frac(i * 2654435761 / 2^32) - 1/2 (Knuth's multiplicative hash)."""
    i = np.arange(n, dtype=np.uint64)
    h = (i * np.uint64(HASH_MUL)) & np.uint64(0xFFFFFFFF)
    return h.astype(np.float64) / 4294967296.0 - 0.5


def interp_1d(p_f, p_c):
    """I[i, j] = l^c_j(xi^f_i): coarse GLL Lagrange basis at the fine GLL nodes."""
    B, _ = lagrange.basis_1d(rules.gll_nodes(p_c), rules.gll_nodes(p_f))
    return B


def _signature(L, p):
    """Entity signature of lattice points: per axis 0 (at 0), 2 (at p), 1 (inside)."""
    s = np.where(L == 0, 0, np.where(L == p, 2, 1))
    return s[:, 0] + 3 * s[:, 1] + 9 * s[:, 2]


def coarse_essential(e2l_f, p_f, ess_f_mask, e2l_c, p_c, n_c):
    """Coarse DOF essential iff all fine DOFs of its entity (per element) are."""
    sf = _signature(numbering.lattice(p_f), p_f)
    sc = _signature(numbering.lattice(p_c), p_c)
    ess_c = np.zeros(n_c, dtype=bool)
    fine_ess = ess_f_mask[e2l_f]                       # [E, nd_f]
    for s in np.unique(sc):
        ks = np.nonzero(sf == s)[0]
        allf = np.all(fine_ess[:, ks], axis=1)           # [E]
        for kc in np.nonzero(sc == s)[0]:
            ess_c[e2l_c[allf, kc]] = True
    return ess_c


def prolongation(e2l_f, p_f, n_f, e2l_c, p_c, n_c):
    """P (n_f x n_c) by the first-slot rule."""
    I = interp_1d(p_f, p_c)
    Lf, Lc = numbering.lattice(p_f), numbering.lattice(p_c)
    I3 = I[Lf[:, 0]][:, Lc[:, 0]] * I[Lf[:, 1]][:, Lc[:, 1]] * I[Lf[:, 2]][:, Lc[:, 2]]   # [nd_f, nd_c]
    E, ndf = e2l_f.shape
    flat = e2l_f.ravel()
    _, first = np.unique(flat, return_index=True)          # first slot of every fine DOF
    e, k = first // ndf, first % ndf
    rows = np.repeat(flat[first], I3.shape[1])
    cols = e2l_c[e].ravel()
    vals = I3[k].ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, n_c))


class Level:
    def __init__(self, prob, ess_mask):
        self.prob = prob
        self.n = prob.K.shape[0]
        self.ess = ess_mask
        K = prob.K
        self.A = osolve.constrain(K, np.nonzero(ess_mask)[0])
        d = self.A.diagonal().copy()
        self.D = d
        self.lam = None
        self.P = None     # to the next coarser level


def power_lambda(A, D, free, m):
    v = start_vector(A.shape[0]) * free
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(m):
        w = A @ v
        lam = (v @ w) / (v @ (D * v))
        u = w / D
        v = u / np.linalg.norm(u)
    return lam


class PMG:
    """Hierarchy and V-cycle. coords/hexes/p/q/kappa define the fine form;
    ess: fine essential DOF ids. lame = (lambda, mu): the elasticity form
    instead (kappa unused; ess ids index the 3 ndof vector)."""

    def __init__(self, coords, hexes, p, q, kappa, ess, cheb_order=2, alpha=0.25, beta=1.1, power_its=20,
                 coarse_its=30, fine_prob=None, lame=None):
        self.K, self.alpha, self.beta = cheb_order, alpha, beta
        self.coarse_its = coarse_its
        orders = level_orders(p)
        self.orders = orders
        dq = q - p
        if lame is None:
            vd = 1
            make = lambda pl: assemble.Problem(coords, hexes, pl, pl + dq, kappa=kappa)
        else:
            vd = 3
            make = lambda pl: elasticity.ElasticityProblem(coords, hexes, pl, pl + dq, lame[0], lame[1])
        self.vdim = vd
        probs = [fine_prob if fine_prob is not None else make(p)]
        for pl in orders[1:]:
            probs.append(make(pl))
        mask = np.zeros(vd * probs[0].ndof, dtype=bool)
        mask[np.asarray(ess, dtype=np.int64)] = True
        self.levels = [Level(probs[0], mask)]
        for l in range(1, len(orders)):
            f, c = probs[l - 1], probs[l]
            fm = self.levels[-1].ess
            m = np.concatenate([coarse_essential(f.e2l, f.p, fm[k * f.ndof:(k + 1) * f.ndof], c.e2l, c.p, c.ndof)
                                for k in range(vd)])
            self.levels.append(Level(c, m))
            Pm = prolongation(f.e2l, f.p, f.ndof, c.e2l, c.p, c.ndof)
            if vd > 1:
                Pm = sp.block_diag([Pm] * vd, format="csr")
            Ef = sp.diags((~self.levels[l - 1].ess).astype(np.float64))
            Ec = sp.diags((~m).astype(np.float64))
            self.levels[l - 1].P = (Ef @ Pm @ Ec).tocsr()
        for lv in self.levels[:-1]:
            lv.lam = power_lambda(lv.A, lv.D, (~lv.ess).astype(np.float64), power_its)

    def cheb_coeffs(self, lam):
        hi = self.beta * lam
        lo = self.alpha * hi
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        c = []
        for _ in range(1, self.K):
            rho_new = 1.0 / (2.0 * sigma - rho)
            c.append((rho_new * rho, 2.0 * rho_new / delta))
            rho = rho_new
        return theta, c

    def smooth(self, lv, r, z=None):
        """K Chebyshev steps; z = None starts from zero. Returns (z, res) with
        res = r - A z for the pre-smoother (z None), res unused otherwise."""
        theta, c = self.cheb_coeffs(lv.lam)
        pre = z is None
        if pre:
            res = r.copy()
            d = res / lv.D / theta
            z = d.copy()
        else:
            res = r - lv.A @ z
            d = res / lv.D / theta
            z = z + d
        for c1, c2 in c:
            res = res - lv.A @ d
            d = c1 * d + c2 * (res / lv.D)
            z = z + d
        if pre:
            res = res - lv.A @ d
        return z, res

    def coarse_solve(self, lv, r):
        """Fixed-count Jacobi-PCG from zero (stops early only on pq <= 0)."""
        x = np.zeros_like(r)
        res = r.copy()
        z = res / lv.D
        p = z.copy()
        rz = res @ z
        for _ in range(self.coarse_its):
            q = lv.A @ p
            pq = p @ q
            if not (pq > 0.0):
                break
            a = rz / pq
            x = x + a * p
            res = res - a * q
            z = res / lv.D
            rz_new = res @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x

    def vcycle(self, r, l=0):
        lv = self.levels[l]
        if l == len(self.levels) - 1:
            return self.coarse_solve(lv, r)
        z, res = self.smooth(lv, r)
        rc = lv.P.T @ res
        ec = self.vcycle(rc, l + 1)
        z = z + lv.P @ ec
        z, _ = self.smooth(lv, r, z)
        return z

    def fcg(self, b, x0=None, rtol=1e-10, maxit=500):
        """Flexible CG on the fine constrained operator, preconditioned by one
        V-cycle. Stops on the recursive residual; returns (x, iterations,
        true relative residual)."""
        A = self.levels[0].A
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
        r = b - A @ x
        bn = np.linalg.norm(b)
        z = self.vcycle(r)
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit and np.linalg.norm(r) > rtol * bn:
            q = A @ p
            a = rz / (p @ q)
            x = x + a * p
            rn = r - a * q
            it += 1
            if np.linalg.norm(rn) <= rtol * bn:
                r = rn
                break
            zn = self.vcycle(rn)
            beta = (zn @ (rn - r)) / rz
            rz = rn @ zn
            p = zn + beta * p
            r = rn
        return x, it, np.linalg.norm(b - A @ x) / bn
