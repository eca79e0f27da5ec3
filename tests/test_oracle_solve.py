"""Pins for the oracle's solve, RHS, gradient and sampled rows: PCG against
dense Cholesky, convergence order against a smooth exact solution, finite
differences for the compliance gradient, and the sampled-row apply against
the assembled matrix."""

import numpy as np
import pytest

from fem_inputs import hex_lattice, lognormal, rho_uniform, x_uniform
from oracle import assemble, solve, gradient


def _sin3(Y):
    return np.sin(np.pi * Y[..., 0]) * np.sin(np.pi * Y[..., 1]) * np.sin(np.pi * Y[..., 2])


def _f_sin3(Y):
    return 3 * np.pi ** 2 * _sin3(Y)


def test_pcg_matches_cholesky_config1():
    c, hx = hex_lattice(4, 0.1, seed=1)
    P = assemble.Problem(c, hx, 2, 4)
    ess = P.num["boundary_dofs"]
    b = P.load(_f_sin3)
    Ac = solve.constrain(P.K, ess)
    bc = solve.constrain_rhs(P.K, b, ess)
    u_chol = solve.cholesky_solve(Ac, bc)
    u, info = solve.pcg(Ac, bc, rtol=1e-10)
    assert info["converged"] and info["true_relres"] <= 1e-10
    cond = np.linalg.cond(Ac.toarray())
    assert np.abs(u - u_chol).max() <= cond * 1e-10 * np.abs(u_chol).max()
    assert np.all(u[ess] == 0.0)


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_order(p):
    errs = []
    for N in (2, 4, 8) if p == 1 else (2, 4, 6):
        c, hx = hex_lattice(N, 0.1, seed=2)
        P = assemble.Problem(c, hx, p, p + 2)
        ess = P.num["boundary_dofs"]
        b = P.load(_f_sin3)
        Ac = solve.constrain(P.K, ess)
        bc = solve.constrain_rhs(P.K, b, ess)
        u, info = solve.pcg(Ac, bc, rtol=1e-12)
        ui = _sin3(P.dof_coords())
        e = u - ui
        errs.append((N, np.sqrt(e @ (P.M @ e))))
    rates = [np.log(errs[i][1] / errs[i + 1][1]) / np.log(errs[i + 1][0] / errs[i][0]) for i in range(2)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)


def test_compliance_gradient_finite_differences():
    N, p = 3, 2
    c, hx = hex_lattice(N, 0.1, seed=50)
    E = hx.shape[0]
    rho = rho_uniform(50, E)

    def compliance(r):
        P = assemble.Problem(c, hx, p, p + 2, kappa=0.01 + r ** 3)
        ess = P.num["boundary_dofs"]
        b = P.load(lambda Y: np.ones(Y.shape[:-1]))
        bc = solve.constrain_rhs(P.K, b, ess)
        u = solve.cholesky_solve(solve.constrain(P.K, ess), bc)
        return b @ u, P, u

    J0, P, u = compliance(rho)
    g = gradient.dJ_dkappa(P, u) * 3 * rho ** 2
    rng = np.random.default_rng(51)
    for _ in range(4):
        v = rng.uniform(-1, 1, E)
        h = 1e-5
        fd = (compliance(rho + h * v)[0] - compliance(rho - h * v)[0]) / (2 * h)
        assert fd == pytest.approx(g @ v, rel=1e-7)
    assert np.all(g < 0)                      # more stiffness, less compliance


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
def test_sampled_rows_match_assembled(kind):
    c, hx = hex_lattice(3, 0.15, seed=13, shuffle=True)
    kappa = lognormal(23, hx.shape[0])
    P = assemble.Problem(c, hx, 3, 5, kappa=kappa, rho=kappa)
    x = x_uniform(33, P.ndof)
    y = P.apply(kind, x)
    rows = np.array([0, 5, 17, P.ndof // 2, P.ndof - 1])
    ys = assemble.sampled_apply(c, hx, P.e2l, 3, 5, kind, kappa, x, rows)
    np.testing.assert_allclose(ys, y[rows], rtol=1e-13, atol=1e-14 * np.abs(y).max())


def test_load_from_qvalues_matches_function():
    c, hx = hex_lattice(2, 0.1, seed=4)
    P = assemble.Problem(c, hx, 3, 5)
    xq = P.qpoint_coords()
    b1 = P.load(_f_sin3)
    b2 = P.load_from_qvalues(_f_sin3(xq))
    np.testing.assert_allclose(b1, b2, atol=1e-15)
    # f = 1: b sums to the volume
    b3 = P.load(lambda Y: np.ones(Y.shape[:-1]))
    assert b3.sum() == pytest.approx(1.0, abs=1e-14)
