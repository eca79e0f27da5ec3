"""Jacobi-PCG on the GPU (FP64 and FP32-inner / FP64-outer refinement) against
the oracle: the GPU solution's true residual measured by the oracle's CSR,
agreement with the oracle's dense Cholesky solution within kappa * tol, the
stopping rule, failure reporting, and the compliance gradient."""

import numpy as np
import pytest

from fem_inputs import lognormal, rho_uniform, x_uniform
from oracle import assemble, gradient, solve as osolve

from gpu_util import Case, cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _sin3(X):
    return np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])


def _gpu_rhs(cs, f):
    """b on the GPU from f evaluated at the library's own quadrature points."""
    import torch
    xq = cs.form.qpoint_coords()
    fq = f(xq)
    b = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.rhs(fq.contiguous(), b)
    return b


def _torch_f_sin3(xq):
    import torch
    return 3 * np.pi ** 2 * torch.sin(np.pi * xq[..., 0]) * torch.sin(np.pi * xq[..., 1]) * torch.sin(np.pi * xq[..., 2])


@pytest.mark.parametrize("precision", ["f64", "mixed", "df64", "mixed_ru"])
@pytest.mark.parametrize("graph", [True, False])
def test_config1_solve(precision, graph):
    """4x4x4 mesh, +-0.1h, Q2, 4^3 Gauss points, kappa = 1, 729 DOFs,
    RHS from u = sin sin sin with homogeneous Dirichlet conditions."""
    import torch
    c, h = make_mesh(4, perturb=0.1, seed=1)
    cs = Case(c, h, 2, coef_seed=None)
    assert cs.n == 729
    ess = cs.prob.num["boundary_dofs"]
    assert len(ess) == 386
    cs.form.set_essential(ess)
    b = _gpu_rhs(cs, _torch_f_sin3)
    b_or = cs.prob.load(lambda Y: 3 * np.pi ** 2 * _sin3(Y))
    assert relerr(b.cpu().numpy(), b_or) <= 1e-12
    g = torch.zeros(cs.n, dtype=torch.float64, device="cuda")
    bc = torch.empty_like(b)
    cs.form.lift_rhs(b, g, bc)
    x = torch.zeros_like(b)
    info = cs.form.solve(bc, x, rtol=1e-10, precision=precision, use_graph=graph, check_every=8)
    assert info["converged"] and info["relres"] <= 1e-10
    u = x.cpu().numpy()
    Ac = osolve.constrain(cs.prob.K, ess)
    bco = osolve.constrain_rhs(cs.prob.K, b_or, ess)
    true_rel = np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco)
    assert true_rel <= 1e-10 * (1 + 1e-2)
    uc = osolve.cholesky_solve(Ac, bco)
    cond = np.linalg.cond(Ac.toarray())
    assert np.abs(u - uc).max() <= cond * 1e-10 * np.abs(uc).max()
    assert np.all(u[ess] == 0.0)
    # the discrete solution approximates sin sin sin
    assert np.abs(u - _sin3(cs.prob.dof_coords())).max() < 0.02


@pytest.mark.parametrize("p", [1, 3, 5])
def test_solve_lognormal_nonzero_dirichlet(p):
    import torch
    c, h = make_mesh(3, perturb=0.15, seed=12, shuffle=True)
    cs = Case(c, h, p, coef_seed=22)
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    bvec = x_uniform(32, cs.n)
    gvec = x_uniform(33, cs.n)
    bc = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.lift_rhs(cuda(bvec), cuda(gvec), bc)
    x = cuda(np.where(np.isin(np.arange(cs.n), ess), gvec, 0.0))
    for precision in ("f64", "mixed", "df64", "mixed_ru"):
        xx = x.clone()
        info = cs.form.solve(bc, xx, rtol=1e-10, precision=precision)
        u = xx.cpu().numpy()
        Ac = osolve.constrain(cs.prob.K, ess)
        bco = osolve.constrain_rhs(cs.prob.K, bvec, ess, gvec[ess])
        assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10, (precision, info)
        np.testing.assert_array_equal(u[ess], gvec[ess])


def test_solve_reports_failures():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(3, seed=2)
    cs = Case(c, h, 2, oracle=False)
    cs.form.set_essential(np.array([], dtype=np.int32))   # pure Neumann mass-free: singular
    b = cuda(x_uniform(3, cs.n))
    x = torch.zeros_like(b)
    # tiny iteration cap: FEM_ENOCONV with the iteration count reported
    ess = cs.space.boundary_dofs()
    cs.form.set_essential(ess)
    info = cs.form.solve(b, x, rtol=1e-10, maxit=3, raise_on_error=False)
    assert info["status"] == 4 and not info["converged"] and info["iterations"] <= 3 + 16
    # non-finite right-hand side (host-injected): reported as breakdown, no device fault
    b2 = b.clone()
    b2[5] = float("nan")
    x.zero_()
    info = cs.form.solve(b2, x, rtol=1e-10, raise_on_error=False)
    assert info["status"] in (4, 5) and not info["converged"]
    # b = 0 gives x = 0
    x.fill_(3.0)
    info = cs.form.solve(torch.zeros_like(b), x)
    assert info["converged"] and torch.count_nonzero(x).item() == 0


def test_solve_is_deterministic():
    import torch
    c, h = make_mesh(4, seed=4)
    cs = Case(c, h, 2, oracle=False)
    cs.form.set_essential(cs.space.boundary_dofs())
    b = cuda(x_uniform(5, cs.n))
    bc = torch.empty_like(b)
    cs.form.lift_rhs(b, torch.zeros_like(b), bc)
    xs = []
    for _ in range(2):
        x = torch.zeros_like(b)
        info = cs.form.solve(bc, x)
        xs.append((x.clone(), info["iterations"]))
    assert torch.equal(xs[0][0], xs[1][0]) and xs[0][1] == xs[1][1]


@pytest.mark.parametrize("p", [1, 2, 4])
def test_compliance_gradient_kernel(p):
    """g_e = -u_e^T Khat_e u_e for a seeded u (any u: a quadratic form)."""
    import torch
    c, h = make_mesh(3, seed=50 + p, shuffle=True, drop=1)
    E = h.shape[0]
    rho = rho_uniform(50, E)
    kappa = 0.01 + rho ** 3
    import paper_1911_09220_gb300 as F
    mesh = F.Mesh(c, h)
    space = F.Space(mesh, p)
    form = F.Form(space, "diffusion", p + 2, coef=cuda(kappa))
    prob = assemble.Problem(c, h, p, p + 2, kappa=kappa)
    u = x_uniform(51, space.ndof)
    g = torch.empty(E, dtype=torch.float64, device="cuda")
    form.compliance_grad(cuda(u), g)
    assert relerr(g.cpu().numpy(), gradient.dJ_dkappa(prob, u)) <= 1e-12
