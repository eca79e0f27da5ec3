"""Differentiation: compliance J = b^T u through the PA solve, gradient by the
library's adjoint kernel behind torch.autograd, checked against the oracle's
gradient and against central finite differences.

Workload of the full-size case: 64^3 hexahedra perturbed by 0.1h, p = 2,
q = 4 (2,146,689 DOFs), kappa_e = 0.01 + rho_e^3 with rho_e ~ U[0.2, 1],
source f = 1, homogeneous Dirichlet conditions on the whole boundary."""

import numpy as np
import pytest

from fem_inputs import rho_uniform, x_uniform, uniform
from oracle import assemble, gradient, solve as osolve

from gpu_util import cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _problem(N, p, seed):
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, perturb=0.1, seed=seed)
    E = h.shape[0]
    rho = rho_uniform(seed, E)
    mesh = F.Mesh(c, h)
    space = F.Space(mesh, p)
    form = F.Form(space, "diffusion", p + 2, coef=cuda(0.01 + rho ** 3))
    ess = space.boundary_dofs()
    form.set_essential(ess)
    fq = torch.ones((E, form.nq), dtype=torch.float64, device="cuda")
    b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.rhs(fq, b)
    bc = torch.empty_like(b)
    form.lift_rhs(b, torch.zeros_like(b), bc)
    return c, h, rho, mesh, space, form, bc


def test_gradient_small_vs_oracle():
    import torch
    from paper_1911_09220_gb300.autograd import compliance
    c, h, rho, mesh, space, form, bc = _problem(6, 2, 50)
    r = torch.tensor(rho, device="cuda", requires_grad=True)
    J, u = compliance(0.01 + r ** 3, form, bc, rtol=1e-13)
    J.backward()
    g = r.grad.cpu().numpy()
    kappa = 0.01 + rho ** 3
    prob = assemble.Problem(c, h, 2, 4, kappa=kappa)
    ess = prob.num["boundary_dofs"]
    bo = prob.load(lambda Y: np.ones(Y.shape[:-1]))
    bco = osolve.constrain_rhs(prob.K, bo, ess)
    uo = osolve.cholesky_solve(osolve.constrain(prob.K, ess), bco)
    Jo = bco @ uo
    go = gradient.dJ_dkappa(prob, uo) * 3 * rho ** 2
    assert abs(J.item() - Jo) <= 1e-11 * abs(Jo)
    assert relerr(g, go) <= 1e-9
    assert np.all(g < 0)


def test_gradient_config_finite_differences_and_oracle():
    """64^3, p = 2: 16 seeded directions, central differences with
    h = 1e-4 (rho in [0.2, 1]); the adjoint gradient agrees to 1e-5
    relative. The oracle's element formula, evaluated on 512 seeded elements
    with the GPU solution, agrees to 1e-12."""
    import torch
    from paper_1911_09220_gb300.autograd import compliance
    c, h, rho, mesh, space, form, bc = _problem(64, 2, 50)
    assert space.ndof == 2146689 and space.ne == 262144
    r = torch.tensor(rho, device="cuda", requires_grad=True)
    J, u = compliance(0.01 + r ** 3, form, bc, rtol=1e-12)
    J.backward()
    g = r.grad.clone()
    E = h.shape[0]
    hstep = 1e-4
    for k in range(16):
        v = torch.tensor(uniform(51 * 1000 + k, E, -1.0, 1.0), device="cuda")
        with torch.no_grad():
            Jp, _ = compliance(0.01 + (r + hstep * v) ** 3, form, bc, rtol=1e-12, precision="mixed")
            Jm, _ = compliance(0.01 + (r - hstep * v) ** 3, form, bc, rtol=1e-12, precision="mixed")
        fd = (Jp.item() - Jm.item()) / (2 * hstep)
        ad = float((g * v).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (k, fd, ad)
    # oracle element formula on a seeded sample of elements, with the GPU solution
    kappa = 0.01 + rho ** 3
    sel = np.sort((uniform(52, 512, 0.0, 1.0) * E).astype(np.int64))
    form.set_coef(cuda(kappa))
    gk = torch.empty(E, dtype=torch.float64, device="cuda")
    form.compliance_grad(u, gk)
    e2l = space.element_dofs()
    from oracle import element
    ref = element.Reference(2, 4)
    X = c[h[sel].astype(np.int64)]
    Khat = element.stiffness(ref, X, np.ones(sel.size))
    ue = u.cpu().numpy()[e2l[sel]]
    go = -np.einsum("ei,eij,ej->e", ue, Khat, ue)
    assert relerr(gk.cpu().numpy()[sel], go) <= 1e-12


@pytest.mark.parametrize("precision", ["mixed", "mixed_ru"])
def test_tight_tolerance_mixed_solves(precision):
    """rtol = 1e-12 on the gradient workload's coefficient field (kappa =
    0.01 + rho^3, a hundredfold range; 24^3 hexes, p = 2): both FP32-inner
    solvers reach it, checked by the test's own FP64 constrained apply. The
    reliable-update solver computes its update residuals with the
    double-float operator only above 1e-6 relative: below that, the
    double-float rounding on this field (about 1e-11) would stall it."""
    import torch
    c, h, rho, mesh, space, form, bc = _problem(24, 2, 52)
    u = torch.zeros_like(bc)
    info = form.solve(bc, u, rtol=1e-12, precision=precision)
    assert info["converged"] and info["relres"] <= 1e-12, info
    y = torch.empty_like(u)
    form.apply(u, y, constrained=True)
    rel = float(torch.linalg.norm(bc - y) / torch.linalg.norm(bc))
    assert rel <= 1.01e-12, rel
