"""Parity of the quadrilateral (2D) path of the CUDA library with the 2D
oracle (oracle.twod) on the same seeded inputs: numbering, boundary and DOF
coordinates; apply (mass and diffusion, p = 1..8, q = p+1 and p+2, FP64,
FP32 and double-float, ragged element counts, shuffled and rotated meshes);
diagonal; quadrature points and load vector; Jacobi-PCG and plain CG;
compliance gradient; error paths.

Tolerances as for 3D: FP64 and double-float max-norm relative error
<= 1e-12, FP32 2e-5."""

import numpy as np
import pytest

from fem_inputs import lognormal, quad_lattice, submesh, x_uniform
from oracle import solve as osolve, twod

from gpu_util import cuda, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12

# (p, N, dropped elements): element counts that leave a ragged last block
SIZES = {1: (13, 5), 2: (11, 3), 3: (9, 4), 4: (8, 3), 5: (7, 2), 6: (6, 5), 7: (5, 2), 8: (5, 3)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _mesh(N, perturb=0.2, seed=10, shuffle=False, drop=0):
    c, q = quad_lattice(N, perturb, seed=seed, shuffle=shuffle)
    if drop:
        c, q = submesh(c, q, np.arange(q.shape[0] - drop))
    return c, q


class Case2:
    def __init__(self, c, qd, p, q=None, kind="diffusion", coef_seed=20):
        import paper_1911_09220_gb300 as F
        self.p, self.q = p, (p + 2 if q is None else q)
        E = qd.shape[0]
        self.coef = lognormal(coef_seed, E) if coef_seed is not None else np.ones(E)
        self.mesh = F.Mesh2D(c, qd)
        self.space = F.Space(self.mesh, p)
        self.form = F.Form(self.space, kind, self.q, coef=cuda(self.coef))
        self.prob = twod.Problem2(c, qd, p, self.q, kappa=self.coef, rho=self.coef)
        self.n = self.space.ndof
        self.kind = kind


@pytest.mark.parametrize("p,shuffle", [(1, False), (2, True), (3, True), (5, False), (8, True)])
def test_numbering_boundary_and_dof_coords(p, shuffle):
    N, drop = SIZES[p]
    c, qd = _mesh(N, seed=11, shuffle=shuffle, drop=drop)
    cs = Case2(c, qd, p)
    assert cs.space.ndof == cs.prob.ndof
    np.testing.assert_array_equal(cs.space.element_dofs(), cs.prob.e2l)
    np.testing.assert_array_equal(cs.space.boundary_dofs(), cs.prob.num["boundary_dofs"])
    np.testing.assert_allclose(cs.space.dof_coords().cpu().numpy(), cs.prob.dof_coords(), atol=1e-14)


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("qoff", [1, 2])
def test_apply_parity(kind, p, qoff):
    import torch
    N, drop = SIZES[p]
    c, qd = _mesh(N, seed=10 + p, shuffle=(p % 2 == 0), drop=drop)
    cs = Case2(c, qd, p, q=p + qoff, kind=kind, coef_seed=20 + p)
    x = x_uniform(30 + p, cs.n)
    ref = cs.prob.apply(kind, x)
    y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    yd = torch.empty_like(y)
    cs.form.apply(cuda(x), yd, arith="df64")
    assert relerr(yd.cpu().numpy(), ref) <= TOL
    y32 = torch.empty(cs.n, dtype=torch.float32, device="cuda")
    cs.form.apply(cuda(x, torch.float32), y32)
    assert relerr(y32.cpu().numpy().astype(np.float64), ref) <= 2e-5
    # element kernel + scatter through the ABI give the same bits as fem_apply
    ye = torch.empty(cs.space.ne * (p + 1) ** 2, dtype=torch.float64, device="cuda")
    y2 = torch.empty_like(y)
    cs.form.apply_element(cuda(x), ye)
    cs.form.scatter(ye, y2)
    assert torch.equal(y, y2)


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_diagonal(kind, p):
    import torch
    N, drop = SIZES[p]
    c, qd = _mesh(N, seed=3 + p, shuffle=True, drop=drop)
    cs = Case2(c, qd, p, kind=kind, coef_seed=40 + p)
    d = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.diagonal(d)
    assert relerr(d.cpu().numpy(), cs.prob.matrix(kind).diagonal()) <= TOL
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    cs.form.diagonal(d, constrained=True)
    ref = cs.prob.matrix(kind).diagonal().copy()
    ref[ess] = 1.0
    assert relerr(d.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("p", [1, 3, 6])
def test_qpoints_and_load(p):
    import torch
    N, drop = SIZES[p]
    c, qd = _mesh(N, seed=7, shuffle=True, drop=drop)
    cs = Case2(c, qd, p)
    xq = cs.form.qpoint_coords()
    np.testing.assert_allclose(xq.cpu().numpy(), cs.prob.qpoint_coords(), atol=1e-14)
    fq = torch.sin(3.0 * xq[..., 0]) * torch.cos(2.0 * xq[..., 1]) + 0.5
    b = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.rhs(fq.contiguous(), b)
    assert relerr(b.cpu().numpy(), cs.prob.load_from_qvalues(fq.cpu().numpy())) <= TOL


@pytest.mark.parametrize("precision", ["f64", "mixed", "df64", "mixed_ru"])
@pytest.mark.parametrize("p", [1, 4])
def test_poisson_solve(precision, p):
    """-div(kappa grad u) = f on a perturbed, shuffled mesh with lognormal
    kappa and homogeneous Dirichlet conditions: true residual by the oracle's
    CSR and agreement with its dense Cholesky solution."""
    import torch
    c, qd = _mesh(6, seed=2, shuffle=True)
    cs = Case2(c, qd, p, coef_seed=5)
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    bvec = x_uniform(9, cs.n)
    bc = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.lift_rhs(cuda(bvec), torch.zeros(cs.n, dtype=torch.float64, device="cuda"), bc)
    x = torch.zeros_like(bc)
    info = cs.form.solve(bc, x, rtol=1e-10, precision=precision)
    assert info["converged"]
    u = x.cpu().numpy()
    Ac = osolve.constrain(cs.prob.K, ess)
    bco = osolve.constrain_rhs(cs.prob.K, bvec, ess)
    assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10
    uc = osolve.cholesky_solve(Ac, bco)
    cond = np.linalg.cond(Ac.toarray())
    assert np.abs(u - uc).max() <= cond * 1e-10 * np.abs(uc).max()


@pytest.mark.parametrize("p", [2, 8])
def test_plain_cg_iterates(p):
    """precond='none' runs plain CG: k iterations from x0 = 0 match the
    oracle's CG with unit diagonal after the same k iterations."""
    import torch
    c, qd = _mesh(4, seed=6)
    cs = Case2(c, qd, p, coef_seed=None)
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    bvec = x_uniform(13, cs.n)
    bco = osolve.constrain_rhs(cs.prob.K, bvec, ess)
    Ac = osolve.constrain(cs.prob.K, ess)
    for k in (1, 5, 12):
        x = torch.zeros(cs.n, dtype=torch.float64, device="cuda")
        info = cs.form.solve(cuda(bco), x, rtol=1e-14, maxit=k, precond="none", raise_on_error=False,
                             check_every=4)
        assert info["iterations"] == k
        xo, io = osolve.pcg(Ac, bco, diag=np.ones(cs.n), rtol=1e-14, maxit=k)
        assert io["iterations"] == k
        assert relerr(x.cpu().numpy(), xo) <= 1e-9
    # Jacobi and plain CG both converge to the same solution
    xs = []
    for pc in ("jacobi", "none"):
        x = torch.zeros(cs.n, dtype=torch.float64, device="cuda")
        info = cs.form.solve(cuda(bco), x, rtol=1e-11, precond=pc)
        assert info["converged"]
        xs.append(x.cpu().numpy())
    assert relerr(xs[0], xs[1]) <= 1e-9


def test_compliance_gradient():
    """g_e = -u_e^T Khat_e u_e with Khat_e the oracle's element stiffness for
    kappa_e = 1."""
    import torch
    c, qd = _mesh(5, seed=8, shuffle=True, drop=2)
    cs = Case2(c, qd, 3, coef_seed=12)
    u = x_uniform(14, cs.n)
    g = torch.empty(cs.space.ne, dtype=torch.float64, device="cuda")
    cs.form.compliance_grad(cuda(u), g)
    Kh = twod.stiffness2(cs.prob.ref, cs.prob.coords[cs.prob.quads], np.ones(cs.space.ne))
    ue = u[cs.prob.e2l]
    ref = -np.einsum("ei,eij,ej->e", ue, Kh, ue)
    assert relerr(g.cpu().numpy(), ref) <= TOL


def test_no_alloc_entry_point_2d():
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    c, qd = _mesh(6, seed=1)
    cs = Case2(c, qd, 3)
    x = cuda(x_uniform(2, cs.n))
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    cs.form.apply(x, y0)
    B.check(F.lib().fem_apply_noalloc(cs.form._h, x.data_ptr(), y1.data_ptr(), None))
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)


def test_errors():
    import paper_1911_09220_gb300 as F
    c, qd = _mesh(3, perturb=0.0)
    # clockwise element: det J < 0
    bad = qd.copy()
    bad[4] = bad[4][::-1]
    m = F.Mesh2D(c, bad)
    s = F.Space(m, 2)
    with pytest.raises(F.FemError) as ei:
        F.Form(s, "diffusion", 4)
    assert ei.value.status == 3
    # vertex index out of range
    bad2 = qd.copy()
    bad2[0, 0] = c.shape[0]
    with pytest.raises(F.FemError):
        F.Mesh2D(c, bad2)
    # batches hold p <= 6 on quadrilaterals as on hexahedra
    m2 = F.Mesh2D(c, qd)
    f2 = F.Form(F.Space(m2, 7), "diffusion", 9)
    with pytest.raises(F.FemError) as ei:
        F.Batch([f2], 1)
    assert ei.value.status == 7
