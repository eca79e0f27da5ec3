"""Parity of the curved-geometry path of the CUDA library (fem_mesh_set_nodes)
with the curved oracle (oracle.curved) on the same seeded inputs: apply
(diffusion and mass; FP64, double-float and FP32), diagonal, quadrature and
DOF coordinates, load vector, a Jacobi-PCG and a p-multigrid solve; order-1
nodes reproduce the vertex-geometry path; error paths. The same on
quadrilateral meshes (apply, diagonal, coordinates, load, Jacobi-PCG;
multigrid is hexahedral only). Tolerances as for the
trilinear path (FP64 and double-float 1e-12 relative, FP32 2e-5)."""

import numpy as np
import pytest

from fem_inputs import curved_nodes, lognormal, x_uniform
from oracle import curved, solve as osolve

from gpu_util import cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _case(p, k, N=3, drop=0, shuffle=True, kind="diffusion", seed=3):
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, perturb=0.1, seed=seed, shuffle=shuffle, drop=drop)
    Xn = curved_nodes(c, h, k, amp=0.05)
    kap = lognormal(seed + 2, h.shape[0])
    mesh = F.Mesh(c, h)
    mesh.set_nodes(Xn, k)
    space = F.Space(mesh, p)
    form = F.Form(space, kind, p + 2, coef=cuda(kap))
    prob = curved.CurvedProblem(h, Xn, k, p, p + 2, kappa=kap, rho=kap)
    return mesh, space, form, prob


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p,k", [(1, 1), (2, 2), (3, 2), (4, 3), (6, 4), (8, 2)])
def test_apply_parity(p, k, kind):
    import torch
    mesh, space, form, prob = _case(p, k, N=3 if p < 6 else 2, drop=1, kind=kind)
    x = x_uniform(7 + p, space.ndof)
    ref = prob.apply(kind, x)
    y = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    form.apply(cuda(x), y, arith="df64")
    assert relerr(y.cpu().numpy(), ref) <= TOL
    y32 = torch.empty(space.ndof, dtype=torch.float32, device="cuda")
    form.apply(cuda(x, torch.float32), y32)
    assert relerr(y32.cpu().numpy().astype(np.float64), ref) <= 2e-5
    d = torch.empty_like(y)
    form.diagonal(d)
    assert relerr(d.cpu().numpy(), prob.matrix(kind).diagonal()) <= TOL


@pytest.mark.parametrize("p,k", [(2, 2), (3, 3), (5, 2)])
def test_coordinates_and_load(p, k):
    import torch
    mesh, space, form, prob = _case(p, k)
    np.testing.assert_allclose(space.dof_coords().cpu().numpy(), prob.dof_coords(), atol=1e-14)
    xq = form.qpoint_coords()
    np.testing.assert_allclose(xq.cpu().numpy(), prob.qpoint_coords(), atol=1e-14)
    fq = (torch.sin(2.0 * xq[..., 0]) * xq[..., 1] + xq[..., 2] ** 2).contiguous()
    b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.rhs(fq, b)
    assert relerr(b.cpu().numpy(), prob.load_from_qvalues(fq.cpu().numpy())) <= TOL


def test_order_one_nodes_are_the_vertex_geometry():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(3, perturb=0.15, seed=9, shuffle=True)
    kap = cuda(lognormal(1, h.shape[0]))
    m0, m1 = F.Mesh(c, h), F.Mesh(c, h)
    m1.set_nodes(c[h.astype(np.int64)][:, [0, 1, 3, 2, 4, 5, 7, 6]], 1)
    f0 = F.Form(F.Space(m0, 3), "diffusion", 5, coef=kap)
    s1 = F.Space(m1, 3)
    f1 = F.Form(s1, "diffusion", 5, coef=kap)
    x = cuda(x_uniform(2, s1.ndof))
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    f0.apply(x, y0)
    f1.apply(x, y1)
    assert relerr(y1.cpu().numpy(), y0.cpu().numpy()) <= TOL
    # back to the vertex map: the next setup uses it
    m1.set_nodes(None, 0)
    f1.set_coef(kap)
    f1.apply(x, y1)
    assert relerr(y1.cpu().numpy(), y0.cpu().numpy()) <= TOL


@pytest.mark.parametrize("p,k", [(2, 2), (4, 3)])
def test_solves_on_a_curved_mesh(p, k):
    """Jacobi-PCG and p-multigrid FCG (every level on the curved geometry)
    to 1e-10, checked with the oracle's CSR."""
    import torch
    import paper_1911_09220_gb300 as F
    mesh, space, form, prob = _case(p, k, N=3)
    ess = prob.num["boundary_dofs"]
    form.set_essential(ess)
    bvec = x_uniform(4, space.ndof)
    bc = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    Ac = osolve.constrain(prob.K, ess)
    bco = osolve.constrain_rhs(prob.K, bvec, ess)
    for solver in ("pcg", "mg"):
        x = torch.zeros_like(bc)
        if solver == "pcg":
            info = form.solve(bc, x, rtol=1e-10)
        else:
            info = F.Multigrid(form).solve(bc, x, rtol=1e-10)
        assert info["converged"], (solver, info)
        u = x.cpu().numpy()
        assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10, solver


def test_errors():
    import paper_1911_09220_gb300 as F
    from fem_inputs import quad_lattice
    c, h = make_mesh(2)
    m = F.Mesh(c, h)
    Xn = curved_nodes(c, h, 2)
    assert F.lib().fem_mesh_set_nodes(m._h, 9, Xn.ctypes.data) == 1       # order out of range
    with pytest.raises(ValueError):
        m.set_nodes(Xn[:, :5], 2)
    bad = Xn.copy()
    bad[0, 3, 1] = np.nan
    with pytest.raises(F.FemError):
        m.set_nodes(bad, 2)
    # an inverted element: reflect its nodes through x = const
    inv = Xn.copy()
    inv[1, :, 0] = 2.0 * inv[1, :, 0].mean() - inv[1, :, 0]
    m.set_nodes(inv, 2)
    with pytest.raises(F.FemError) as ei:
        F.Form(F.Space(m, 2), "diffusion", 4)
    assert ei.value.status == 3
    # quadrilateral meshes: [ne, (k+1)^2, 2] nodes, the same checks
    c2, q2 = quad_lattice(2)
    m2 = F.Mesh2D(c2, q2)
    X2 = curved_nodes(c2, q2, 2)
    with pytest.raises(ValueError):
        m2.set_nodes(Xn, 2)                 # 3D nodes on a 2D mesh
    bad2 = X2.copy()
    bad2[1, 4, 0] = np.inf
    with pytest.raises(F.FemError):
        m2.set_nodes(bad2, 2)
    inv2 = X2.copy()
    inv2[2, :, 1] = 2.0 * inv2[2, :, 1].mean() - inv2[2, :, 1]
    m2.set_nodes(inv2, 2)
    with pytest.raises(F.FemError) as ei:
        F.Form(F.Space(m2, 2), "mass", 4)
    assert ei.value.status == 3


# ---------------------------------------------------------------- 2D ----
def _case2(p, k, N=4, drop=0, shuffle=True, kind="diffusion", seed=23):
    import paper_1911_09220_gb300 as F
    from fem_inputs import quad_lattice, submesh
    c, q = quad_lattice(N, 0.1, seed=seed, shuffle=shuffle)
    if drop:
        c, q = submesh(c, q, np.arange(q.shape[0] - drop))
    Xn = curved_nodes(c, q, k, amp=0.05)
    kap = lognormal(seed + 2, q.shape[0])
    mesh = F.Mesh2D(c, q)
    mesh.set_nodes(Xn, k)
    space = F.Space(mesh, p)
    form = F.Form(space, kind, p + 2, coef=cuda(kap))
    prob = curved.CurvedProblem2(q, Xn, k, p, p + 2, kappa=kap, rho=kap, nv=c.shape[0])
    return mesh, space, form, prob


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p,k", [(1, 1), (2, 2), (3, 2), (4, 3), (6, 4), (8, 8)])
def test_apply_parity_2d(p, k, kind):
    import torch
    mesh, space, form, prob = _case2(p, k, N=5 if p < 6 else 3, drop=2, kind=kind)
    x = x_uniform(31 + p, space.ndof)
    ref = prob.apply(kind, x)
    y = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    form.apply(cuda(x), y, arith="df64")
    assert relerr(y.cpu().numpy(), ref) <= TOL
    y32 = torch.empty(space.ndof, dtype=torch.float32, device="cuda")
    form.apply(cuda(x, torch.float32), y32)
    assert relerr(y32.cpu().numpy().astype(np.float64), ref) <= 2e-5
    d = torch.empty_like(y)
    form.diagonal(d)
    assert relerr(d.cpu().numpy(), prob.matrix(kind).diagonal()) <= TOL


@pytest.mark.parametrize("p,k", [(2, 2), (3, 3), (5, 2), (7, 4)])
def test_coordinates_and_load_2d(p, k):
    import torch
    mesh, space, form, prob = _case2(p, k)
    np.testing.assert_allclose(space.dof_coords().cpu().numpy(), prob.dof_coords(), atol=1e-14)
    xq = form.qpoint_coords()
    np.testing.assert_allclose(xq.cpu().numpy(), prob.qpoint_coords(), atol=1e-14)
    fq = (torch.sin(2.0 * xq[..., 0]) * xq[..., 1] + xq[..., 1] ** 2).contiguous()
    b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.rhs(fq, b)
    assert relerr(b.cpu().numpy(), prob.load_from_qvalues(fq.cpu().numpy())) <= TOL


def test_order_one_nodes_are_the_vertex_geometry_2d():
    import torch
    import paper_1911_09220_gb300 as F
    from fem_inputs import quad_lattice
    c, q = quad_lattice(5, 0.2, seed=29, shuffle=True)
    kap = cuda(lognormal(3, q.shape[0]))
    m0, m1 = F.Mesh2D(c, q), F.Mesh2D(c, q)
    m1.set_nodes(c[q.astype(np.int64)][:, [0, 1, 3, 2]], 1)
    f0 = F.Form(F.Space(m0, 4), "diffusion", 6, coef=kap)
    s1 = F.Space(m1, 4)
    f1 = F.Form(s1, "diffusion", 6, coef=kap)
    x = cuda(x_uniform(5, s1.ndof))
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    f0.apply(x, y0)
    f1.apply(x, y1)
    assert relerr(y1.cpu().numpy(), y0.cpu().numpy()) <= TOL
    np.testing.assert_allclose(s1.dof_coords().cpu().numpy(), F.Space(m0, 4).dof_coords().cpu().numpy(), atol=1e-14)
    m1.set_nodes(None, 0)
    f1.set_coef(kap)
    f1.apply(x, y1)
    assert relerr(y1.cpu().numpy(), y0.cpu().numpy()) <= TOL


@pytest.mark.parametrize("p,k", [(2, 2), (4, 3)])
def test_pcg_on_a_curved_quad_mesh(p, k):
    """Jacobi-PCG to 1e-10 on the curved quadrilateral mesh, checked with
    the oracle's CSR."""
    import torch
    mesh, space, form, prob = _case2(p, k, N=6)
    ess = prob.num["boundary_dofs"]
    form.set_essential(ess)
    bvec = x_uniform(6, space.ndof)
    bc = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    Ac = osolve.constrain(prob.K, ess)
    bco = osolve.constrain_rhs(prob.K, bvec, ess)
    x = torch.zeros_like(bc)
    info = form.solve(bc, x, rtol=1e-10)
    assert info["converged"], info
    u = x.cpu().numpy()
    assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10
