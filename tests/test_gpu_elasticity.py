"""Parity of the linear elasticity form (fem_form_create_elasticity) of the
CUDA library with the elasticity oracle on the same seeded inputs:
the apply in FP64, double-float and FP32 for p = 1..8 (shuffled vertex
orders, ragged last blocks, trilinear and curved geometry, both compiled
quadrature orders), its two halves, the no-allocation entry point, the
constrained apply, the assembled diagonal, the vector load vector,
Jacobi-PCG solves against the oracle's dense solution, set_lame, and the
entry points that reject a vector form (the vector p-multigrid hierarchy is
tested in test_gpu_multigrid.py). Tolerances as for diffusion
(1e-12 relative to the largest entry; FP32 2e-5)."""

import numpy as np
import pytest

from fem_inputs import curved_nodes, lognormal, x_uniform
from oracle import assemble, elasticity as oel, solve as osolve

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


# (N, dropped elements): every p spans several element blocks where the
# block holds more than one element, with a ragged last block
SIZES = {1: (4, 3), 2: (3, 2), 3: (3, 1), 4: (2, 1), 5: (2, 1), 6: (2, 3), 7: (1, 0), 8: (1, 0)}


def _setup(p, q=None, curvedk=0, seed=0):
    import paper_1911_09220_gb300 as F
    N, drop = SIZES[p]
    q = p + 2 if q is None else q
    c, h = make_mesh(N, perturb=0.15, seed=30 + p + seed, shuffle=(p % 2 == 0), drop=drop)
    mesh = F.Mesh(c, h)
    Xn = None
    if curvedk:
        Xn = curved_nodes(c, h, curvedk)
        mesh.set_nodes(Xn, curvedk)
    space = F.Space(mesh, p)
    E = h.shape[0]
    lam, mu = lognormal(40 + p, E), lognormal(50 + p, E)
    form = F.Form.elasticity(space, cuda(lam), cuda(mu), q1d=q)
    prob = oel.ElasticityProblem(c, h, p, q, lam, mu, Xn=Xn, k=curvedk)
    assert prob.ndof == space.ndof
    return form, prob, (c, h, lam, mu)


def _apply_all(form, prob, seed):
    import torch
    x = x_uniform(seed, form.n)
    ref = prob.apply(x)
    y = torch.empty(form.n, dtype=torch.float64, device="cuda")
    form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    form.apply(cuda(x), y, arith="df64")
    assert relerr(y.cpu().numpy(), ref) <= TOL
    y32 = torch.empty(form.n, dtype=torch.float32, device="cuda")
    form.apply(cuda(x, torch.float32), y32)
    assert relerr(y32.cpu().numpy().astype(np.float64), ref) <= 2e-5


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("curvedk", [0, 2])
def test_apply_parity(p, curvedk):
    if curvedk and p > 6:
        pytest.skip("curved cases up to p = 6 keep the oracle's dense element matrices small")
    form, prob, _ = _setup(p, curvedk=curvedk)
    _apply_all(form, prob, 60 + p)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_apply_parity_q_p1(p):
    """The other compiled quadrature order, q = p + 1."""
    form, prob, _ = _setup(p, q=p + 1)
    _apply_all(form, prob, 70 + p)


def test_halves_noalloc_and_constrained():
    import torch
    form, prob, (c, h, lam, mu) = _setup(3)
    n, nd, ne = form.n, (3 + 1) ** 3, h.shape[0]
    x = cuda(x_uniform(5, n))
    y = torch.empty_like(x)
    form.apply(x, y)
    ye = torch.empty(3 * ne * nd, dtype=torch.float64, device="cuda")
    form.apply_element(x, ye)
    y2 = torch.empty_like(x)
    form.scatter(ye, y2)
    assert torch.equal(y, y2)
    # the E-vector is component-major: component c of element e at (c * ne + e) * nd
    ref = prob.apply(x.cpu().numpy())
    import paper_1911_09220_gb300 as F
    import ctypes
    y3 = torch.empty_like(x)
    assert F.lib().fem_apply_noalloc(form._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y3.data_ptr()),
                                     None) == 0
    torch.cuda.synchronize()
    assert torch.equal(y, y3)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    # constrained apply: clamp the x-component of the boundary and all of one face
    ndof = form.space.ndof
    bd = form.space.boundary_dofs()
    ess = np.unique(np.concatenate([bd, bd[: len(bd) // 2] + 2 * ndof]))
    form.set_essential(ess)
    yc = torch.empty_like(x)
    form.apply(x, yc, constrained=True)
    Ac = osolve.constrain(prob.K, ess)
    assert relerr(yc.cpu().numpy(), Ac @ x.cpu().numpy()) <= TOL


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("curvedk", [0, 2])
def test_diagonal(p, curvedk):
    import torch
    form, prob, _ = _setup(p, curvedk=curvedk)
    d = torch.empty(form.n, dtype=torch.float64, device="cuda")
    form.diagonal(d)
    ref = prob.K.diagonal()
    assert relerr(d.cpu().numpy(), ref) <= TOL
    ess = np.arange(0, form.n, 7)
    form.set_essential(ess)
    form.diagonal(d, constrained=True)
    ref = ref.copy()
    ref[ess] = 1.0
    assert relerr(d.cpu().numpy(), ref) <= TOL


def test_body_force_load():
    """fem_rhs of an elasticity form: component c of the load vector is the
    scalar load of fq[c]."""
    import torch
    p = 2
    form, prob, (c, h, lam, mu) = _setup(p)
    xq = form.qpoint_coords()
    fq = torch.stack([torch.sin(xq[..., 0] + 2 * xq[..., 1]), xq[..., 2] ** 2 - 0.3, torch.cos(3 * xq[..., 0])])
    b = torch.empty(form.n, dtype=torch.float64, device="cuda")
    form.rhs(fq.contiguous(), b)
    sc = assemble.Problem(c, h, p, p + 2)
    ref = np.concatenate([sc.load_from_qvalues(fq[k].cpu().numpy()) for k in range(3)])
    assert relerr(b.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("precision", ["f64", "mixed", "df64"])
def test_solve_clamped(precision):
    """Clamped boundary (all three components), body force: Jacobi-PCG
    against the oracle's dense Cholesky solution of the constrained system."""
    import torch
    p = 2
    form, prob, (c, h, lam, mu) = _setup(p)
    ndof = form.space.ndof
    bd = form.space.boundary_dofs()
    ess = np.concatenate([bd + k * ndof for k in range(3)])
    form.set_essential(ess)
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, form.n)
    b[ess] = 0.0
    x = torch.zeros(form.n, dtype=torch.float64, device="cuda")
    info = form.solve(cuda(b), x, rtol=1e-11, precision=precision)
    assert info["converged"]
    Ac = osolve.constrain(prob.K, ess)
    ref = osolve.cholesky_solve(Ac, b)
    xs = x.cpu().numpy()
    assert np.linalg.norm(Ac @ xs - b) <= 1e-10 * np.linalg.norm(b)
    assert relerr(xs, ref) <= 1e-7


def test_set_lame_and_rejections():
    import ctypes
    import torch
    import paper_1911_09220_gb300 as F
    form, prob, (c, h, lam, mu) = _setup(2)
    E = h.shape[0]
    lam2, mu2 = lognormal(91, E), lognormal(92, E)
    form.set_lame(cuda(lam2), cuda(mu2))
    x = x_uniform(8, form.n)
    y = torch.empty(form.n, dtype=torch.float64, device="cuda")
    form.apply(cuda(x), y)
    ref = oel.ElasticityProblem(c, h, 2, 4, lam2, mu2).apply(x)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    with pytest.raises(F.FemError):
        form.set_coef(cuda(lam2))
    form.set_essential(form.space.boundary_dofs())
    with pytest.raises(F.FemError):
        F.Batch([form], 1)
    with pytest.raises(F.FemError):
        form.compliance_grad(cuda(x), torch.empty(E, dtype=torch.float64, device="cuda"))
    h_out = ctypes.c_void_p()
    L = F.lib()
    # fem_form_create refuses the kind (it needs both Lame coefficients)
    assert L.fem_form_create(form.space._h, 3, 4, None, None, ctypes.byref(h_out)) == 1
    assert L.fem_form_create_elasticity(form.space._h, 4, None, None, None, ctypes.byref(h_out)) == 1
    # quadrilateral meshes are not supported
    from fem_inputs import quad_lattice
    c2, q2 = quad_lattice(3, 0.1, seed=1)
    sp2 = F.Space(F.Mesh2D(c2, q2), 2)
    one = cuda(np.ones(q2.shape[0]))
    assert L.fem_form_create_elasticity(sp2._h, 4, ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                        None, ctypes.byref(h_out)) == 7
    # out-of-range vector DOF ids
    with pytest.raises(F.FemError):
        form.set_essential(np.array([form.n], dtype=np.int32))


@pytest.mark.parametrize("p,curvedk", [(3, 0), (3, 2), (4, 3)])
def test_multigrid_solve_trilinear_and_curved(p, curvedk):
    """p-multigrid flexible CG on the elasticity form (every level on the
    same, possibly curved, geometry; FP64 and FP32 V-cycles) to 1e-10,
    checked with the oracle's assembled operator."""
    import torch
    import paper_1911_09220_gb300 as F
    N = 2
    c, h = make_mesh(N, perturb=0.15, seed=7 + p, shuffle=True)
    mesh = F.Mesh(c, h)
    Xn = None
    if curvedk:
        Xn = curved_nodes(c, h, curvedk)
        mesh.set_nodes(Xn, curvedk)
    space = F.Space(mesh, p)
    E = h.shape[0]
    lam, mu = lognormal(11, E), lognormal(12, E)
    form = F.Form.elasticity(space, cuda(lam), cuda(mu), q1d=p + 2)
    prob = oel.ElasticityProblem(c, h, p, p + 2, lam, mu, Xn=Xn, k=curvedk)
    ndof = space.ndof
    bd = space.boundary_dofs()
    ess = np.concatenate([bd + k * ndof for k in range(3)])
    form.set_essential(ess)
    bvec = x_uniform(13, form.n)
    bc = torch.empty(form.n, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    Ac = osolve.constrain(prob.K, ess)
    bco = osolve.constrain_rhs(prob.K, bvec, ess)
    for precision in ("f64", "f32"):
        x = torch.zeros_like(bc)
        info = F.Multigrid(form, precision=precision).solve(bc, x, rtol=1e-10)
        assert info["converged"], (precision, info)
        u = x.cpu().numpy()
        assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10, precision


def test_deterministic():
    """Fixed-order scatter and reductions: repeated applies and multigrid
    solves give bit-identical results."""
    import torch
    import paper_1911_09220_gb300 as F
    form, prob, (c, h, lam, mu) = _setup(3)
    x = cuda(x_uniform(21, form.n))
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    for arith in (None, "df64"):
        form.apply(x, y1, arith=arith)
        form.apply(x, y2, arith=arith)
        assert torch.equal(y1, y2)
    ndof = form.space.ndof
    bd = form.space.boundary_dofs()
    form.set_essential(np.concatenate([bd + k * ndof for k in range(3)]))
    bc = torch.empty_like(x)
    form.lift_rhs(x, torch.zeros_like(x), bc)
    mg = F.Multigrid(form, precision="f32")
    u1, u2 = torch.zeros_like(x), torch.zeros_like(x)
    i1 = mg.solve(bc, u1, rtol=1e-10)
    i2 = mg.solve(bc, u2, rtol=1e-10)
    assert i1["iterations"] == i2["iterations"] and torch.equal(u1, u2)


def test_sampled_rows_at_bench_size():
    """The elasticity bench configuration (p = 4, q = 6, 28^3 hexes perturbed
    0.15h, 4.3M vector DOFs, the bench's seeds): sampled rows of the FP64,
    double-float and FP32 applies against the oracle's row-by-row apply."""
    import torch
    import paper_1911_09220_gb300 as F
    from fem_inputs import hex_lattice
    from oracle import numbering
    p, N = 4, 28
    c, h = hex_lattice(N, 0.15, seed=60 + p)
    E = h.shape[0]
    lam, mu = lognormal(70 + p, E), lognormal(80 + p, E)
    space = F.Space(F.Mesh(c, h), p)
    form = F.Form.elasticity(space, cuda(lam), cuda(mu), q1d=p + 2)
    num = numbering.build(h, p, nv=c.shape[0])
    assert num["ndof"] == space.ndof
    x = x_uniform(90 + p, form.n)
    rng = np.random.default_rng(7)
    bd = np.asarray(num["boundary_dofs"])
    rows = np.unique(np.concatenate([rng.integers(0, form.n, 30),
                                     rng.choice(bd, 6, replace=False) + space.ndof * rng.integers(0, 3, 6)]))
    ref = oel.sampled_apply(c, h, num["e2l"], p, p + 2, lam, mu, x, rows)
    scale = np.abs(ref).max()
    rt = torch.as_tensor(rows, device="cuda")
    xd = cuda(x)
    y = torch.empty_like(xd)
    form.apply(xd, y)
    assert np.abs(y[rt].cpu().numpy() - ref).max() <= TOL * scale
    form.apply(xd, y, arith="df64")
    assert np.abs(y[rt].cpu().numpy() - ref).max() <= TOL * scale
    y32 = torch.empty(form.n, dtype=torch.float32, device="cuda")
    form.apply(xd.float(), y32)
    assert np.abs(y32[rt].double().cpu().numpy() - ref).max() <= 2e-5 * scale
