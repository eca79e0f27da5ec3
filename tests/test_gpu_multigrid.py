"""Parity of the p-multigrid preconditioner and flexible CG of the CUDA
library (fem_mg_*) with the oracle (oracle.multigrid) on the same seeded
inputs: level orders and sizes, lambda estimates, one V-cycle (FP64 and
FP32 arithmetic; whole-boundary and one-face essential sets; p = 1..8,
shuffled meshes, ragged element counts), the solve (true residual by the
oracle's CSR, iteration count against the oracle's FCG), determinism and
error reporting.

Tolerances: the FP64 V-cycle runs ~4K + 20 operator applications and a
20-step CG whose coefficients are ratios of dot products; rounding-order
differences of ~1e-16 per operation grow to at most ~1e-12 relative in the
max norm on these sizes, so 1e-10 is required. The FP32 V-cycle is
compared at 1e-4 (single precision, amplified by the same ratios)."""

import numpy as np
import pytest

from fem_inputs import lognormal, x_uniform
from oracle import assemble, multigrid as omg, solve as osolve

from gpu_util import cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _setup(p, N=3, drop=0, shuffle=True, face_only=False, seed=5, **kw):
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, perturb=0.15, seed=seed, shuffle=shuffle, drop=drop)
    kap = lognormal(seed + 1, h.shape[0])
    fine = assemble.Problem(c, h, p, p + 2, kappa=kap)
    if face_only:
        X = fine.dof_coords()
        ess = np.nonzero(np.abs(X[:, 0]) < 1e-12)[0]
    else:
        ess = fine.num["boundary_dofs"]
    mesh = F.Mesh(c, h)
    space = F.Space(mesh, p)
    form = F.Form(space, "diffusion", p + 2, coef=cuda(kap))
    form.set_essential(ess)
    okw = {k: v for k, v in kw.items() if k != "precision"}
    M = omg.PMG(c, h, p, p + 2, kap, ess, fine_prob=fine, **okw)
    G = F.Multigrid(form, **kw)
    return M, G, form, fine, ess, (mesh, space)


@pytest.mark.parametrize("p,N,drop", [(2, 4, 3), (3, 3, 1), (4, 3, 2), (5, 2, 1), (8, 2, 0), (1, 4, 5)])
def test_levels_and_lambdas(p, N, drop):
    M, G, *_ = _setup(p, N, drop)
    info = G.info()
    assert info["orders"] == omg.level_orders(p)
    assert info["ndofs"] == [lv.n for lv in M.levels]
    for l, lv in enumerate(M.levels[:-1]):
        assert abs(info["lambdas"][l] - lv.lam) <= 1e-10 * lv.lam


@pytest.mark.parametrize("face_only", [False, True])
@pytest.mark.parametrize("p,N,drop", [(2, 4, 3), (4, 3, 2), (7, 2, 0), (8, 2, 1)])
def test_level_operators_and_transfers(p, N, drop, face_only):
    """Every level's constrained operator and diagonal (coarse essential
    DOFs included) and both transfers against the oracle's matrices."""
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, drop, face_only=face_only)
    for l, lv in enumerate(M.levels):
        f = G.level_form(l)
        x = x_uniform(40 + l, lv.n)
        y = torch.empty(lv.n, dtype=torch.float64, device="cuda")
        f.apply(cuda(x), y, constrained=True)
        assert relerr(y.cpu().numpy(), lv.A @ x) <= 1e-12
        d = torch.empty_like(y)
        f.diagonal(d, constrained=True)
        assert relerr(d.cpu().numpy(), lv.D) <= 1e-12
        if l + 1 < len(M.levels):
            nc = M.levels[l + 1].n
            zc = x_uniform(50 + l, nc)
            zf = torch.empty(lv.n, dtype=torch.float64, device="cuda")
            G.prolong(l, cuda(zc), zf)
            assert relerr(zf.cpu().numpy(), lv.P @ zc) <= 1e-13
            rc = torch.empty(nc, dtype=torch.float64, device="cuda")
            G.restrict(l, cuda(x), rc)
            assert relerr(rc.cpu().numpy(), lv.P.T @ x) <= 1e-13
    with pytest.raises(IndexError):
        G.level_form(len(M.levels))


@pytest.mark.parametrize("face_only", [False, True])
@pytest.mark.parametrize("p,N,drop", [(2, 4, 3), (3, 3, 1), (4, 3, 2), (5, 2, 1), (6, 2, 1), (7, 2, 0), (8, 2, 1),
                                      (1, 4, 5)])
def test_vcycle_parity_fp64(p, N, drop, face_only):
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, drop, face_only=face_only)
    r = x_uniform(10 + p, fine.ndof)
    r[ess] = 0.0
    z = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    G.vcycle(cuda(r), z)
    ref = M.vcycle(r)
    assert relerr(z.cpu().numpy(), ref) <= 1e-10
    # entries of r on essential DOFs are ignored
    r2 = r.copy()
    r2[ess] = 7.0
    z2 = torch.empty_like(z)
    G.vcycle(cuda(r2), z2)
    assert torch.equal(z, z2)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("p,N,drop,face_only", [(2, 4, 3, False), (4, 3, 2, True), (6, 2, 1, False),
                                                (1, 4, 5, False)])
def test_assembled_coarsest_level(p, N, drop, face_only, precision, tol):
    """The order-1 coarsest level as an assembled matrix (the default) gives
    the V-cycle of the matrix-free coarsest level: same operator, other
    summation order."""
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, drop, face_only=face_only, precision=precision)
    import paper_1911_09220_gb300 as F
    G0 = F.Multigrid(form, precision=precision, coarse_assembled=False)
    r = x_uniform(60 + p, fine.ndof)
    r[ess] = 0.0
    z = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    z0 = torch.empty_like(z)
    G.vcycle(cuda(r), z)
    G0.vcycle(cuda(r), z0)
    assert relerr(z.cpu().numpy(), z0.cpu().numpy()) <= tol
    assert relerr(z.cpu().numpy(), M.vcycle(r)) <= (1e-10 if precision == "f64" else 1e-4)


@pytest.mark.parametrize("p,N", [(2, 4), (4, 3), (8, 2)])
def test_vcycle_parity_fp32(p, N):
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, precision="f32")
    r = x_uniform(20 + p, fine.ndof)
    r[ess] = 0.0
    z = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    G.vcycle(cuda(r), z)
    assert relerr(z.cpu().numpy(), M.vcycle(r)) <= 1e-4


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("p,N,face_only", [(2, 5, False), (4, 3, False), (4, 3, True), (8, 2, False), (3, 4, True)])
def test_solve(p, N, face_only, precision):
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, face_only=face_only, precision=precision)
    bvec = x_uniform(30 + p, fine.ndof)
    bc = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    x = torch.zeros_like(bc)
    info = G.solve(bc, x, rtol=1e-10)
    assert info["converged"]
    u = x.cpu().numpy()
    Ac = M.levels[0].A
    bco = osolve.constrain_rhs(fine.K, bvec, ess)
    assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10
    xo, ito, relo = M.fcg(bco, rtol=1e-10)
    if precision == "f64":
        assert abs(info["iterations"] - ito) <= 1, (info, ito)
    else:
        assert info["iterations"] <= ito + 3, (info, ito)
    # far fewer iterations than Jacobi-PCG
    _, ij = osolve.pcg(Ac, bco, rtol=1e-10)
    assert info["iterations"] * 4 < ij["iterations"]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_solve_double_float_outer(precision):
    """arith='df64': the outer operator in double-float; same stopping rule
    on the FP64 true residual, iteration count within one of FP64."""
    import torch
    M, G, form, fine, ess, keep = _setup(4, 3, precision=precision)
    bvec = x_uniform(31, fine.ndof)
    bc = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    x64, xdf = torch.zeros_like(bc), torch.zeros_like(bc)
    i64 = G.solve(bc, x64, rtol=1e-10)
    idf = G.solve(bc, xdf, rtol=1e-10, arith="df64")
    assert idf["converged"] and abs(idf["iterations"] - i64["iterations"]) <= 1
    bco = osolve.constrain_rhs(fine.K, bvec, ess)
    u = xdf.cpu().numpy()
    assert np.linalg.norm(bco - M.levels[0].A @ u) / np.linalg.norm(bco) <= 1.01e-10
    with pytest.raises(ValueError):
        G.solve(bc, xdf, arith="mixed")


def test_solve_deterministic_and_graph_free_path():
    import torch
    M, G, form, fine, ess, keep = _setup(4, 3)
    b = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(x_uniform(3, fine.ndof)), torch.zeros_like(b), b)
    xs = []
    for graph in (True, True, False):
        x = torch.zeros_like(b)
        info = G.solve(b, x, use_graph=graph, check_every=3)
        xs.append((x, info["iterations"]))
    assert torch.equal(xs[0][0], xs[1][0]) and xs[0][1] == xs[1][1]
    assert torch.equal(xs[0][0], xs[2][0]) and xs[0][1] == xs[2][1]


def test_errors():
    import paper_1911_09220_gb300 as F
    from fem_inputs import quad_lattice
    c, h = make_mesh(2)
    form = F.Form(F.Space(F.Mesh(c, h), 2), "diffusion", 4)
    with pytest.raises(F.FemError) as ei:
        F.Multigrid(form)                      # no essential list yet
    assert ei.value.status == 1
    form.set_essential(np.array([], dtype=np.int32))
    with pytest.raises(F.FemError) as ei:
        F.Multigrid(form, cheb_lo=1.5)
    assert ei.value.status == 1
    c2, q2 = quad_lattice(3)
    f2 = F.Form(F.Space(F.Mesh2D(c2, q2), 2), "diffusion", 4)
    f2.set_essential(np.array([0], dtype=np.int32))
    with pytest.raises(F.FemError) as ei:
        F.Multigrid(f2)
    assert ei.value.status == 7


# ---- vector hierarchy of an elasticity form
def _esetup(p, N=3, drop=0, ess_kind="clamped", seed=15, **kw):
    import paper_1911_09220_gb300 as F
    from oracle import elasticity as oel
    c, h = make_mesh(N, perturb=0.15, seed=seed, shuffle=True, drop=drop)
    E = h.shape[0]
    lam, mu = lognormal(seed + 1, E), lognormal(seed + 2, E)
    fine = oel.ElasticityProblem(c, h, p, p + 2, lam, mu)
    n = fine.ndof
    bd = assemble.Problem(c, h, p, p + 2).num["boundary_dofs"]
    if ess_kind == "clamped":
        ess = np.concatenate([bd + k * n for k in range(3)])
    else:  # one face clamped in all components, the normal component elsewhere on the boundary
        X = assemble.Problem(c, h, p, p + 2).dof_coords()
        face = np.nonzero(np.abs(X[:, 0]) < 1e-12)[0]
        ess = np.unique(np.concatenate([face, face + n, face + 2 * n, bd]))
    space = F.Space(F.Mesh(c, h), p)
    form = F.Form.elasticity(space, cuda(lam), cuda(mu), q1d=p + 2)
    form.set_essential(ess)
    okw = {k: v for k, v in kw.items() if k != "precision"}
    M = omg.PMG(c, h, p, p + 2, None, ess, fine_prob=fine, lame=(lam, mu), **okw)
    G = F.Multigrid(form, **kw)
    return M, G, form, fine, ess


@pytest.mark.parametrize("ess_kind", ["clamped", "mixed"])
@pytest.mark.parametrize("p,N,drop", [(2, 3, 2), (4, 2, 1), (5, 2, 0)])
def test_elasticity_levels_transfers_vcycle(p, N, drop, ess_kind):
    import torch
    M, G, form, fine, ess = _esetup(p, N, drop, ess_kind=ess_kind)
    info = G.info()
    assert info["orders"] == omg.level_orders(p)
    assert info["ndofs"] == [lv.n for lv in M.levels]
    for l, lv in enumerate(M.levels[:-1]):
        assert abs(info["lambdas"][l] - lv.lam) <= 1e-10 * lv.lam
    for l, lv in enumerate(M.levels):
        f = G.level_form(l)
        x = x_uniform(60 + l, lv.n)
        y = torch.empty(lv.n, dtype=torch.float64, device="cuda")
        f.apply(cuda(x), y, constrained=True)
        assert relerr(y.cpu().numpy(), lv.A @ x) <= 1e-12
        d = torch.empty_like(y)
        f.diagonal(d, constrained=True)
        assert relerr(d.cpu().numpy(), lv.D) <= 1e-12
        if l + 1 < len(M.levels):
            nc = M.levels[l + 1].n
            zc = x_uniform(70 + l, nc)
            zf = torch.empty(lv.n, dtype=torch.float64, device="cuda")
            G.prolong(l, cuda(zc), zf)
            assert relerr(zf.cpu().numpy(), lv.P @ zc) <= 1e-13
            rc = torch.empty(nc, dtype=torch.float64, device="cuda")
            G.restrict(l, cuda(x), rc)
            assert relerr(rc.cpu().numpy(), lv.P.T @ x) <= 1e-13
    r = x_uniform(80 + p, fine.K.shape[0])
    r[ess] = 0.0
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    G.vcycle(cuda(r), z)
    assert relerr(z.cpu().numpy(), M.vcycle(r)) <= 1e-10


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("p,N", [(2, 3), (4, 2)])
def test_elasticity_solve(p, N, precision):
    import torch
    M, G, form, fine, ess = _esetup(p, N, precision=precision)
    n = fine.K.shape[0]
    if precision == "f32":
        r = x_uniform(90 + p, n)
        r[ess] = 0.0
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        G.vcycle(cuda(r), z)
        assert relerr(z.cpu().numpy(), M.vcycle(r)) <= 1e-4
    bvec = x_uniform(95 + p, n)
    bc = torch.empty(n, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    x = torch.zeros_like(bc)
    info = G.solve(bc, x, rtol=1e-10)
    assert info["converged"]
    Ac = M.levels[0].A
    bco = osolve.constrain_rhs(fine.K, bvec, ess)
    u = x.cpu().numpy()
    assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10
    xo, ito, relo = M.fcg(bco, rtol=1e-10)
    assert abs(info["iterations"] - ito) <= 1
    _, pinfo = osolve.pcg(Ac, bco, rtol=1e-10)
    assert 3 * info["iterations"] < pinfo["iterations"]


def test_solve_with_dirichlet_values_from_zero_guess():
    """Non-zero essential values g: b_c = lift(b, g) has b_ess = g; starting
    from x = 0 the solve takes x_ess = g and converges on the free DOFs."""
    import torch
    M, G, form, fine, ess, keep = _setup(3, 3)
    n = fine.ndof
    g = np.zeros(n)
    g[ess] = x_uniform(41, len(ess))
    bvec = x_uniform(42, n)
    bc = torch.empty(n, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), cuda(g), bc)
    x = torch.zeros_like(bc)
    info = G.solve(bc, x, rtol=1e-10)
    assert info["converged"]
    u = x.cpu().numpy()
    assert np.array_equal(u[ess], g[ess])
    Ac = M.levels[0].A
    bco = osolve.constrain_rhs(fine.K, bvec, ess, g[ess])
    assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10


@pytest.mark.parametrize("p,N,face_only", [(2, 4, False), (4, 3, True), (8, 2, False)])
def test_solve_fp32_outer_operator(p, N, face_only):
    """Flexible CG with the FP32 outer operator inside FP64 iterative
    refinement (arith="f32") reaches the same 1e-10 true residual (oracle
    CSR) and the FP64-outer solution."""
    import torch
    M, G, form, fine, ess, keep = _setup(p, N, face_only=face_only, precision="f32")
    bvec = x_uniform(60 + p, fine.ndof)
    bc = torch.empty(fine.ndof, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    x64 = torch.zeros_like(bc)
    G.solve(bc, x64, rtol=1e-10)
    for inner in (1e-2, 1e-4):
        x = torch.zeros_like(bc)
        info = G.solve(bc, x, rtol=1e-10, arith="f32", inner_rtol=inner)
        assert info["converged"] and info["outer"] >= 2
        u = x.cpu().numpy()
        Ac = M.levels[0].A
        bco = osolve.constrain_rhs(fine.K, bvec, ess)
        assert np.linalg.norm(bco - Ac @ u) / np.linalg.norm(bco) <= 1.01e-10
        assert relerr(u, x64.cpu().numpy()) <= 1e-7
    import paper_1911_09220_gb300 as F
    with pytest.raises(F.FemError):
        G.solve(bc, x, rtol=1e-10, arith="f32", inner_rtol=1.5)


def test_elasticity_solve_fp32_outer_operator():
    import torch
    M, G, form, fine, ess = _esetup(4, 2, precision="f32")
    n = fine.K.shape[0]
    bvec = x_uniform(99, n)
    bc = torch.empty(n, dtype=torch.float64, device="cuda")
    form.lift_rhs(cuda(bvec), torch.zeros_like(bc), bc)
    x = torch.zeros_like(bc)
    info = G.solve(bc, x, rtol=1e-10, arith="f32")
    assert info["converged"]
    Ac = M.levels[0].A
    bco = osolve.constrain_rhs(fine.K, bvec, ess)
    assert np.linalg.norm(bco - Ac @ x.cpu().numpy()) / np.linalg.norm(bco) <= 1.01e-10
