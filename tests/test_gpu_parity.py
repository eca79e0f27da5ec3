"""Parity of the CUDA library (through its C ABI) with the CPU FP64 oracle on
the same seeded inputs: numbering, D setup through the operator, apply
(mass and diffusion, p = 1..8, ragged element counts, shuffled and rotated
meshes), brute-force dense operators, diagonal, quadrature points, load
vector, constrained operator and error paths.

Tolerance for FP64 results: max-norm relative error <= 1e-12 (the bar the
partial-assembly path must meet against the assembled oracle). FP32 applies
are compared at 2e-5 relative (single-precision rounding of sums of a few
hundred terms)."""

import numpy as np
import pytest

from fem_inputs import hex_lattice, x_uniform, uniform
from oracle import assemble, solve as osolve

from gpu_util import Case, cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12

# (p, N, dropped elements): element counts that leave a ragged last block
SIZES = {1: (5, 3), 2: (4, 5), 3: (3, 2), 4: (3, 1), 5: (3, 2), 6: (2, 1), 7: (2, 1), 8: (2, 1)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


@pytest.mark.parametrize("p,shuffle", [(1, False), (2, True), (3, True), (4, False), (5, True)])
def test_numbering_boundary_and_dof_coords(p, shuffle):
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=11, shuffle=shuffle, drop=drop)
    cs = Case(c, h, p)
    assert cs.space.ndof == cs.prob.ndof
    np.testing.assert_array_equal(cs.space.element_dofs(), cs.prob.e2l)
    np.testing.assert_array_equal(cs.space.boundary_dofs(), cs.prob.num["boundary_dofs"])
    X = cs.space.dof_coords().cpu().numpy()
    np.testing.assert_allclose(X, cs.prob.dof_coords(), atol=1e-14)


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", range(1, 9))
def test_apply_parity_fp64(kind, p):
    import torch
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=10 + p, shuffle=(p % 2 == 0), drop=drop)
    cs = Case(c, h, p, kind=kind, coef_seed=20 + p)
    x = x_uniform(30 + p, cs.n)
    y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.apply(cuda(x), y)
    ref = cs.prob.apply(kind, x)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    # the two halves through the ABI give the same bits
    ye = torch.empty((cs.space.ne, (p + 1) ** 3), dtype=torch.float64, device="cuda")
    y2 = torch.empty_like(y)
    cs.form.apply_element(cuda(x), ye)
    cs.form.scatter(ye, y2)
    assert torch.equal(y, y2)


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", range(1, 9))
def test_apply_parity_df64(kind, p):
    """Double-float element arithmetic: same 1e-12 bar as native FP64."""
    import torch
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=110 + p, shuffle=(p % 2 == 1), drop=drop)
    cs = Case(c, h, p, kind=kind, coef_seed=120 + p)
    x = x_uniform(130 + p, cs.n)
    y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.apply(cuda(x), y, arith="df64")
    ref = cs.prob.apply(kind, x)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    # and against the native FP64 path
    y64 = torch.empty_like(y)
    cs.form.apply(cuda(x), y64)
    assert relerr(y.cpu().numpy(), y64.cpu().numpy()) <= TOL
    # the two public halves: a float64 E-vector, then the FP64 scatter
    ye = torch.empty(cs.space.ne * (p + 1) ** 3, dtype=torch.float64, device="cuda")
    cs.form.apply_element(cuda(x), ye, arith="df64")
    y2 = torch.empty_like(y)
    cs.form.scatter(ye, y2)
    assert relerr(y2.cpu().numpy(), ref) <= TOL


def test_df64_constrained_and_small_magnitudes():
    import torch
    c, h = make_mesh(3, seed=140, shuffle=True)
    cs = Case(c, h, 4)
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    for scale in (1.0, 1e-20, 1e20):
        x = x_uniform(141, cs.n) * scale
        y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
        cs.form.apply(cuda(x), y, constrained=True, arith="df64")
        ref = osolve.constrain(cs.prob.K, ess) @ x
        assert relerr(y.cpu().numpy(), ref) <= TOL, scale


@pytest.mark.parametrize("q_off", [1, 2])
@pytest.mark.parametrize("p", [2, 5])
def test_apply_both_quadrature_sizes(p, q_off):
    import torch
    c, h = make_mesh(3, seed=5, shuffle=True)
    cs = Case(c, h, p, q=p + q_off)
    x = x_uniform(7, cs.n)
    y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), cs.prob.apply("diffusion", x)) <= TOL


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", [1, 3, 4, 6, 8])
def test_apply_parity_fp32(kind, p):
    import torch
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=40 + p, drop=drop)
    cs = Case(c, h, p, kind=kind)
    x = x_uniform(41 + p, cs.n)
    y = torch.empty(cs.n, dtype=torch.float32, device="cuda")
    cs.form.apply(cuda(x, torch.float32), y)
    ref = cs.prob.apply(kind, x.astype(np.float32).astype(np.float64))
    assert relerr(y.cpu().double().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("p,N", [(1, 1), (2, 1), (3, 2), (4, 1), (8, 1)])
def test_brute_force_dense_operator(p, N):
    """Apply to every unit vector: the dense operator equals the oracle's
    assembled matrix on 1-8 element meshes (shuffled, rotated elements)."""
    import torch
    c, h = make_mesh(N, seed=60 + p, shuffle=True)
    for kind in ("diffusion", "mass"):
        cs = Case(c, h, p, kind=kind, coef_seed=61)
        n = cs.n
        A = np.zeros((n, n))
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(e)
        for j in range(n):
            e.zero_()
            e[j] = 1.0
            cs.form.apply(e, y)
            A[:, j] = y.cpu().numpy()
        R = cs.prob.matrix(kind).toarray()
        assert np.abs(A - R).max() <= TOL * np.abs(R).max()


def test_brute_force_two_elements_every_shared_face_orientation():
    """Two hexahedra sharing a face, the second one re-oriented by each of
    the 24 proper rotations: the assembled operators agree with the oracle."""
    import torch
    from fem_inputs import CUBE_ROTATIONS
    c, h = hex_lattice(2, 0.1, seed=3)
    h2 = h[:2].astype(np.int64)                        # elements (0,0,0) and (1,0,0) share a face
    for r in range(24):
        hh = h2.copy()
        hh[1] = hh[1][CUBE_ROTATIONS[r]]
        from fem_inputs import submesh
        cc, hx = submesh(c, hh, [0, 1])
        cs = Case(cc, hx, 3, kind="diffusion", coef_seed=None)
        n = cs.n
        A = np.zeros((n, n))
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(e)
        for j in range(n):
            e.zero_()
            e[j] = 1.0
            cs.form.apply(e, y)
            A[:, j] = y.cpu().numpy()
        R = cs.prob.K.toarray()
        assert np.abs(A - R).max() <= TOL * np.abs(R).max(), r


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_diagonal_parity(kind, p):
    import torch
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=70 + p, shuffle=True, drop=drop)
    cs = Case(c, h, p, kind=kind)
    d = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.diagonal(d)
    assert relerr(d.cpu().numpy(), cs.prob.diagonal(kind)) <= TOL
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    cs.form.diagonal(d, constrained=True)
    ref = cs.prob.diagonal(kind).copy()
    ref[ess] = 1.0
    assert relerr(d.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("p", [1, 2, 3, 6])
def test_qpoints_and_rhs(p):
    import torch
    N, drop = SIZES[p]
    c, h = make_mesh(N, seed=80 + p, shuffle=True, drop=drop)
    cs = Case(c, h, p)
    xq = cs.form.qpoint_coords().cpu().numpy()
    np.testing.assert_allclose(xq, cs.prob.qpoint_coords(), atol=2e-16 * 8)
    # seeded source values at the quadrature points: identical input on both sides
    fq = uniform(81, cs.space.ne * cs.form.nq, -1.0, 1.0).reshape(cs.space.ne, cs.form.nq)
    b = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.rhs(cuda(fq), b)
    assert relerr(b.cpu().numpy(), cs.prob.load_from_qvalues(fq)) <= TOL


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_constrained_apply_and_lift(dtype):
    import torch
    c, h = make_mesh(3, seed=90, shuffle=True)
    cs = Case(c, h, 3)
    ess = cs.prob.num["boundary_dofs"]
    cs.form.set_essential(ess)
    x = x_uniform(91, cs.n)
    Ac = osolve.constrain(cs.prob.K, ess)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = torch.empty(cs.n, dtype=tdt, device="cuda")
    cs.form.apply(cuda(x, tdt), y, constrained=True)
    xin = x if dtype == "f64" else x.astype(np.float32).astype(np.float64)
    assert relerr(y.cpu().double().numpy(), Ac @ xin) <= (TOL if dtype == "f64" else 2e-5)
    # lifting b_c = (I-E)(b - A g) + E g
    b = x_uniform(92, cs.n)
    g = x_uniform(93, cs.n)
    bc = torch.empty(cs.n, dtype=torch.float64, device="cuda")
    cs.form.lift_rhs(cuda(b), cuda(g), bc)
    ref = osolve.constrain_rhs(cs.prob.K, b, ess, g[ess])
    assert relerr(bc.cpu().numpy(), ref) <= TOL


def test_single_element_every_order():
    import torch
    c, h = hex_lattice(1, 0.0)
    c = c * np.array([1.0, 2.0, 0.5]) + np.array([0.1, -0.3, 0.2])
    for p in range(1, 9):
        cs = Case(c, h, p, coef_seed=None)
        x = x_uniform(100 + p, cs.n)
        y = torch.empty(cs.n, dtype=torch.float64, device="cuda")
        cs.form.apply(cuda(x), y)
        assert relerr(y.cpu().numpy(), cs.prob.apply("diffusion", x)) <= TOL


def test_zero_input_and_errors():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(2, seed=1)
    cs = Case(c, h, 2, oracle=False)
    x = torch.zeros(cs.n, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 7.0)
    cs.form.apply(x, y)
    assert torch.count_nonzero(y).item() == 0
    with pytest.raises(F.FemError):
        cs.form.apply(x, x)                                 # aliasing
    with pytest.raises(F.FemError):
        F.Space(cs.mesh, 9)                                 # not compiled
    with pytest.raises(F.FemError):
        F.Form(cs.space, "diffusion", q1d=9)                # (2, 9) not compiled
    bad = h.copy()
    bad[0] = bad[0][[4, 5, 6, 7, 0, 1, 2, 3]]               # mirrored: det J < 0
    m = F.Mesh(c, bad)
    sp = F.Space(m, 2)
    with pytest.raises(F.FemError) as ei:
        F.Form(sp, "diffusion", 4)
    assert "FEM_EINVERTED" in str(ei.value)
    bad2 = h.copy()
    bad2[1, 0] = bad2[1, 1]
    with pytest.raises(F.FemError):
        F.Mesh(c, bad2)                                     # repeated vertex
    with pytest.raises(F.FemError):
        cs.form.set_essential(np.array([cs.n + 5], dtype=np.int32))   # out of range
