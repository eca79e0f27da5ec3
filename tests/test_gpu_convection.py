"""Parity of the convection form (fem_form_create_convection) of the CUDA
library with the convection oracle on the same seeded inputs: apply (FP64,
double-float, FP32; p = 1..8; shuffled and ragged meshes; trilinear and
curved geometry; a variable velocity evaluated at the library's own
quadrature points); set_velocity and set_coef; the entry points that need a
symmetric form reject it. Tolerances as for diffusion (1e-12; FP32 2e-5)."""

import numpy as np
import pytest

from fem_inputs import curved_nodes, lognormal, x_uniform
from oracle import convection as oconv

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


def _velocity(xq):
    import torch
    return torch.stack([1.0 + xq[..., 1], torch.sin(2.0 * xq[..., 2]), xq[..., 0] * xq[..., 1] - 0.5], -1)


SIZES = {1: (5, 3), 2: (4, 5), 3: (3, 2), 4: (3, 1), 5: (3, 2), 6: (2, 1), 7: (2, 1), 8: (2, 1)}


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("curvedk", [0, 2])
def test_apply_parity(p, curvedk):
    import torch
    import paper_1911_09220_gb300 as F
    N, drop = SIZES[p]
    c, h = make_mesh(N, perturb=0.15, seed=20 + p, shuffle=(p % 2 == 1), drop=drop)
    mesh = F.Mesh(c, h)
    Xn = None
    if curvedk:
        Xn = curved_nodes(c, h, curvedk)
        mesh.set_nodes(Xn, curvedk)
    space = F.Space(mesh, p)
    q = p + 2
    coef = lognormal(30 + p, h.shape[0])
    # the velocity at the library's quadrature points
    probe = F.Form(space, "mass", q)
    beta = _velocity(probe.qpoint_coords()).contiguous()
    form = F.Form.convection(space, beta, q1d=q, coef=cuda(coef))
    bref = beta.cpu().numpy() * coef[:, None, None]
    prob = oconv.ConvectionProblem(c, h, p, q, bref, Xn=Xn, k=curvedk)
    x = x_uniform(40 + p, space.ndof)
    ref = prob.apply(x)
    y = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.apply(cuda(x), y)
    assert relerr(y.cpu().numpy(), ref) <= TOL
    form.apply(cuda(x), y, arith="df64")
    assert relerr(y.cpu().numpy(), ref) <= TOL
    y32 = torch.empty(space.ndof, dtype=torch.float32, device="cuda")
    form.apply(cuda(x, torch.float32), y32)
    assert relerr(y32.cpu().numpy().astype(np.float64), ref) <= 2e-5


def test_set_velocity_coef_and_rejections():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(3, perturb=0.1, seed=2)
    space = F.Space(F.Mesh(c, h), 3)
    xq = F.Form(space, "mass", 5).qpoint_coords()
    b1 = _velocity(xq).contiguous()
    b2 = torch.ones_like(b1)
    form = F.Form.convection(space, b1, q1d=5)
    x = cuda(x_uniform(1, space.ndof))
    y = torch.empty_like(x)
    form.set_velocity(b2)
    form.apply(x, y)
    ref = oconv.ConvectionProblem(c, h, 3, 5, b2.cpu().numpy()).apply(x.cpu().numpy())
    assert relerr(y.cpu().numpy(), ref) <= TOL
    kap = lognormal(3, h.shape[0])
    form.set_coef(cuda(kap))
    form.apply(x, y)
    ref = oconv.ConvectionProblem(c, h, 3, 5, b2.cpu().numpy() * kap[:, None, None]).apply(x.cpu().numpy())
    assert relerr(y.cpu().numpy(), ref) <= TOL
    # symmetric-only entry points
    form.set_essential(space.boundary_dofs())
    with pytest.raises(F.FemError) as ei:
        form.diagonal(torch.empty_like(x))
    assert ei.value.status == 7
    with pytest.raises(F.FemError) as ei:
        form.solve(x, torch.zeros_like(x))
    assert ei.value.status == 1
    with pytest.raises(F.FemError):
        F.Multigrid(form)
    with pytest.raises(F.FemError):
        F.Batch([form], 1)
    import ctypes
    h_out = ctypes.c_void_p()
    assert F.lib().fem_form_create(space._h, 2, 5, None, None, ctypes.byref(h_out)) == 1  # needs a velocity
    with pytest.raises(ValueError):
        F.Form.convection(space, b1[:, :3])
