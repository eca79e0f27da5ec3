"""The DOF-sorted E-vector of fem_apply (and the solvers and multigrid
levels built on it): where a form's E-vector exceeds half the L2, the
element kernel writes each value at its slot's position in the inverse map
and the scatter reads every DOF's values contiguously. The sums and their
order are those of the element-major path, so fem_apply must equal the
public halves (fem_apply_element into an element-major E-vector, then
fem_scatter) bit for bit, for scalar and vector (elasticity) forms, every
arithmetic, constrained or not. The sizes are chosen so that the sorted
order is taken."""

import numpy as np
import pytest

from fem_inputs import lognormal, x_uniform

from gpu_util import cuda, make_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _halves(form, x, arith=None):
    import torch
    ye = torch.empty(form.vdim * form.space.ne * (form.space.p + 1) ** 3, dtype=x.dtype, device="cuda")
    form.apply_element(x, ye, arith=arith)
    y = torch.empty_like(x)
    form.scatter(ye, y)
    return y


# E-vector bytes: 8 B (FP64, double-float) or 4 B (FP32) x vdim x ne x 125 > 64 MB
@pytest.mark.parametrize("kind,N,arith", [("diffusion", 42, "f64"), ("diffusion", 42, "df64"),
                                          ("diffusion", 56, "f32"), ("mass", 42, "f64")])
def test_scalar_sorted_apply_equals_halves(kind, N, arith):
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, seed=300 + N, shuffle=True)
    form = F.Form(F.Space(F.Mesh(c, h), 4), kind, 6, coef=cuda(lognormal(301, h.shape[0])))
    dt = torch.float32 if arith == "f32" else torch.float64
    ar = "df64" if arith == "df64" else None  # the vector dtype selects FP32 / FP64
    x = cuda(x_uniform(302, form.space.ndof), dt)
    y = torch.empty_like(x)
    form.apply(x, y, arith=ar)
    ref = _halves(form, x, arith=ar)
    assert torch.equal(y, ref)
    # constrained: zeroed essential inputs, identity rows
    ess = form.space.boundary_dofs()
    form.set_essential(cuda(ess))
    form.apply(x, y, constrained=True, arith=ar)
    xz = x.clone()
    xz[torch.as_tensor(ess, device="cuda", dtype=torch.int64)] = 0
    ref = _halves(form, xz, arith=ar)
    ref[torch.as_tensor(ess, device="cuda", dtype=torch.int64)] = x[torch.as_tensor(ess, device="cuda",
                                                                                    dtype=torch.int64)]
    assert torch.equal(y, ref)


@pytest.mark.parametrize("N,arith", [(29, "f64"), (36, "f32")])
def test_elasticity_sorted_apply_equals_halves(N, arith):
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, seed=310 + N, shuffle=True)
    E = h.shape[0]
    form = F.Form.elasticity(F.Space(F.Mesh(c, h), 4), cuda(lognormal(311, E)), cuda(lognormal(312, E)), q1d=6)
    dt = torch.float32 if arith == "f32" else torch.float64
    x = cuda(x_uniform(313, form.n), dt)
    y = torch.empty_like(x)
    form.apply(x, y)
    assert torch.equal(y, _halves(form, x))
