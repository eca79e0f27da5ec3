"""fem_apply_noalloc: the FP64 apply whose E-vector scratch is a fixed device
array inside the library, for callers that cannot have the library allocate
device memory during the call (a pool that already holds nearly all GPU
memory, or a loop where cudaMalloc's synchronisation and failure modes are
not acceptable). Its output must match fem_apply's on two calls in a row
(the second call reuses the array the first one filled), and sizes beyond
the fixed scratch must be refused with FEM_EINVAL.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""

import ctypes as C

import numpy as np
import pytest

from fem_inputs import x_uniform

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


def _noalloc(form, x, y):
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    st = F.lib().fem_apply_noalloc(form._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, F.lib().fem_last_error().decode()


@pytest.mark.parametrize("p,N,kind", [(2, 4, "diffusion"), (4, 3, "mass"), (7, 2, "diffusion")])
def test_noalloc_matches_apply_twice(p, N, kind):
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    c, h = make_mesh(N, seed=200 + p, shuffle=True, drop=1)
    mesh = F.Mesh(c, h)
    space = F.Space(mesh, p)
    form = F.Form(space, kind, p + 2, coef=cuda(np.linspace(0.5, 2.0, h.shape[0])))
    for call in range(2):
        x = cuda(x_uniform(201 + call, space.ndof))
        ref = torch.empty_like(x)
        form.apply(x, ref)
        y = torch.full_like(x, np.nan)
        st, msg = _noalloc(form, x, y)
        assert st == B.FEM_OK, msg
        torch.cuda.synchronize()
        assert relerr(y.cpu().numpy(), ref.cpu().numpy()) <= TOL, call


def test_noalloc_refuses_oversize():
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    # 28^3 elements at p = 4: 21,952 * 125 = 2,744,000 entries fits; 33^3 * 125 = 4,492,125 does not
    c, h = make_mesh(33, perturb=0.0, seed=1)
    form = F.Form(F.Space(F.Mesh(c, h), 4), "mass", 6)
    x = torch.zeros(form.space.ndof, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st, msg = _noalloc(form, x, y)
    assert st == B.FEM_EINVAL and "exceeds the fixed scratch" in msg
