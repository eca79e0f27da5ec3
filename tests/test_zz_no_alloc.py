"""fem_apply_noalloc: the FP64 apply whose E-vector scratch is a fixed device
array inside the library, for callers that cannot have the library allocate
device memory during the call (a pool that already holds nearly all GPU
memory, or a loop where cudaMalloc's synchronisation and failure modes are
not acceptable). Its output must match fem_apply's on two calls in a row
(the second call reuses the array the first one filled) and the oracle's
assembled operator, for scalar 3D, elasticity (three components in the one
array) and 2D forms; a problem whose E-vector fills the array exactly must
be accepted, and sizes beyond it refused with FEM_EINVAL, the vector
dimension counted.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""

import ctypes as C

import numpy as np
import pytest

from fem_inputs import lognormal, quad_lattice, x_uniform
from oracle import assemble, elasticity as oel, twod

from gpu_util import cuda, make_mesh, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12
LIMIT = 1 << 22  # entries of the fixed E-vector array


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


def _twice(form, n, seed, oracle_apply=None):
    """Two no-allocation applies in a row, each against fem_apply (and the
    oracle's operator when given)."""
    import torch
    from paper_1911_09220_gb300 import _binding as B
    for call in range(2):
        xh = x_uniform(seed + call, n)
        x = cuda(xh)
        ref = torch.empty_like(x)
        form.apply(x, ref)
        y = torch.full_like(x, np.nan)
        st, msg = _noalloc(form, x, y)
        assert st == B.FEM_OK, msg
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        assert relerr(yh, ref.cpu().numpy()) <= TOL, call
        if oracle_apply is not None:
            assert relerr(yh, oracle_apply(xh)) <= TOL, call


@pytest.mark.parametrize("p,N,kind", [(2, 4, "diffusion"), (4, 3, "mass"), (7, 2, "diffusion")])
def test_noalloc_matches_apply_twice(p, N, kind):
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(N, seed=200 + p, shuffle=True, drop=1)
    coef = np.linspace(0.5, 2.0, h.shape[0])
    form = F.Form(F.Space(F.Mesh(c, h), p), kind, p + 2, coef=cuda(coef))
    prob = assemble.Problem(c, h, p, p + 2, kappa=coef, rho=coef)
    _twice(form, form.space.ndof, 201, lambda x: prob.apply(kind, x))


def test_noalloc_elasticity_twice():
    import paper_1911_09220_gb300 as F
    p = 3
    c, h = make_mesh(3, seed=230, shuffle=True, drop=2)
    E = h.shape[0]
    lam, mu = lognormal(231, E), lognormal(232, E)
    form = F.Form.elasticity(F.Space(F.Mesh(c, h), p), cuda(lam), cuda(mu), q1d=p + 2)
    prob = oel.ElasticityProblem(c, h, p, p + 2, lam, mu)
    _twice(form, form.n, 233, prob.apply)


@pytest.mark.parametrize("p,kind", [(3, "diffusion"), (5, "mass")])
def test_noalloc_2d_twice(p, kind):
    import paper_1911_09220_gb300 as F
    c, qd = quad_lattice(5, 0.2, seed=240 + p, shuffle=True)
    coef = lognormal(241 + p, qd.shape[0])
    form = F.Form(F.Space(F.Mesh2D(c, qd), p), kind, p + 2, coef=cuda(coef))
    prob = twod.Problem2(c, qd, p, p + 2, kappa=coef, rho=coef)
    _twice(form, form.space.ndof, 242, lambda x: prob.apply(kind, x))


def test_noalloc_limit_is_exact():
    """512^2 quadrilaterals at p = 3 fill the array exactly (262,144 x 16 =
    4,194,304 entries) and are accepted; 513^2 are refused."""
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    for N, ok in ((512, True), (513, False)):
        c, qd = quad_lattice(N, 0.0, seed=1)
        form = F.Form(F.Space(F.Mesh2D(c, qd), 3), "mass", 5)
        assert (N * N * 16 <= LIMIT) == ok
        n = form.space.ndof
        if ok:
            _twice(form, n, 250)
        else:
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            st, msg = _noalloc(form, x, y)
            assert st == B.FEM_EINVAL and "exceeds the fixed scratch" in msg


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


def test_noalloc_counts_vector_components():
    """64^3 elements at p = 1: 2,097,152 entries for a scalar form (accepted),
    three times that for elasticity (refused)."""
    import torch
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import _binding as B
    c, h = make_mesh(64, perturb=0.0, seed=2)
    space = F.Space(F.Mesh(c, h), 1)
    E = h.shape[0]
    scalar = F.Form(space, "diffusion", 3)
    x = torch.zeros(space.ndof, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st, msg = _noalloc(scalar, x, y)
    assert st == B.FEM_OK, msg
    el = F.Form.elasticity(space, cuda(np.ones(E)), cuda(np.ones(E)), q1d=3)
    x3 = torch.zeros(el.n, dtype=torch.float64, device="cuda")
    y3 = torch.empty_like(x3)
    st, msg = _noalloc(el, x3, y3)
    assert st == B.FEM_EINVAL and "exceeds the fixed scratch" in msg
