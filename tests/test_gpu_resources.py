"""Resource and failure behaviour on the GPU: every form kind reports an
inverted element at setup (FEM_EINVERTED) and leaves nothing behind; forms,
multigrid hierarchies and batches of every kind release their device memory
when destroyed (repeated create / destroy returns the device to the same
free memory)."""

import gc

import numpy as np
import pytest

from fem_inputs import lognormal

from gpu_util import cuda, make_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def test_inverted_element_every_kind():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(2, perturb=0.1, seed=3)
    bad = h.copy()
    bad[1] = bad[1][[4, 5, 6, 7, 0, 1, 2, 3]]        # mirrored: det J < 0
    space = F.Space(F.Mesh(c, bad), 2)
    E = h.shape[0]
    one = cuda(np.ones(E))
    makers = [lambda: F.Form(space, "diffusion", 4), lambda: F.Form(space, "mass", 4),
              lambda: F.Form.elasticity(space, one, one, q1d=4)]
    probe = F.Form(F.Space(F.Mesh(c, h), 2), "mass", 4)
    beta = torch.ones((E, 64, 3), dtype=torch.float64, device="cuda")
    makers.append(lambda: F.Form.convection(space, beta, q1d=4))
    del probe
    for make in makers:
        with pytest.raises(F.FemError) as ei:
            make()
        assert ei.value.status == 3 and "FEM_EINVERTED" in str(ei.value)


def _free():
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_create_destroy_releases_device_memory():
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(6, perturb=0.1, seed=5)
    E = h.shape[0]
    kap = cuda(lognormal(6, E))
    mesh = F.Mesh(c, h)

    def cycle():
        space = F.Space(mesh, 3)
        forms = [F.Form(space, "diffusion", 5, coef=kap), F.Form(space, "mass", 5, coef=kap),
                 F.Form.elasticity(space, kap, kap, q1d=5)]
        x = torch.ones(space.ndof, dtype=torch.float64, device="cuda")
        for f in forms[:2]:
            f.apply(x, torch.empty_like(x))
            f.apply(x.float(), torch.empty_like(x.float()))      # FP32 copy of D
            f.apply(x, torch.empty_like(x), arith="df64")        # double-float copy of D
        xv = torch.ones(forms[2].n, dtype=torch.float64, device="cuda")
        forms[2].apply(xv, torch.empty_like(xv))
        for f in (forms[0], forms[2]):
            n = f.n
            ess = space.boundary_dofs() if f.vdim == 1 else np.concatenate(
                [space.boundary_dofs() + k * space.ndof for k in range(3)])
            f.set_essential(ess)
            b = torch.ones(n, dtype=torch.float64, device="cuda")
            u = torch.zeros_like(b)
            f.solve(b, u, rtol=1e-6, precision="mixed")
            mg = F.Multigrid(f, precision="f32")
            mg.solve(b, torch.zeros_like(b), rtol=1e-6)
            del mg
        batch = F.Batch([forms[0], forms[1]], 2)
        del batch, forms, space, x, xv

    cycle()
    base = _free()
    for _ in range(3):
        cycle()
    after = _free()
    # allow the allocator's granularity, nothing that grows per cycle
    assert base - after <= 64 * 2 ** 20, (base, after)
