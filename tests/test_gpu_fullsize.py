"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: p = 4, q = 6, 68^3 hexes perturbed 0.15h (20,346,417 DOFs), the
same seeded generators (mesh seed 14, lognormal seed 24, x seed 34); the
precision configuration's p = 6, 45^3 (19,902,511 DOFs); and the sweep
configuration at its 1e6-DOF size for every p = 1..8. The oracle cannot
assemble these matrices, so it computes sampled outputs one DOF at a time
from the rows of the element matrices that hold the DOF
(oracle.assemble.sampled_apply, with its own numbering); properties that
hold at any size are checked on the whole output vector."""

import numpy as np
import pytest

from fem_inputs import hex_lattice, lognormal, x_uniform
from oracle import assemble, numbering

from gpu_util import cuda

pytestmark = pytest.mark.gpu

P, Q, N = 4, 6, 68


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()
    import paper_1911_09220_gb300 as F
    c, h = hex_lattice(N, 0.15, seed=10 + P)
    kap = lognormal(20 + P, h.shape[0])
    num = numbering.build(h, P, nv=c.shape[0])
    n = num["ndof"]
    x = x_uniform(30 + P, n)
    space = F.Space(F.Mesh(c, h), P)
    assert space.ndof == n == 20346417
    # samples: every kind of DOF (vertices, edges, faces, interiors), on and
    # off the boundary, plus uniformly drawn ones
    rng = np.random.default_rng(5)
    nv = c.shape[0]
    n_edge_dofs = num["n_edges"] * (P - 1)
    n_face_dofs = num["n_faces"] * (P - 1) ** 2
    starts = [0, nv, nv + n_edge_dofs, nv + n_edge_dofs + n_face_dofs, n]
    rows = [rng.integers(starts[k], starts[k + 1], 12) for k in range(4)]
    rows.append(rng.choice(num["boundary_dofs"], 12, replace=False))
    rows.append(rng.integers(0, n, 20))
    rows = np.unique(np.concatenate(rows))
    return {"c": c, "h": h, "kap": kap, "num": num, "x": x, "space": space, "rows": rows, "F": F}


def _sampled(full, kind):
    return assemble.sampled_apply(full["c"], full["h"], full["num"]["e2l"], P, Q, kind, full["kap"], full["x"],
                                  full["rows"])


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
def test_sampled_rows(full, kind):
    import torch
    F = full["F"]
    form = F.Form(full["space"], kind, Q, coef=cuda(full["kap"]))
    xd = cuda(full["x"])
    y = torch.empty_like(xd)
    ref = _sampled(full, kind)
    scale = np.abs(ref).max()
    rows = torch.as_tensor(full["rows"], device="cuda")
    form.apply(xd, y)
    assert np.abs(y[rows].cpu().numpy() - ref).max() <= 1e-12 * scale
    form.apply(xd, y, arith="df64")
    assert np.abs(y[rows].cpu().numpy() - ref).max() <= 1e-12 * scale
    y32 = torch.empty(xd.numel(), dtype=torch.float32, device="cuda")
    form.apply(xd.float(), y32)
    assert np.abs(y32[rows].double().cpu().numpy() - ref).max() <= 2e-5 * scale


def test_properties_on_the_whole_vector(full):
    """Constants in the diffusion kernel, symmetry u.(A v) = v.(A u), and
    positivity of u.(A u), evaluated on all 20.3M entries."""
    import torch
    F = full["F"]
    form = F.Form(full["space"], "diffusion", Q, coef=cuda(full["kap"]))
    n = full["space"].ndof
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(one)
    form.apply(one, y)
    u = cuda(full["x"])
    v = cuda(x_uniform(99, n))
    Au, Av = torch.empty_like(u), torch.empty_like(u)
    form.apply(u, Au)
    form.apply(v, Av)
    assert y.abs().max().item() <= 1e-12 * Au.abs().max().item()
    a, b = torch.dot(u, Av).item(), torch.dot(v, Au).item()
    assert abs(a - b) <= 1e-12 * (u.abs() * Av.abs()).sum().item()
    assert torch.dot(u, Au).item() > 0


# (p, N): the sweep's 1e6-DOF lattices (p = 1..8) and the precision
# configuration's p = 6 at ~2e7 DOFs; q = p + 2, the sweep's seeds
CONFIG_SIZES = [(1, 99), (2, 49), (3, 33), (4, 25), (5, 20), (6, 16), (7, 14), (8, 12), (6, 45)]


@pytest.mark.parametrize("p,N", CONFIG_SIZES)
def test_sampled_rows_config_sizes(p, N):
    import torch
    import paper_1911_09220_gb300 as F
    q = p + 2
    c, h = hex_lattice(N, 0.15, seed=10 + p)
    kap = lognormal(20 + p, h.shape[0])
    num = numbering.build(h, p, nv=c.shape[0])
    n = num["ndof"]
    space = F.Space(F.Mesh(c, h), p)
    assert space.ndof == n
    x = x_uniform(30 + p, n)
    rng = np.random.default_rng(100 + p)
    nv = c.shape[0]
    starts = [0, nv, nv + num["n_edges"] * (p - 1), nv + num["n_edges"] * (p - 1) + num["n_faces"] * (p - 1) ** 2, n]
    rows = [rng.integers(starts[k], starts[k + 1], 6) for k in range(4) if starts[k + 1] > starts[k]]
    rows.append(rng.choice(num["boundary_dofs"], 6, replace=False))
    rows.append(rng.integers(0, n, 10))
    rows = np.unique(np.concatenate(rows))
    xd = cuda(x)
    rt = torch.as_tensor(rows, device="cuda")
    for kind in ("diffusion", "mass"):
        ref = assemble.sampled_apply(c, h, num["e2l"], p, q, kind, kap, x, rows)
        scale = np.abs(ref).max()
        form = F.Form(space, kind, q, coef=cuda(kap))
        y = torch.empty_like(xd)
        form.apply(xd, y)
        assert np.abs(y[rt].cpu().numpy() - ref).max() <= 1e-12 * scale, (kind, "f64")
        form.apply(xd, y, arith="df64")
        assert np.abs(y[rt].cpu().numpy() - ref).max() <= 1e-12 * scale, (kind, "df64")
        y32 = torch.empty(n, dtype=torch.float32, device="cuda")
        form.apply(xd.float(), y32)
        assert np.abs(y32[rt].double().cpu().numpy() - ref).max() <= 2e-5 * scale, (kind, "f32")
        del form, y, y32


def test_solves_at_full_size(full):
    """Mixed-precision PCG and p-multigrid (FP32 V-cycle, double-float outer)
    at 20.3M DOFs to 1e-10, with the true residual recomputed by the test
    from the constrained FP64 apply (parity-checked above at this size)."""
    import torch
    F = full["F"]
    space = full["space"]
    form = F.Form(space, "diffusion", Q, coef=cuda(full["kap"]))
    form.set_essential(full["num"]["boundary_dofs"])
    n = space.ndof
    b = cuda(x_uniform(77, n))
    bc = torch.empty_like(b)
    form.lift_rhs(b, torch.zeros_like(b), bc)
    bn = torch.linalg.norm(bc).item()
    r = torch.empty_like(bc)

    def resid(u):
        form.apply(u, r, constrained=True)
        return torch.linalg.norm(bc - r).item() / bn

    u = torch.zeros_like(bc)
    info = form.solve(bc, u, rtol=1e-10, precision="mixed")
    assert info["converged"] and resid(u) <= 1.01e-10
    mg = F.Multigrid(form, precision="f32")
    u2 = torch.zeros_like(bc)
    info = mg.solve(bc, u2, rtol=1e-10, arith="df64")
    assert info["converged"] and info["iterations"] <= 25 and resid(u2) <= 1.01e-10
    # the two solutions agree to the conditioning of the problem
    assert (u - u2).abs().max().item() <= 1e-6 * u.abs().max().item()
