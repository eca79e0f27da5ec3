"""Batched PA applies and Jacobi-PCG over many independent problems (mixed
orders, sizes and kinds, several right-hand sides each, hexahedral and
quadrilateral meshes in one batch) against the oracle and against the
single-problem path; the tile autotuner and its cache."""

import json
import os

import numpy as np
import pytest

from fem_inputs import lognormal, quad_lattice, x_uniform, splitmix64
from oracle import assemble, solve as osolve, twod

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


def _batch(nprob=10, nrhs=3, seed=300, kinds=("diffusion",), oracle=True, Nmax=4):
    import paper_1911_09220_gb300 as F
    draws = splitmix64(seed, 3 * nprob)
    probs = []
    for i in range(nprob):
        N = 1 + int(draws[3 * i] % np.uint64(Nmax))
        p = 1 + int(draws[3 * i + 1] % np.uint64(6))
        kind = kinds[int(draws[3 * i + 2] % np.uint64(len(kinds)))]
        c, h = make_mesh(N, seed=seed + i, shuffle=(i % 2 == 1), drop=(1 if N > 1 and i % 3 == 0 else 0))
        kappa = lognormal(seed + 100 + i, h.shape[0])
        mesh = F.Mesh(c, h)
        space = F.Space(mesh, p)
        form = F.Form(space, kind, p + 2, coef=cuda(kappa))
        prob = assemble.Problem(c, h, p, p + 2, kappa=kappa, rho=kappa) if oracle else None
        probs.append(dict(mesh=mesh, space=space, form=form, prob=prob, kind=kind, p=p))
    return probs, F.Batch([q["form"] for q in probs], nrhs)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_apply_matches_oracle_and_single(dtype):
    import torch
    probs, bt = _batch(kinds=("diffusion", "mass"))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    X = cuda(x_uniform(301, bt.total_len), tdt)
    Y = torch.full_like(X, np.nan)
    bt.apply(X, Y)
    bt.apply(X, Y)   # graph replay
    for i, q in enumerate(probs):
        for r in range(bt.nrhs):
            x = bt.block(X, i, r).contiguous()
            y1 = torch.empty_like(x)
            q["form"].apply(x, y1)
            yb = bt.block(Y, i, r)
            assert relerr(yb.cpu().double().numpy(), y1.cpu().double().numpy()) <= (TOL if dtype == "f64" else 1e-6)
            if dtype == "f64":
                ref = q["prob"].apply(q["kind"], x.cpu().numpy())
                assert relerr(yb.cpu().numpy(), ref) <= TOL


def test_batched_constrained_apply():
    import torch
    probs, bt = _batch(nprob=6, nrhs=2, seed=320)
    for q in probs:
        q["form"].set_essential(q["prob"].num["boundary_dofs"])
    X = cuda(x_uniform(321, bt.total_len))
    Y = torch.empty_like(X)
    bt.apply(X, Y, constrained=True)
    for i, q in enumerate(probs):
        Ac = osolve.constrain(q["prob"].K, q["prob"].num["boundary_dofs"])
        for r in range(bt.nrhs):
            ref = Ac @ bt.block(X, i, r).cpu().numpy()
            assert relerr(bt.block(Y, i, r).cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_batched_solve(precision):
    import torch
    probs, bt = _batch(nprob=8, nrhs=3, seed=340)
    Bc = torch.empty(bt.total_len, dtype=torch.float64, device="cuda")
    raw = cuda(x_uniform(341, bt.total_len))
    for i, q in enumerate(probs):
        q["form"].set_essential(q["prob"].num["boundary_dofs"])
        for r in range(bt.nrhs):
            q["form"].lift_rhs(bt.block(raw, i, r).contiguous(), torch.zeros(q["space"].ndof, dtype=torch.float64,
                                                                              device="cuda"), bt.block(Bc, i, r))
    X = torch.zeros_like(Bc)
    info = bt.solve(Bc, X, rtol=1e-10, precision=precision, check_every=8)
    assert np.all(info["relres"] <= 1e-10)
    for i, q in enumerate(probs):
        ess = q["prob"].num["boundary_dofs"]
        Ac = osolve.constrain(q["prob"].K, ess)
        for r in range(bt.nrhs):
            b = osolve.constrain_rhs(q["prob"].K, bt.block(raw, i, r).cpu().numpy(), ess)
            u = bt.block(X, i, r).cpu().numpy()
            assert np.linalg.norm(b - Ac @ u) / np.linalg.norm(b) <= 1.01e-10, (i, r)


def test_autotuner_cache(tmp_path):
    import torch
    probs, bt = _batch(nprob=6, nrhs=2, seed=360, oracle=False)
    X = cuda(x_uniform(361, bt.total_len))
    Y0 = torch.empty_like(X)
    bt.apply(X, Y0)
    path = tmp_path / "tiles.json"
    tiles = bt.tune("f64", path)
    lines = [json.loads(l) for l in open(path)]
    ps = sorted({(q["p"], q["p"] + 2) for q in probs})
    assert len(lines) == len(ps)
    for p, q in ps:
        t = tiles[2 * p + 1]
        assert 1 <= t <= 256 // (q * q)
    Y1 = torch.empty_like(X)
    bt.apply(X, Y1)
    assert torch.equal(Y0, Y1)        # tiles change the schedule, not the arithmetic
    # a second tuning reads the cache
    tiles2 = bt.tune("f64", path)
    assert np.array_equal(tiles, tiles2)


def test_batch_rejects_high_order():
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(1)
    form = F.Form(F.Space(F.Mesh(c, h), 7), "diffusion", 9)
    with pytest.raises(F.FemError) as ei:
        F.Batch([form], 2)
    assert "FEM_EUNSUPPORTED" in str(ei.value)


@pytest.mark.parametrize("kind", ["diffusion", "mass"])
def test_vector_form_is_a_one_problem_batch(kind):
    """A vector mass / diffusion form (the scalar operator on each of vdim
    components with the same D, components node-major) is a batch of one
    problem with nrhs = vdim: against the oracle's block-diagonal I (x) A."""
    import scipy.sparse as sp
    import torch
    import paper_1911_09220_gb300 as F
    c, h = make_mesh(3, seed=77, shuffle=True, drop=2)
    kappa = lognormal(78, h.shape[0])
    space = F.Space(F.Mesh(c, h), 3)
    form = F.Form(space, kind, 5, coef=cuda(kappa))
    prob = assemble.Problem(c, h, 3, 5, kappa=kappa, rho=kappa)
    vdim = 3
    bt = F.Batch([form], vdim)
    X = cuda(x_uniform(79, bt.total_len))
    Y = torch.empty_like(X)
    bt.apply(X, Y)
    A = sp.kron(sp.identity(vdim), prob.matrix(kind)).tocsr()
    assert relerr(Y.cpu().numpy(), A @ X.cpu().numpy()) <= TOL


def test_config_size_batch():
    """The batching configuration at full size, in the bench's launch
    configuration: 256 diffusion problems, N_i ~ U{2..24} and p_i ~ U{1..6}
    from SplitMix64 seed 40 (N = 2 + d mod 23, p = 1 + d mod 6 on
    alternating draws), meshes seeded 4000 + i, kappa 5000 + i, 8
    right-hand sides from x seed 41 (71.5M DOFs, 572M unknowns). Every
    problem and right-hand side against the single-problem apply (FP64
    1e-12, FP32 2e-5 relative), and sampled rows of three problems against
    the oracle's row-by-row apply."""
    import torch
    import paper_1911_09220_gb300 as F
    from fem_inputs import hex_lattice
    from oracle import numbering
    d = splitmix64(40, 512)
    Ns = [2 + int(v % np.uint64(23)) for v in d[0::2]]
    ps = [1 + int(v % np.uint64(6)) for v in d[1::2]]
    forms, meshes = [], []
    for i, (N, p) in enumerate(zip(Ns, ps)):
        c, h = hex_lattice(N, 0.15, seed=4000 + i)
        kap = lognormal(5000 + i, h.shape[0])
        sp = F.Space(F.Mesh(c, h), p)
        forms.append(F.Form(sp, "diffusion", p + 2, coef=cuda(kap)))
        meshes.append((c, h, kap))
    bt = F.Batch(forms, 8)
    assert bt.total_len == 8 * int(bt.off[-1])
    X = cuda(x_uniform(41, bt.total_len))
    Y = torch.empty_like(X)
    bt.apply(X, Y)
    for i, f in enumerate(forms):
        for r in (0, 7):
            x = bt.block(X, i, r).contiguous()
            y = torch.empty_like(x)
            f.apply(x, y)
            assert relerr(bt.block(Y, i, r).cpu().numpy(), y.cpu().numpy()) <= TOL, (i, r)
    # FP32 batch on the same systems
    X32 = X.float()
    Y32 = torch.empty_like(X32)
    bt.apply(X32, Y32)
    for i in range(0, 256, 17):
        x = bt.block(X32, i, 3).contiguous()
        y = torch.empty_like(x)
        forms[i].apply(x, y)
        assert relerr(bt.block(Y32, i, 3).double().cpu().numpy(), y.double().cpu().numpy()) <= 2e-5, i
    # oracle rows for the three largest problems
    big = sorted(range(256), key=lambda i: -forms[i].space.ndof)[:3]
    for i in big:
        c, h, kap = meshes[i]
        p = ps[i]
        num = numbering.build(h, p, nv=c.shape[0])
        x = bt.block(X, i, 5).cpu().numpy()
        rows = np.unique(np.random.default_rng(i).integers(0, num["ndof"], 40))
        ref = assemble.sampled_apply(c, h, num["e2l"], p, p + 2, "diffusion", kap, x, rows)
        got = bt.block(Y, i, 5).cpu().numpy()[rows]
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max(), i


def _mixed_dims(nprob=10, nrhs=3, seed=380):
    """Every other problem on a perturbed quadrilateral mesh, the others on
    hexahedra; p = 1..6, diffusion and mass."""
    import paper_1911_09220_gb300 as F
    draws = splitmix64(seed, 3 * nprob)
    probs = []
    for i in range(nprob):
        p = 1 + int(draws[3 * i] % np.uint64(6))
        kind = ("diffusion", "mass")[int(draws[3 * i + 1] % np.uint64(2))]
        if i % 2 == 0:
            N = 2 + int(draws[3 * i + 2] % np.uint64(5))
            c, qd = quad_lattice(N, 0.2, seed=seed + i, shuffle=(i % 4 == 0))
            kappa = lognormal(seed + 100 + i, qd.shape[0])
            space = F.Space(F.Mesh2D(c, qd), p)
            prob = twod.Problem2(c, qd, p, p + 2, kappa=kappa, rho=kappa)
        else:
            N = 1 + int(draws[3 * i + 2] % np.uint64(3))
            c, h = make_mesh(N, seed=seed + i, shuffle=True)
            kappa = lognormal(seed + 100 + i, h.shape[0])
            space = F.Space(F.Mesh(c, h), p)
            prob = assemble.Problem(c, h, p, p + 2, kappa=kappa, rho=kappa)
        form = F.Form(space, kind, p + 2, coef=cuda(kappa))
        probs.append(dict(space=space, form=form, prob=prob, kind=kind, p=p))
    return probs, F.Batch([q["form"] for q in probs], nrhs)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_mixes_quadrilaterals_and_hexahedra(dtype):
    import torch
    probs, bt = _mixed_dims()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    X = cuda(x_uniform(381, bt.total_len), tdt)
    Y = torch.full_like(X, np.nan)
    bt.apply(X, Y)
    bt.apply(X, Y)   # graph replay
    for i, q in enumerate(probs):
        for r in range(bt.nrhs):
            x = bt.block(X, i, r).contiguous()
            y1 = torch.empty_like(x)
            q["form"].apply(x, y1)
            yb = bt.block(Y, i, r)
            assert relerr(yb.cpu().double().numpy(), y1.cpu().double().numpy()) <= (TOL if dtype == "f64" else 1e-6)
            ref = q["prob"].apply(q["kind"], x.cpu().double().numpy())
            assert relerr(yb.cpu().double().numpy(), ref) <= (TOL if dtype == "f64" else 2e-5), (i, r)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_batch_mixed_dims_constrained_and_solve(precision):
    import torch
    probs, bt = _mixed_dims(nprob=8, nrhs=2, seed=390)
    raw = cuda(x_uniform(391, bt.total_len))
    Bc = torch.empty_like(raw)
    for i, q in enumerate(probs):
        ess = q["space"].boundary_dofs()
        q["form"].set_essential(cuda(ess))
        for r in range(bt.nrhs):
            q["form"].lift_rhs(bt.block(raw, i, r).contiguous(),
                               torch.zeros(q["space"].ndof, dtype=torch.float64, device="cuda"), bt.block(Bc, i, r))
    Y = torch.empty_like(raw)
    bt.apply(raw, Y, constrained=True)
    for i, q in enumerate(probs):
        ess = q["space"].boundary_dofs()
        Ac = osolve.constrain(q["prob"].matrix(q["kind"]), ess)
        for r in range(bt.nrhs):
            assert relerr(bt.block(Y, i, r).cpu().numpy(), Ac @ bt.block(raw, i, r).cpu().numpy()) <= TOL
    X = torch.zeros_like(Bc)
    info = bt.solve(Bc, X, rtol=1e-10, precision=precision, check_every=8)
    assert np.all(info["relres"] <= 1e-10)
    for i, q in enumerate(probs):
        ess = q["space"].boundary_dofs()
        A = q["prob"].matrix(q["kind"])
        Ac = osolve.constrain(A, ess)
        for r in range(bt.nrhs):
            b = osolve.constrain_rhs(A, bt.block(raw, i, r).cpu().numpy(), ess)
            u = bt.block(X, i, r).cpu().numpy()
            assert np.linalg.norm(b - Ac @ u) / np.linalg.norm(b) <= 1.01e-10, (i, r)
