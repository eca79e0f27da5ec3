"""The sharded operator on the GPU: two and three ranks as separate processes
on the one GPU (each its own CUDA context), exchanging halos through gloo
(fem_comm callbacks with host copies; no kernel waits for another rank).
Each rank builds the global space, its shard, and a form on the shard's
local space; through the C ABI it runs the sharded apply (unconstrained and
constrained), the assembled diagonal, the load vector and Jacobi-PCG. The
results must equal the oracle's on every local DOF (1e-12 relative in the
max norm), agree bit for bit between ranks holding the same DOF, and the
sharded PCG must converge to the single-GPU solution in the same number of
iterations (dot products are summed over ranks in another order, so a
difference of a few iterations is allowed) with the oracle's true residual
below 1e-10. The elasticity form checks the three-component exchange."""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_09220_gb300 import build
    build.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _rank_main(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1911_09220_gb300 as F
        from paper_1911_09220_gb300 import shard as S
        from fem_inputs import hex_lattice, lognormal, x_uniform
        from oracle import assemble, elasticity as oel, solve as osolve
        res = {}
        p, N = case["p"], case["N"]
        q = p + 2
        c, h = hex_lattice(N, 0.15, seed=31 + p, shuffle=True)
        E = h.shape[0]
        gmesh = F.Mesh(c, h)
        gspace = F.Space(gmesh, p)
        part = S.partition_slabs(gmesh, world)
        sh = S.Shard(gspace, part, world, rank)
        t = sh.tables()
        elems, l2g, owned = t["elems"], t["l2g"], t["owned"]
        comm = S.TorchComm()
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")

        def assemble_global(yl, vdim=1):
            """Owned entries of every rank summed into the global vector."""
            full = torch.zeros(vdim * sh.ndof_global, dtype=torch.float64)
            yh = yl.cpu().numpy().reshape(vdim, -1)
            for cc in range(vdim):
                full[torch.from_numpy(cc * sh.ndof_global + l2g[owned])] = torch.from_numpy(yh[cc][owned])
            dist.all_reduce(full)
            return full.numpy()

        def consistent(yl, vdim=1):
            full = assemble_global(yl, vdim).reshape(vdim, -1)
            return int(np.count_nonzero(full[:, l2g].ravel() != yl.cpu().numpy()))

        if case["kind"] == "diffusion":
            kappa = lognormal(32 + p, E)
            form = F.Form(sh.space, "diffusion", q, coef=cu(kappa[elems]))
            gform = F.Form(gspace, "diffusion", q, coef=cu(kappa))
            prob = assemble.Problem(c, h, p, q, kappa=kappa)
            xg = x_uniform(33, gspace.ndof)
            xl = sh.to_local(cu(xg), torch.empty(sh.ndof, dtype=torch.float64, device="cuda"))
            yl = torch.empty_like(xl)
            sh.apply(form, xl, yl, comm)
            ref = prob.apply("diffusion", xg)
            res["apply"] = _relerr(yl.cpu().numpy(), ref[l2g])
            res["apply_consistent"] = consistent(yl)
            # essential DOFs: the global boundary, localized
            ess_g = gspace.boundary_dofs()
            ess_l = sh.localize(ess_g)
            form.set_essential(cu(ess_l[ess_l >= 0]))
            gform.set_essential(cu(ess_g))
            sh.apply(form, xl, yl, comm, constrained=True)
            Ac = osolve.constrain(prob.K, ess_g)
            res["apply_c"] = _relerr(yl.cpu().numpy(), (Ac @ xg)[l2g])
            dl = torch.empty_like(xl)
            sh.diagonal(form, dl, comm, constrained=True)
            res["diag_c"] = _relerr(dl.cpu().numpy(), np.asarray(Ac.diagonal())[l2g])
            # load vector from quadrature-point values of the local elements
            xq = form.qpoint_coords()
            fq = (torch.sin(np.pi * xq[..., 0]) * torch.cos(xq[..., 1]) + xq[..., 2]).contiguous()
            bl = torch.empty_like(xl)
            sh.rhs(form, fq, bl, comm)
            xqg = gform.qpoint_coords()
            fqg = (torch.sin(np.pi * xqg[..., 0]) * torch.cos(xqg[..., 1]) + xqg[..., 2]).contiguous()
            bg = torch.empty(gspace.ndof, dtype=torch.float64, device="cuda")
            gform.rhs(fqg, bg)
            res["rhs"] = _relerr(bl.cpu().numpy(), bg.cpu().numpy()[l2g])
            res["rhs_consistent"] = consistent(bl)
            # PCG: the single-GPU constrained system, solved sharded
            bcg = torch.empty_like(bg)
            gform.lift_rhs(bg, torch.zeros_like(bg), bcg)
            ug = torch.zeros_like(bg)
            info_g = gform.solve(bcg, ug, rtol=1e-10)
            bcl = sh.to_local(bcg, torch.empty_like(xl))
            ul = torch.zeros_like(xl)
            info = sh.solve(form, bcl, ul, comm, rtol=1e-10)
            uf = assemble_global(ul)
            bch = bcg.cpu().numpy()
            res["solve_relres"] = float(np.linalg.norm(bch - Ac @ uf) / np.linalg.norm(bch))
            res["solve_vs_single"] = _relerr(uf, ug.cpu().numpy())
            res["iters"] = (info["iterations"], info_g["iterations"])
            res["dot"] = abs(sh.dot(bcl, bcl, comm) - float(bch @ bch)) / float(bch @ bch)
        else:
            lam, mu = lognormal(34 + p, E), lognormal(35 + p, E)
            form = F.Form.elasticity(sh.space, cu(lam[elems]), cu(mu[elems]), q1d=q)
            prob = oel.ElasticityProblem(c, h, p, q, lam, mu)
            xg = x_uniform(36, 3 * gspace.ndof)
            xl = sh.to_local(cu(xg), torch.empty(3 * sh.ndof, dtype=torch.float64, device="cuda"), vdim=3)
            yl = torch.empty_like(xl)
            sh.apply(form, xl, yl, comm)
            ref = prob.apply(xg).reshape(3, -1)
            res["apply"] = _relerr(yl.cpu().numpy(), ref[:, l2g].ravel())
            res["apply_consistent"] = consistent(yl, 3)
        res["nnbr"] = sh.nnbr
        out[rank] = res
    finally:
        dist.barrier()
        dist.destroy_process_group()


CASES = [
    (2, {"kind": "diffusion", "p": 2, "N": 5}),
    (3, {"kind": "diffusion", "p": 3, "N": 4}),
    (2, {"kind": "elasticity", "p": 2, "N": 3}),
]


@pytest.mark.parametrize("world,case", CASES)
def test_sharded_operator_matches_oracle(world, case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=600)
        assert pr.exitcode == 0
    for r in range(world):
        res = out[r]
        assert res["nnbr"] >= 1
        assert res["apply"] <= 1e-12, (r, res)
        assert res["apply_consistent"] == 0, (r, res)
        if case["kind"] == "diffusion":
            assert res["apply_c"] <= 1e-12, (r, res)
            assert res["diag_c"] <= 1e-12, (r, res)
            assert res["rhs"] <= 1e-12 and res["rhs_consistent"] == 0, (r, res)
            assert res["solve_relres"] <= 1.01e-10, (r, res)
            assert res["solve_vs_single"] <= 1e-8, (r, res)
            its, its_single = res["iters"]
            assert abs(its - its_single) <= 3, (r, res)
            assert res["dot"] <= 1e-13, (r, res)
