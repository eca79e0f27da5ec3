"""The sharded operator's host side on CPU: the element partition and the
plan of each rank's shard (csrc/fem_shard.cpp, compiled with the library's
host code against the test-only CUDA runtime stand-in of tests/host_stub),
and the exchange protocol run by world_size-2 and -3 gloo ranks.

The plan must hold the invariants the parallel operator
A = P^T G^T B^T D B G P (Sec. 4.3) rests on: every global DOF owned by
exactly one rank, the local -> global map agreeing with both numberings,
neighbour slot lists that match on both ends, and a combine table that adds
every holder's partial once. Then each rank applies its local part of the
oracle's assembled operator (the oracle's own element matrices on the
rank's elements), exchanges the partials of its shared DOFs through gloo
and combines them in the plan's order: the result must equal the oracle's
global product on every local DOF, and ranks holding the same DOF must hold
the same bits."""

import ctypes as C
import os
import socket
import subprocess

import numpy as np
import pytest

from fem_inputs import hex_lattice, lognormal, quad_lattice, x_uniform
from oracle import assemble, numbering, twod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_09220_gb300", "csrc")
P, I64, I = C.c_void_p, C.c_int64, C.c_int


def build_host_lib(out):
    cmd = ["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-Wl,-Bsymbolic",
           "-I", os.path.join(ROOT, "tests", "host_stub"), "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(CSRC, "fem_host.cpp"), os.path.join(CSRC, "fem_basis.cpp"), os.path.join(CSRC, "fem_shard.cpp"),
           os.path.join(ROOT, "tests", "host_stub", "stub.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def load_host_lib(path):
    L = C.CDLL(path, mode=C.RTLD_LOCAL)
    for name, res, args in [("fem_mesh_create", I, [P, I64, P, I64, C.POINTER(P)]),
                            ("fem_mesh2d_create", I, [P, I64, P, I64, C.POINTER(P)]),
                            ("fem_space_create", I, [P, I, C.POINTER(P)]),
                            ("fem_space_info", I, [P, P, P, P, P]),
                            ("fem_space_element_dofs", I, [P, P]),
                            ("fem_partition_slabs", I, [P, I, P]),
                            ("fem_shard_create", I, [P, P, I, I, C.POINTER(P)]),
                            ("fem_shard_space", P, [P]),
                            ("fem_shard_info", I, [P, P, P, P, P, P, P]),
                            ("fem_shard_tables", I, [P, P, P, P, P, P, P]),
                            ("fem_shard_combine_table", I, [P, P, P, P, P, P]),
                            ("fem_shard_localize", I, [P, P, I64, P]),
                            ("fem_shard_destroy", None, [P]), ("fem_space_destroy", None, [P]),
                            ("fem_mesh_destroy", None, [P]), ("fem_last_error", C.c_char_p, [])]:
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    return L


@pytest.fixture(scope="module")
def libpath(tmp_path_factory):
    return build_host_lib(str(tmp_path_factory.mktemp("shardlib") / "libfem_shard_test.so"))


@pytest.fixture(scope="module")
def hostlib(libpath):
    return load_host_lib(libpath)


class Global:
    def __init__(self, L, coords, cells, p):
        self.L = L
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.cells = np.ascontiguousarray(cells, dtype=np.int32)
        self.dim = self.coords.shape[1]
        self.p = p
        self.m = P()
        create = L.fem_mesh_create if self.dim == 3 else L.fem_mesh2d_create
        assert create(self.coords.ctypes.data, self.coords.shape[0], self.cells.ctypes.data, self.cells.shape[0],
                      C.byref(self.m)) == 0, L.fem_last_error()
        self.s = P()
        assert L.fem_space_create(self.m, p, C.byref(self.s)) == 0, L.fem_last_error()
        ndof = I64()
        assert L.fem_space_info(self.s, C.byref(ndof), None, None, None) == 0
        self.ndof = ndof.value
        self.nd = (p + 1) ** self.dim
        self.e2l = np.empty((self.cells.shape[0], self.nd), dtype=np.int32)
        assert L.fem_space_element_dofs(self.s, self.e2l.ctypes.data) == 0

    def partition(self, nparts):
        part = np.empty(self.cells.shape[0], dtype=np.int32)
        st = self.L.fem_partition_slabs(self.m, nparts, part.ctypes.data)
        assert st == 0, self.L.fem_last_error()
        return part

    def shard(self, part, nparts, rank):
        L = self.L
        h = P()
        assert L.fem_shard_create(self.s, part.ctypes.data, nparts, rank, C.byref(h)) == 0, L.fem_last_error()
        ne, nl, no, ns, ng = I64(), I64(), I64(), I64(), I64()
        nn = I()
        assert L.fem_shard_info(h, C.byref(ne), C.byref(nl), C.byref(no), C.byref(nn), C.byref(ns), C.byref(ng)) == 0
        t = {"ne": ne.value, "ndof": nl.value, "n_owned": no.value, "nnbr": nn.value, "nslots": ns.value,
             "ndof_global": ng.value}
        t["elems"] = np.empty(t["ne"], dtype=np.int64)
        t["l2g"] = np.empty(t["ndof"], dtype=np.int64)
        t["owned"] = np.empty(t["ndof"], dtype=np.uint8)
        t["nbr"] = np.empty(t["nnbr"], dtype=np.int32)
        t["slot_off"] = np.empty(t["nnbr"] + 1, dtype=np.int64)
        t["slot_dof"] = np.empty(t["nslots"], dtype=np.int32)
        assert L.fem_shard_tables(h, t["elems"].ctypes.data, t["l2g"].ctypes.data, t["owned"].ctypes.data,
                                  t["nbr"].ctypes.data, t["slot_off"].ctypes.data, t["slot_dof"].ctypes.data) == 0
        nsh, nent = I64(), I64()
        assert L.fem_shard_combine_table(h, C.byref(nsh), C.byref(nent), None, None, None) == 0
        t["comb_dof"] = np.empty(nsh.value, dtype=np.int32)
        t["comb_off"] = np.empty(nsh.value + 1, dtype=np.int32)
        t["comb_src"] = np.empty(nent.value, dtype=np.int32)
        assert L.fem_shard_combine_table(h, None, None, t["comb_dof"].ctypes.data, t["comb_off"].ctypes.data,
                                         t["comb_src"].ctypes.data) == 0
        ls = L.fem_shard_space(h)
        t["e2l"] = np.empty((t["ne"], self.nd), dtype=np.int32)
        assert L.fem_space_element_dofs(ls, t["e2l"].ctypes.data) == 0
        g = np.ascontiguousarray(t["l2g"].astype(np.int32))
        loc = np.empty(g.shape[0], dtype=np.int32)
        assert L.fem_shard_localize(h, g.ctypes.data, g.shape[0], loc.ctypes.data) == 0
        t["localized"] = loc
        missing = np.setdiff1d(np.arange(self.ndof, dtype=np.int32), g)[:50]
        loc2 = np.empty(missing.shape[0], dtype=np.int32)
        if missing.shape[0]:
            assert L.fem_shard_localize(h, np.ascontiguousarray(missing).ctypes.data, missing.shape[0],
                                        loc2.ctypes.data) == 0
        t["localized_missing"] = loc2
        L.fem_shard_destroy(h)
        return t


def local_mesh(coords, cells, elems):
    """The shard's local mesh as the plan defines it: its elements in
    ascending global number, their vertices in ascending global number."""
    sub = cells[elems]
    used = np.unique(sub)
    remap = -np.ones(coords.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    return coords[used], remap[sub]


def mesh3(N, seed, shuffle):
    return hex_lattice(N, 0.15, seed=seed, shuffle=shuffle)


def centroid_axis_values(coords, cells):
    cen = coords[cells].mean(axis=1)
    axis = int(np.argmax(cen.max(axis=0) - cen.min(axis=0)))
    return cen[:, axis]


@pytest.mark.parametrize("dim,shuffle", [(3, False), (3, True), (2, True)])
def test_partition_is_balanced_slabs(hostlib, dim, shuffle):
    c, h = mesh3(6, 3, shuffle) if dim == 3 else quad_lattice(9, 0.2, seed=3, shuffle=shuffle)
    g = Global(hostlib, c, h, 1)
    ax = centroid_axis_values(g.coords, g.cells)
    for R in (1, 2, 3, 5):
        part = g.partition(R)
        counts = np.bincount(part, minlength=R)
        assert counts.max() - counts.min() <= 1 and counts.sum() == h.shape[0]
        for r in range(R - 1):  # slabs: part r lies below part r + 1 along the axis
            assert ax[part == r].max() <= ax[part == r + 1].min()
        assert np.array_equal(part, g.partition(R))
    bad = np.empty(h.shape[0], dtype=np.int32)
    assert hostlib.fem_partition_slabs(g.m, 0, bad.ctypes.data) != 0
    assert hostlib.fem_partition_slabs(g.m, h.shape[0] + 1, bad.ctypes.data) != 0


@pytest.mark.parametrize("dim,p,R,shuffle", [(3, 2, 2, False), (3, 2, 3, True), (3, 1, 4, True), (2, 3, 3, True)])
def test_plan_invariants(hostlib, dim, p, R, shuffle):
    c, h = mesh3(4, 5, shuffle) if dim == 3 else quad_lattice(7, 0.2, seed=5, shuffle=shuffle)
    g = Global(hostlib, c, h, p)
    part = g.partition(R)
    plans = [g.shard(part, R, r) for r in range(R)]
    owners = np.zeros(g.ndof, dtype=np.int64)
    holders = [set() for _ in range(g.ndof)]
    for e in range(h.shape[0]):
        for gi in g.e2l[e]:
            holders[gi].add(int(part[e]))
    for r, t in enumerate(plans):
        assert np.array_equal(t["elems"], np.flatnonzero(part == r))
        # the local numbering is the documented one on the local mesh (the
        # oracle's independent construction) and l2g matches both tables
        lc, lh = local_mesh(g.coords, g.cells, t["elems"])
        num = numbering.build(lh, p, nv=lc.shape[0]) if dim == 3 else twod.numbering2(lh, p, nv=lc.shape[0])
        assert np.array_equal(t["e2l"], num["e2l"])
        assert np.array_equal(t["l2g"][t["e2l"]], g.e2l[t["elems"]])
        assert np.unique(t["l2g"]).shape[0] == t["ndof"]
        # ownership: the lowest holding rank
        for i in range(t["ndof"]):
            assert bool(t["owned"][i]) == (min(holders[t["l2g"][i]]) == r)
        owners[t["l2g"][t["owned"].astype(bool)]] += 1
        assert t["n_owned"] == int(t["owned"].sum())
        # neighbours: the other ranks that hold one of this rank's DOFs
        nb = sorted(set().union(*[holders[gi] for gi in t["l2g"]]) - {r})
        assert list(t["nbr"]) == nb
        # localize: inverse of l2g, -1 off the shard
        assert np.array_equal(t["localized"], np.arange(t["ndof"]))
        assert np.all(t["localized_missing"] == -1)
    assert np.all(owners == 1)  # every global DOF owned exactly once
    # slot lists agree on both ends: same global DOFs in the same (ascending) order
    for a, ta in enumerate(plans):
        for k, b in enumerate(ta["nbr"]):
            tb = plans[b]
            kb = list(tb["nbr"]).index(a)
            ga = ta["l2g"][ta["slot_dof"][ta["slot_off"][k]:ta["slot_off"][k + 1]]]
            gb = tb["l2g"][tb["slot_dof"][tb["slot_off"][kb]:tb["slot_off"][kb + 1]]]
            assert np.array_equal(ga, gb) and np.all(np.diff(ga) > 0)
            assert set(ga) == {gi for gi in range(g.ndof) if a in holders[gi] and b in holders[gi]}
    # combine table: every DOF held by several ranks, one entry per holder,
    # the own partial once, received partials from the slot of that DOF
    for r, t in enumerate(plans):
        shared = [i for i in range(t["ndof"]) if len(holders[t["l2g"][i]]) > 1]
        assert list(t["comb_dof"]) == shared
        slot_nbr = np.repeat(np.arange(t["nnbr"]), np.diff(t["slot_off"]))
        for j, i in enumerate(t["comb_dof"]):
            ent = t["comb_src"][t["comb_off"][j]:t["comb_off"][j + 1]]
            hs = sorted(holders[t["l2g"][i]])
            assert len(ent) == len(hs) and list(ent).count(-1) == 1 and ent[hs.index(r)] == -1
            for rank_, src in zip(hs, ent):
                if src >= 0:
                    assert t["slot_dof"][src] == i and t["nbr"][slot_nbr[src]] == rank_


def test_shard_errors(hostlib):
    c, h = mesh3(2, 1, False)
    g = Global(hostlib, c, h, 1)
    part = np.zeros(h.shape[0], dtype=np.int32)
    out = P()
    assert hostlib.fem_shard_create(g.s, part.ctypes.data, 2, 1, C.byref(out)) != 0   # rank 1 has no elements
    assert b"no elements" in hostlib.fem_last_error()
    assert hostlib.fem_shard_create(g.s, part.ctypes.data, 65, 0, C.byref(out)) != 0  # more than 64 parts
    part[0] = 7
    assert hostlib.fem_shard_create(g.s, part.ctypes.data, 2, 0, C.byref(out)) != 0   # part out of range


# ------------------------------------------------------- gloo exchange ----
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, libpath, dim, p, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = load_host_lib(libpath)
        if dim == 3:
            c, h = hex_lattice(4, 0.15, seed=21, shuffle=True)
        else:
            c, h = quad_lattice(8, 0.2, seed=21, shuffle=True)
        q = p + 2
        g = Global(L, c, h, p)
        part = g.partition(world)
        t = g.shard(part, world, rank)
        kappa = lognormal(22, h.shape[0])
        x = x_uniform(23, g.ndof)
        # this rank's partial product: the oracle's matrix of its own elements
        lc, lh = local_mesh(g.coords, g.cells, t["elems"])
        if dim == 3:
            loc = assemble.Problem(lc, lh, p, q, kappa=kappa[t["elems"]])
        else:
            loc = twod.Problem2(lc, lh, p, q, kappa=kappa[t["elems"]])
        y = loc.apply("diffusion", x[t["l2g"]])
        # exchange the shared DOFs' partials with every neighbour
        so = t["slot_off"]
        sends = [torch.from_numpy(np.ascontiguousarray(y[t["slot_dof"][so[k]:so[k + 1]]])) for k in range(t["nnbr"])]
        recvs = [torch.empty_like(s_) for s_ in sends]
        ops = []
        for k in range(t["nnbr"]):
            ops.append(dist.P2POp(dist.isend, sends[k], int(t["nbr"][k])))
            ops.append(dist.P2POp(dist.irecv, recvs[k], int(t["nbr"][k])))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        recv = np.concatenate([r_.numpy() for r_ in recvs]) if recvs else np.empty(0)
        # combine in the plan's order
        yc = y.copy()
        for j, i in enumerate(t["comb_dof"]):
            v = 0.0
            for src in t["comb_src"][t["comb_off"][j]:t["comb_off"][j + 1]]:
                v += y[i] if src < 0 else recv[src]
            yc[i] = v
        glob = (assemble.Problem(c, h, p, q, kappa=kappa) if dim == 3
                else twod.Problem2(c, h, p, q, kappa=kappa)).apply("diffusion", x)
        err = float(np.abs(yc - glob[t["l2g"]]).max() / np.abs(glob).max())
        # owned entries reassemble the global vector; shared values agree bit for bit
        full = torch.zeros(g.ndof, dtype=torch.float64)
        own = t["owned"].astype(bool)
        full[torch.from_numpy(t["l2g"][own])] = torch.from_numpy(yc[own])
        dist.all_reduce(full)
        mismatch = int(np.count_nonzero(full.numpy()[t["l2g"]] != yc))
        out[rank] = (err, mismatch, float(np.abs(full.numpy() - glob).max() / np.abs(glob).max()), t["nnbr"])
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dim,p", [(2, 3, 2), (3, 3, 3), (3, 2, 4)])
def test_gloo_ranks_assemble_the_global_operator(libpath, world, dim, p):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, libpath, dim, p, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=240)
        assert pr.exitcode == 0
    for r in range(world):
        err, mismatch, full_err, nnbr = out[r]
        assert err <= 1e-12, (r, err)
        assert mismatch == 0, (r, mismatch)
        assert full_err <= 1e-12
        assert nnbr >= 1
