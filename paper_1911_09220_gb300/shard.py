"""Sharded operator: one rank's element slab of a global problem, its owned +
halo L-vector, and the exchange with the neighbouring ranks (fem_shard_* in
include/fem.h; the paper's parallel A = P^T G^T B^T D B G P, Sec. 4.3, and
the parallel assembly of FormLinearSystem, Sec. 5.1).

Argument marshalling only: the plan is built by the library's host code and
every vector step runs in its kernels. Communication is the caller's: a
`TorchComm` hands the library's exchange and all-reduce callbacks to a
torch.distributed process group (NCCL on device buffers, or gloo through
host copies)."""

import ctypes as C

import numpy as np

from . import _binding as B
from ._binding import FemError
from . import Space, _ptr, _stream

EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                          C.c_void_p, C.c_void_p, C.c_void_p)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p)


class CommStruct(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("host_sync", C.c_int), ("exchange", EXCHANGE_FN),
                ("allreduce", ALLREDUCE_FN)]


class _DeviceArray:
    """A float64 device range as a __cuda_array_interface__ object (a
    zero-copy torch view of a library-owned buffer)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _view(ptr, n):
    import torch
    return torch.as_tensor(_DeviceArray(ptr, n), device="cuda")


class TorchComm:
    """fem_comm over a torch.distributed process group. With the NCCL
    backend the device buffers are sent as they are, ordered on the library's
    stream; any other backend (gloo) gets host copies, and the library
    synchronises its stream before each call."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.group = group
        self.nccl = dist.get_backend(group) == "nccl"
        self._ex = EXCHANGE_FN(self._exchange)
        self._ar = ALLREDUCE_FN(self._allreduce)
        self.struct = CommStruct(None, 0 if self.nccl else 1, self._ex, self._ar)
        self.error = None

    def _run(self, stream, fn):
        import torch
        if self.nccl:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()):
                fn()
        else:
            fn()
            torch.cuda.synchronize()

    def _exchange(self, ctx, nnbr, nbr, off, send, recv, stream):
        import torch.distributed as dist
        try:
            total = int(off[nnbr])
            s_dev, r_dev = _view(send, total), _view(recv, total)

            def go():
                s = s_dev if self.nccl else s_dev.cpu()
                r = r_dev if self.nccl else s.new_empty(total)
                ops = []
                for k in range(nnbr):
                    a, b = int(off[k]), int(off[k + 1])
                    ops.append(dist.P2POp(dist.isend, s[a:b], int(nbr[k]), self.group))
                    ops.append(dist.P2POp(dist.irecv, r[a:b], int(nbr[k]), self.group))
                for q in dist.batch_isend_irecv(ops):
                    q.wait()
                if not self.nccl:
                    r_dev.copy_(r)

            self._run(stream, go)
            return 0
        except Exception as e:  # reported through the library's status
            self.error = e
            return 1

    def _allreduce(self, ctx, vals, n, stream):
        import torch.distributed as dist
        try:
            v_dev = _view(vals, n)

            def go():
                v = v_dev if self.nccl else v_dev.cpu()
                dist.all_reduce(v, op=dist.ReduceOp.SUM, group=self.group)
                if not self.nccl:
                    v_dev.copy_(v)

            self._run(stream, go)
            return 0
        except Exception as e:
            self.error = e
            return 1


def partition_slabs(mesh, nparts):
    """Element -> part (int32 [ne]) of the library's slab partition."""
    part = np.empty(mesh.ne, dtype=np.int32)
    B.check(B.lib().fem_partition_slabs(mesh._h, int(nparts), part.ctypes.data))
    return part


class Shard:
    """Rank `rank` of `nparts` of the global space `gspace` under the element
    partition `part`. Forms for it are built on `shard.space`."""

    def __init__(self, gspace, part, nparts, rank):
        L = B.lib()
        self.gspace = gspace
        self._part = np.ascontiguousarray(part, dtype=np.int32)
        h = C.c_void_p()
        B.check(L.fem_shard_create(gspace._h, self._part.ctypes.data, int(nparts), int(rank), C.byref(h)))
        self._h = h
        self.nparts, self.rank = int(nparts), int(rank)
        ne, nl, no, ns, ng = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        nn = C.c_int()
        B.check(L.fem_shard_info(h, C.byref(ne), C.byref(nl), C.byref(no), C.byref(nn), C.byref(ns), C.byref(ng)))
        self.ne, self.ndof, self.n_owned, self.nnbr = ne.value, nl.value, no.value, nn.value
        self.nslots, self.ndof_global = ns.value, ng.value
        sp = Space.__new__(Space)
        sp._h = C.c_void_p(L.fem_shard_space(h))
        sp.mesh, sp.ndof, sp.ne, sp.p, sp.dim = None, self.ndof, self.ne, gspace.p, gspace.dim
        nb = C.c_int64()
        B.check(L.fem_space_info(sp._h, None, C.byref(nb), None, None))
        sp.nbdr = nb.value
        sp._owner = self       # the shard owns the space; keep it alive
        sp.__class__ = _SpaceView
        self.space = sp

    def tables(self):
        elems = np.empty(self.ne, dtype=np.int64)
        l2g = np.empty(self.ndof, dtype=np.int64)
        owned = np.empty(self.ndof, dtype=np.uint8)
        nbr = np.empty(self.nnbr, dtype=np.int32)
        slot_off = np.empty(self.nnbr + 1, dtype=np.int64)
        slot_dof = np.empty(self.nslots, dtype=np.int32)
        B.check(B.lib().fem_shard_tables(self._h, elems.ctypes.data, l2g.ctypes.data, owned.ctypes.data,
                                         nbr.ctypes.data, slot_off.ctypes.data, slot_dof.ctypes.data))
        return {"elems": elems, "l2g": l2g, "owned": owned.astype(bool), "nbr": nbr, "slot_off": slot_off,
                "slot_dof": slot_dof}

    def combine_table(self):
        ns, nt = C.c_int64(), C.c_int64()
        B.check(B.lib().fem_shard_combine_table(self._h, C.byref(ns), C.byref(nt), None, None, None))
        dof = np.empty(ns.value, dtype=np.int32)
        off = np.empty(ns.value + 1, dtype=np.int32)
        src = np.empty(nt.value, dtype=np.int32)
        B.check(B.lib().fem_shard_combine_table(self._h, None, None, dof.ctypes.data, off.ctypes.data,
                                                src.ctypes.data))
        return {"dof": dof, "off": off, "src": src}

    def localize(self, global_ids):
        g = np.ascontiguousarray(global_ids, dtype=np.int32)
        out = np.empty(g.shape[0], dtype=np.int32)
        B.check(B.lib().fem_shard_localize(self._h, g.ctypes.data, g.shape[0], out.ctypes.data))
        return out

    def to_local(self, xg, xl, vdim=1, stream=None):
        import torch
        B.check(B.lib().fem_shard_to_local(self._h, int(vdim), _ptr(xg, torch.float64, "xg"),
                                           _ptr(xl, torch.float64, "xl"), _stream(stream)))
        return xl

    def to_global(self, xl, xg, vdim=1, stream=None):
        import torch
        B.check(B.lib().fem_shard_to_global(self._h, int(vdim), _ptr(xl, torch.float64, "xl"),
                                            _ptr(xg, torch.float64, "xg"), _stream(stream)))
        return xg

    @staticmethod
    def _comm(comm):
        return None if comm is None else C.byref(comm.struct)

    def _check(self, st, comm):
        if st != B.FEM_OK:
            extra = f" ({comm.error!r})" if comm is not None and comm.error is not None else ""
            raise FemError(st, B.lib().fem_last_error().decode() + extra)

    def apply(self, form, x, y, comm, constrained=False, stream=None):
        import torch
        st = B.lib().fem_shard_apply(self._h, form._h, _ptr(x, torch.float64, "x"), _ptr(y, torch.float64, "y"),
                                     int(bool(constrained)), self._comm(comm), _stream(stream))
        self._check(st, comm)
        return y

    def diagonal(self, form, out, comm, constrained=False, stream=None):
        import torch
        st = B.lib().fem_shard_diagonal(self._h, form._h, _ptr(out, torch.float64, "out"),
                                        int(bool(constrained)), self._comm(comm), _stream(stream))
        self._check(st, comm)
        return out

    def rhs(self, form, fq, b, comm, stream=None):
        import torch
        st = B.lib().fem_shard_rhs(self._h, form._h, _ptr(fq, torch.float64, "fq"), _ptr(b, torch.float64, "b"),
                                   self._comm(comm), _stream(stream))
        self._check(st, comm)
        return b

    def dot(self, a, b, comm, vdim=1, stream=None):
        import torch
        out = C.c_double()
        st = B.lib().fem_shard_dot(self._h, int(vdim), _ptr(a, torch.float64, "a"), _ptr(b, torch.float64, "b"),
                                   C.byref(out), self._comm(comm), _stream(stream))
        self._check(st, comm)
        return out.value

    def solve(self, form, b, x, comm, rtol=1e-10, maxit=20000, max_outer=30, precond="jacobi", stream=None,
              raise_on_error=True):
        import torch
        o = B.SolveOpts()
        B.lib().fem_solve_opts_default(C.byref(o))
        o.rtol, o.maxit, o.max_outer = rtol, maxit, max_outer
        o.precond = {"jacobi": 0, "none": 1}[precond]
        info = B.SolveInfo()
        st = B.lib().fem_shard_solve(self._h, form._h, _ptr(b, torch.float64, "b"), _ptr(x, torch.float64, "x"),
                                     C.byref(o), C.byref(info), self._comm(comm), _stream(stream))
        out = {"status": st, "iterations": info.iterations, "outer": info.outer,
               "converged": bool(info.converged), "relres": info.relres, "bnorm": info.bnorm}
        if st != B.FEM_OK and raise_on_error:
            self._check(st, comm)
        return out

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_shard_destroy(self._h)
            self._h = None


class _SpaceView(Space):
    """The shard's local space (owned by the shard): nothing destroyed on
    collection."""

    def __del__(self):
        pass
