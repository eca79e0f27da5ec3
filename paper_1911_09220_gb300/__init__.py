"""GB300 (sm_103a) partial-assembly finite elements: Python front end.

Thin wrappers over the C ABI of libfem.so (include/fem.h). Tensors are torch
CUDA tensors (torch supplies device memory and streams); every computation
runs in the library's kernels on the current torch stream.

    mesh = Mesh(coords, hexes)                  # numpy float64 [nv,3], int32 [ne,8]
    space = Space(mesh, p)
    form = Form(space, "diffusion", q1d=p + 2, coef=kappa)   # PA setup (D)
    form.apply(x, y)                             # y = A x
    form.diagonal(d); form.rhs(fq, b); form.solve(b, x, rtol=1e-10)
    Multigrid(form, precision="f32").solve(b, x, arith="f32")   # p-multigrid FCG

Also: Mesh2D (quadrilaterals), Mesh.set_nodes (curved geometry),
Form.convection, Form.elasticity (vectors of 3 * ndof), Batch (many problems
and right-hand sides in persistent kernels), and autograd.compliance (the
compliance gradient through torch.autograd).
"""

import ctypes as C

import numpy as np

from . import _binding as B
from ._binding import (FemError, FEM_DIFFUSION, FEM_MASS, FEM_F64, FEM_F32, FEM_DF64, FEM_SOLVE_F64,
                       FEM_SOLVE_MIXED, FEM_SOLVE_DF64, FEM_SOLVE_MIXED_RU)

__all__ = ["Mesh", "Mesh2D", "Space", "Form", "Batch", "Multigrid", "FemError", "lib", "supported", "version"]


def lib():
    return B.lib()


def version():
    return B.lib().fem_version().decode()


def supported(p, q1d):
    return bool(B.lib().fem_supported(int(p), int(q1d)))


def probe_fma_peak(dtype="f64", iters=None, stream=None):
    """Measured FMA rate (TFLOP/s) of the current device in FP64 or FP32
    (fem_probe_fma_peak); about 20 ms of device time by default."""
    code = FEM_F64 if dtype == "f64" else FEM_F32
    if iters is None:
        iters = 5000 if dtype == "f64" else 300000
    out = C.c_double()
    B.check(B.lib().fem_probe_fma_peak(code, int(iters), C.byref(out), _stream(stream)))
    return out.value


def _stream(stream=None):
    """cudaStream_t of a torch.cuda.Stream, a raw handle, or the current stream."""
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return FEM_F64
    if t.dtype == torch.float32:
        return FEM_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


class Mesh:
    """Unstructured hexahedral mesh: vertex coordinates and 8-vertex tuples
    in VTK order (Sec. 3.1, conforming meshes)."""

    def __init__(self, coords, hexes):
        L = B.lib()
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.hexes = np.ascontiguousarray(hexes, dtype=np.int32)
        if self.coords.ndim != 2 or self.coords.shape[1] != 3 or self.hexes.ndim != 2 or self.hexes.shape[1] != 8:
            raise ValueError("coords must be [nv,3] and hexes [ne,8]")
        h = C.c_void_p()
        B.check(L.fem_mesh_create(self.coords.ctypes.data, self.coords.shape[0], self.hexes.ctypes.data,
                                  self.hexes.shape[0], C.byref(h)))
        self._h = h
        self.nv, self.ne = self.coords.shape[0], self.hexes.shape[0]
        self.dim = 3
        self.geo_nodes, self.geo_order = None, 0

    def set_nodes(self, nodes, k):
        """Curved geometry: element nodal coordinates [ne, (k+1)^dim, dim] at
        the order-k GLL lattice (x fastest, element's local frame); k = 0
        returns to the vertex map. Set before creating forms (or call
        set_coef)."""
        if k == 0:
            B.check(B.lib().fem_mesh_set_nodes(self._h, 0, None))
            self.geo_nodes, self.geo_order = None, 0
            return
        n = np.ascontiguousarray(nodes, dtype=np.float64)
        d = self.dim
        if n.shape != (self.ne, (k + 1) ** d, d):
            raise ValueError(f"nodes must be [{self.ne}, {(k + 1) ** d}, {d}]")
        B.check(B.lib().fem_mesh_set_nodes(self._h, int(k), n.ctypes.data))
        self.geo_nodes, self.geo_order = n, int(k)

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_mesh_destroy(self._h)
            self._h = None


class Mesh2D(Mesh):
    """Unstructured quadrilateral mesh: vertex coordinates [nv,2] and 4-vertex
    tuples, counter-clockwise from the local (0,0) corner (Sec. 3.1, d = 2)."""

    def __init__(self, coords, quads):
        L = B.lib()
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.hexes = np.ascontiguousarray(quads, dtype=np.int32)
        if self.coords.ndim != 2 or self.coords.shape[1] != 2 or self.hexes.ndim != 2 or self.hexes.shape[1] != 4:
            raise ValueError("coords must be [nv,2] and quads [ne,4]")
        h = C.c_void_p()
        B.check(L.fem_mesh2d_create(self.coords.ctypes.data, self.coords.shape[0], self.hexes.ctypes.data,
                                    self.hexes.shape[0], C.byref(h)))
        self._h = h
        self.nv, self.ne = self.coords.shape[0], self.hexes.shape[0]
        self.dim = 2


class Space:
    """H1 space of order p (GLL nodal basis) with the global numbering of
    Sec. 3.4 and the element restriction G and its inverse."""

    def __init__(self, mesh, p):
        L = B.lib()
        self.mesh = mesh
        h = C.c_void_p()
        B.check(L.fem_space_create(mesh._h, int(p), C.byref(h)))
        self._h = h
        ndof, nbdr, ne = C.c_int64(), C.c_int64(), C.c_int64()
        pp = C.c_int()
        B.check(L.fem_space_info(h, C.byref(ndof), C.byref(nbdr), C.byref(ne), C.byref(pp)))
        self.ndof, self.nbdr, self.ne, self.p = ndof.value, nbdr.value, ne.value, pp.value
        self.dim = mesh.dim

    def boundary_dofs(self):
        out = np.empty(self.nbdr, dtype=np.int32)
        B.check(B.lib().fem_space_boundary_dofs(self._h, out.ctypes.data))
        return out

    def element_dofs(self):
        out = np.empty((self.ne, (self.p + 1) ** self.dim), dtype=np.int32)
        B.check(B.lib().fem_space_element_dofs(self._h, out.ctypes.data))
        return out

    def dof_coords(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.ndof, self.dim), dtype=torch.float64, device="cuda")
        B.check(B.lib().fem_space_dof_coords(self._h, _ptr(out, torch.float64, "out"), _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_space_destroy(self._h)
            self._h = None


class Form:
    """Partially assembled mass or diffusion form (Sec. 4.3-4.4): setup stores
    D at the quadrature points; apply runs G, B, D, B^T, G^T on the fly."""

    vdim = 1

    def __init__(self, space, kind="diffusion", q1d=None, coef=None, stream=None):
        import torch
        L = B.lib()
        self.space = space
        self.kind = {"diffusion": FEM_DIFFUSION, "mass": FEM_MASS}[kind] if isinstance(kind, str) else int(kind)
        self.q1d = int(q1d) if q1d is not None else space.p + 2
        self.nq = self.q1d ** space.dim
        self._coef = None if coef is None else coef.contiguous()
        h = C.c_void_p()
        B.check(L.fem_form_create(space._h, self.kind, self.q1d, _ptr(self._coef, torch.float64, "coef"),
                                  _stream(stream), C.byref(h)))
        self._h = h
        self.ess = None
        self.vdim = 1

    @property
    def n(self):
        """Length of the form's vectors: vdim * ndof (component-major)."""
        return self.vdim * self.space.ndof

    @classmethod
    def elasticity(cls, space, lam, mu, q1d=None, stream=None):
        """Linear elasticity lambda (div u)(div v) + 2 mu eps(u):eps(v) on the
        three-component vector space: lam, mu device float64 [ne]. Vectors
        hold 3 * ndof entries, component c of DOF i at c * ndof + i."""
        import torch
        L = B.lib()
        self = cls.__new__(cls)
        self.space = space
        self.kind = B.FEM_ELASTICITY
        self.q1d = int(q1d) if q1d is not None else space.p + 2
        self.nq = self.q1d ** space.dim
        self._coef = None
        self._lam, self._mu = lam.contiguous(), mu.contiguous()
        h = C.c_void_p()
        B.check(L.fem_form_create_elasticity(space._h, self.q1d, _ptr(self._lam, torch.float64, "lam"),
                                             _ptr(self._mu, torch.float64, "mu"), _stream(stream), C.byref(h)))
        self._h = h
        self.ess = None
        self.vdim = 3
        return self

    def set_lame(self, lam, mu, stream=None):
        import torch
        self._lam, self._mu = lam.contiguous(), mu.contiguous()
        B.check(B.lib().fem_form_set_lame(self._h, _ptr(self._lam, torch.float64, "lam"),
                                          _ptr(self._mu, torch.float64, "mu"), _stream(stream)))

    @classmethod
    def convection(cls, space, beta, q1d=None, coef=None, stream=None):
        """Convection form (beta . grad u, v): beta [ne, q1d^3, 3] (device
        float64), the physical velocity at the form's quadrature points."""
        import torch
        L = B.lib()
        self = cls.__new__(cls)
        self.space = space
        self.kind = B.FEM_CONVECTION
        self.q1d = int(q1d) if q1d is not None else space.p + 2
        self.nq = self.q1d ** space.dim
        self._coef = None if coef is None else coef.contiguous()
        self._beta = beta.contiguous()
        if tuple(self._beta.shape) != (space.ne, self.nq, 3):
            raise ValueError(f"beta must be [{space.ne}, {self.nq}, 3]")
        h = C.c_void_p()
        B.check(L.fem_form_create_convection(space._h, self.q1d, _ptr(self._beta, torch.float64, "beta"),
                                             _ptr(self._coef, torch.float64, "coef"), _stream(stream), C.byref(h)))
        self._h = h
        self.ess = None
        self.vdim = 1
        return self

    def set_velocity(self, beta, stream=None):
        import torch
        self._beta = beta.contiguous()
        B.check(B.lib().fem_form_set_velocity(self._h, _ptr(self._beta, torch.float64, "beta"), _stream(stream)))

    # ---- configuration
    def set_coef(self, coef, stream=None):
        import torch
        self._coef = coef.contiguous()
        B.check(B.lib().fem_form_set_coef(self._h, _ptr(self._coef, torch.float64, "coef"), _stream(stream)))

    def set_essential(self, ess, stream=None):
        import torch
        if not isinstance(ess, torch.Tensor):
            ess = torch.as_tensor(np.asarray(ess, dtype=np.int32), device="cuda")
        self.ess = ess.to(torch.int32).contiguous()
        B.check(B.lib().fem_form_set_essential(self._h, _ptr(self.ess, torch.int32, "ess") if self.ess.numel() else None,
                                               self.ess.numel(), _stream(stream)))

    # ---- operator
    @staticmethod
    def _code(x, arith):
        if arith is None:
            return _dtype_code(x)
        if arith == "df64":
            import torch
            if x.dtype != torch.float64:
                raise TypeError("arith='df64' takes float64 vectors")
            return FEM_DF64
        raise ValueError(f"unknown arith {arith!r}")

    def apply(self, x, y, constrained=False, stream=None, arith=None):
        """y = A x. arith=None computes in the tensors' dtype; arith='df64'
        takes float64 vectors and computes in double-float."""
        if x.dtype != y.dtype:
            raise TypeError("x and y must have the same dtype")
        B.check(B.lib().fem_apply(self._h, self._code(x, arith), _ptr(x, name="x"), _ptr(y, name="y"),
                                  int(bool(constrained)), _stream(stream)))
        return y

    def apply_element(self, x, ye, stream=None, arith=None):
        B.check(B.lib().fem_apply_element(self._h, self._code(x, arith), _ptr(x, name="x"),
                                          _ptr(ye, x.dtype, "ye"), _stream(stream)))
        return ye

    def scatter(self, ye, y, stream=None):
        B.check(B.lib().fem_scatter(self._h, _dtype_code(ye), _ptr(ye, name="ye"), _ptr(y, ye.dtype, "y"),
                                    _stream(stream)))
        return y

    def diagonal(self, out, constrained=False, stream=None):
        import torch
        B.check(B.lib().fem_assemble_diagonal(self._h, _ptr(out, torch.float64, "out"), int(bool(constrained)),
                                              _stream(stream)))
        return out

    def rhs(self, fq, b, stream=None):
        import torch
        B.check(B.lib().fem_rhs(self._h, _ptr(fq, torch.float64, "fq"), _ptr(b, torch.float64, "b"), _stream(stream)))
        return b

    def qpoint_coords(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.space.ne, self.nq, self.space.dim), dtype=torch.float64, device="cuda")
        B.check(B.lib().fem_qpoint_coords(self._h, _ptr(out, torch.float64, "out"), _stream(stream)))
        return out

    def lift_rhs(self, b, g, bc, stream=None):
        import torch
        B.check(B.lib().fem_lift_rhs(self._h, _ptr(b, torch.float64, "b"), _ptr(g, torch.float64, "g"),
                                     _ptr(bc, torch.float64, "bc"), _stream(stream)))
        return bc

    def solve(self, b, x, rtol=1e-10, maxit=20000, precision="f64", inner_rtol=None, max_outer=30,
              check_every=16, use_graph=True, stream=None, raise_on_error=True, precond="jacobi"):
        """Jacobi-PCG on the constrained operator. precision: "f64", "df64"
        (FP64 CG, double-float operator), "mixed" (FP32 inner CG restarted in
        FP64 refinement; inner_rtol default 1e-4) or "mixed_ru" (FP32 CG with
        FP64 reliable updates; inner_rtol = residual drop between updates,
        default 0.1). None takes the library's measured default.
        precond: "jacobi" or "none" (plain CG)."""
        import torch
        o = B.SolveOpts()
        B.lib().fem_solve_opts_default(C.byref(o))
        o.rtol, o.maxit, o.inner_rtol, o.max_outer = rtol, maxit, inner_rtol or 0.0, max_outer
        o.precision = {"f64": FEM_SOLVE_F64, "mixed": FEM_SOLVE_MIXED, "df64": FEM_SOLVE_DF64,
                       "mixed_ru": FEM_SOLVE_MIXED_RU}[precision]
        o.check_every, o.use_graph = check_every, int(bool(use_graph))
        o.precond = {"jacobi": 0, "none": 1}[precond]
        info = B.SolveInfo()
        st = B.lib().fem_solve(self._h, _ptr(b, torch.float64, "b"), _ptr(x, torch.float64, "x"), C.byref(o),
                               C.byref(info), _stream(stream))
        out = {"status": st, "iterations": info.iterations, "outer": info.outer,
               "converged": bool(info.converged), "relres": info.relres, "bnorm": info.bnorm}
        if st != B.FEM_OK and raise_on_error:
            raise FemError(st, B.lib().fem_last_error().decode())
        return out

    def compliance_grad(self, u, g, stream=None):
        import torch
        B.check(B.lib().fem_compliance_grad(self._h, _ptr(u, torch.float64, "u"), _ptr(g, torch.float64, "g"),
                                            _stream(stream)))
        return g

    def compliance(self, b, u, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=b.device)
        B.check(B.lib().fem_compliance(self._h, _ptr(b, torch.float64, "b"), _ptr(u, torch.float64, "u"),
                                       _ptr(out, torch.float64, "out"), _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_form_destroy(self._h)
            self._h = None


class Batch:
    """Many independent problems (forms) with nrhs right-hand sides each.
    Batched vectors are concatenated problem after problem; problem i's block
    is [nrhs][ndof_i] starting at nrhs * off[i] (see include/fem.h)."""

    def __init__(self, forms, nrhs, stream=None):
        L = B.lib()
        self.forms = list(forms)
        self.nrhs = int(nrhs)
        arr = (C.c_void_p * len(self.forms))(*[f._h.value for f in self.forms])
        h = C.c_void_p()
        B.check(L.fem_batch_create(arr, len(self.forms), self.nrhs, _stream(stream), C.byref(h)))
        self._h = h
        tot = C.c_int64()
        off = np.zeros(len(self.forms) + 1, dtype=np.int64)
        B.check(L.fem_batch_info(h, C.byref(tot), off.ctypes.data))
        self.total_len, self.off = tot.value, off
        self.nsys = len(self.forms) * self.nrhs

    def block(self, V, i, r):
        """View of problem i, right-hand side r inside a batched vector."""
        n = int(self.off[i + 1] - self.off[i])
        s0 = self.nrhs * int(self.off[i]) + r * n
        return V[s0:s0 + n]

    def apply(self, X, Y, constrained=False, stream=None):
        if X.dtype != Y.dtype:
            raise TypeError("X and Y must have the same dtype")
        B.check(B.lib().fem_batch_apply(self._h, _dtype_code(X), _ptr(X, name="X"), _ptr(Y, name="Y"),
                                        int(bool(constrained)), _stream(stream)))
        return Y

    def solve(self, Bv, X, rtol=1e-10, maxit=20000, precision="f64", inner_rtol=None, max_outer=30,
              check_every=16, use_graph=True, stream=None, raise_on_error=True):
        import torch
        o = B.SolveOpts()
        B.lib().fem_solve_opts_default(C.byref(o))
        o.rtol, o.maxit, o.inner_rtol, o.max_outer = rtol, maxit, inner_rtol or 0.0, max_outer
        o.precision = FEM_SOLVE_MIXED if precision == "mixed" else FEM_SOLVE_F64
        o.check_every, o.use_graph = check_every, int(bool(use_graph))
        iters = np.zeros(self.nsys, dtype=np.int32)
        rel = np.zeros(self.nsys, dtype=np.float64)
        st = B.lib().fem_batch_solve(self._h, _ptr(Bv, torch.float64, "B"), _ptr(X, torch.float64, "X"), C.byref(o),
                                     iters.ctypes.data, rel.ctypes.data, _stream(stream))
        if st != B.FEM_OK and raise_on_error:
            raise FemError(st, B.lib().fem_last_error().decode())
        return {"status": st, "iterations": iters, "relres": rel}

    def tune(self, dtype="f64", cache_path=None, stream=None):
        code = FEM_F64 if dtype == "f64" else FEM_F32
        path = None if cache_path is None else str(cache_path).encode()
        B.check(B.lib().fem_batch_tune(self._h, code, path, _stream(stream)))
        return self.tiles()

    def tiles(self):
        t = np.zeros(18, dtype=np.int32)
        B.check(B.lib().fem_batch_tiles(self._h, t.ctypes.data))
        return t

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_batch_destroy(self._h)
            self._h = None


class Multigrid:
    """p-multigrid preconditioner of a form (levels p, p/2, ..., 1; Chebyshev-
    Jacobi smoothing; coarsest level by Jacobi-PCG) and flexible CG with it.
    precision: "f64" or "f32" (arithmetic of the V-cycle; the outer iteration
    is FP64). set_essential must have been called on the form. Elasticity
    forms get a vector hierarchy (vectors of length 3 ndof on every level)."""

    def __init__(self, form, cheb_order=2, cheb_lo=0.25, cheb_hi=1.1, power_its=20, coarse_its=30,
                 precision="f64", stream=None, coarse_assembled=True):
        L = B.lib()
        self.form = form
        o = B.MgOpts()
        L.fem_mg_opts_default(C.byref(o))
        o.cheb_order, o.cheb_lo, o.cheb_hi = int(cheb_order), float(cheb_lo), float(cheb_hi)
        o.power_its, o.coarse_its = int(power_its), int(coarse_its)
        o.coarse_assembled = int(bool(coarse_assembled))
        o.precision = {"f64": FEM_F64, "f32": FEM_F32}[precision]
        h = C.c_void_p()
        B.check(L.fem_mg_create(form._h, C.byref(o), _stream(stream), C.byref(h)))
        self._h = h

    def info(self):
        n = C.c_int()
        B.check(B.lib().fem_mg_info(self._h, C.byref(n), None, None, None))
        orders = np.zeros(n.value, dtype=np.int32)
        lams = np.zeros(n.value, dtype=np.float64)
        ndofs = np.zeros(n.value, dtype=np.int64)
        B.check(B.lib().fem_mg_info(self._h, None, orders.ctypes.data, lams.ctypes.data, ndofs.ctypes.data))
        return {"orders": orders.tolist(), "lambdas": lams.tolist(), "ndofs": ndofs.tolist()}

    def level_form(self, level):
        """A non-owning view of level `level`'s form (apply, diagonal, ...)."""
        h = B.lib().fem_mg_level_form(self._h, int(level))
        if not h:
            raise IndexError(level)
        v = Form.__new__(_FormView)
        v._h, v._owner, v.space, v.ess = C.c_void_p(h), self, None, None
        v.vdim = self.form.vdim
        return v

    def prolong(self, level, zc, zf, stream=None):
        import torch
        B.check(B.lib().fem_mg_prolong(self._h, int(level), _ptr(zc, torch.float64, "zc"), _ptr(zf, torch.float64, "zf"),
                                       _stream(stream)))
        return zf

    def restrict(self, level, rf, rc, stream=None):
        import torch
        B.check(B.lib().fem_mg_restrict(self._h, int(level), _ptr(rf, torch.float64, "rf"),
                                        _ptr(rc, torch.float64, "rc"), _stream(stream)))
        return rc

    def vcycle(self, r, z, stream=None):
        import torch
        B.check(B.lib().fem_mg_vcycle(self._h, _ptr(r, torch.float64, "r"), _ptr(z, torch.float64, "z"),
                                      _stream(stream)))
        return z

    def solve(self, b, x, rtol=1e-10, maxit=500, max_outer=30, check_every=4, use_graph=True, stream=None,
              raise_on_error=True, arith="f64", inner_rtol=None):
        """Flexible CG with one V-cycle per iteration. arith, the outer
        operator apply: "f64", "df64" (double-float), or "f32" (FP32 operator
        inside FP64 iterative refinement: each pass reduces the residual by
        inner_rtol, then restarts from the FP64 true residual)."""
        import torch
        o = B.SolveOpts()
        B.lib().fem_solve_opts_default(C.byref(o))
        o.rtol, o.maxit, o.max_outer = rtol, maxit, max_outer
        if arith not in ("f64", "df64", "f32"):
            raise ValueError(f"arith must be 'f64', 'df64' or 'f32', not {arith!r}")
        o.precision = {"f64": FEM_SOLVE_F64, "df64": FEM_SOLVE_DF64, "f32": FEM_SOLVE_MIXED}[arith]
        o.inner_rtol = inner_rtol or 0.0
        o.check_every, o.use_graph = check_every, int(bool(use_graph))
        info = B.SolveInfo()
        st = B.lib().fem_mg_solve(self._h, _ptr(b, torch.float64, "b"), _ptr(x, torch.float64, "x"), C.byref(o),
                                  C.byref(info), _stream(stream))
        out = {"status": st, "iterations": info.iterations, "outer": info.outer,
               "converged": bool(info.converged), "relres": info.relres, "bnorm": info.bnorm}
        if st != B.FEM_OK and raise_on_error:
            raise FemError(st, B.lib().fem_last_error().decode())
        return out

    def __del__(self):
        if getattr(self, "_h", None) and B._lib is not None:
            B._lib.fem_mg_destroy(self._h)
            self._h = None


class _FormView(Form):
    """A form owned by another handle (a multigrid level): same methods,
    nothing destroyed on collection."""

    def __del__(self):
        pass
