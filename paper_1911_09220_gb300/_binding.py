"""ctypes binding of libfem.so (the C ABI declared in include/fem.h).

Argument marshalling only: every computation runs in the library's sm_103a
kernels. The library must have been built (paper_1911_09220_gb300.build);
loading fails loudly otherwise, there is no fallback.
"""

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfem.so")

FEM_OK, FEM_EINVAL, FEM_ENOMEM, FEM_EINVERTED, FEM_ENOCONV, FEM_EBREAKDOWN, FEM_ECUDA, FEM_EUNSUPPORTED = range(8)
FEM_MASS, FEM_DIFFUSION, FEM_CONVECTION, FEM_ELASTICITY = 0, 1, 2, 3
FEM_F64, FEM_F32, FEM_DF64 = 0, 1, 2
FEM_SOLVE_F64, FEM_SOLVE_MIXED, FEM_SOLVE_DF64, FEM_SOLVE_MIXED_RU = 0, 1, 2, 3

STATUS_NAMES = {
    0: "FEM_OK", 1: "FEM_EINVAL", 2: "FEM_ENOMEM", 3: "FEM_EINVERTED", 4: "FEM_ENOCONV",
    5: "FEM_EBREAKDOWN", 6: "FEM_ECUDA", 7: "FEM_EUNSUPPORTED",
}


class FemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int), ("check_every", C.c_int),
                ("use_graph", C.c_int), ("precond", C.c_int)]


class MgOpts(C.Structure):
    _fields_ = [("cheb_order", C.c_int), ("cheb_lo", C.c_double), ("cheb_hi", C.c_double), ("power_its", C.c_int),
                ("coarse_its", C.c_int), ("precision", C.c_int), ("coarse_assembled", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("converged", C.c_int),
                ("relres", C.c_double), ("bnorm", C.c_double)]


P = C.c_void_p
I64 = C.c_int64
I = C.c_int

# name -> (restype, argtypes); every entry point declared in include/fem.h
SIGNATURES = {
    "fem_version": (C.c_char_p, []),
    "fem_last_error": (C.c_char_p, []),
    "fem_supported": (I, [I, I]),
    "fem_mesh_create": (I, [P, I64, P, I64, C.POINTER(P)]),
    "fem_mesh2d_create": (I, [P, I64, P, I64, C.POINTER(P)]),
    "fem_mesh_set_nodes": (I, [P, I, P]),
    "fem_mesh_destroy": (None, [P]),
    "fem_space_create": (I, [P, I, C.POINTER(P)]),
    "fem_space_destroy": (None, [P]),
    "fem_space_info": (I, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I)]),
    "fem_space_boundary_dofs": (I, [P, P]),
    "fem_space_element_dofs": (I, [P, P]),
    "fem_space_dof_coords": (I, [P, P, P]),
    "fem_form_create": (I, [P, I, I, P, P, C.POINTER(P)]),
    "fem_form_create_convection": (I, [P, I, P, P, P, C.POINTER(P)]),
    "fem_form_set_velocity": (I, [P, P, P]),
    "fem_form_create_elasticity": (I, [P, I, P, P, P, C.POINTER(P)]),
    "fem_form_set_lame": (I, [P, P, P, P]),
    "fem_form_destroy": (None, [P]),
    "fem_form_set_coef": (I, [P, P, P]),
    "fem_form_set_essential": (I, [P, P, I64, P]),
    "fem_apply": (I, [P, I, P, P, I, P]),
    "fem_apply_element": (I, [P, I, P, P, P]),
    "fem_scatter": (I, [P, I, P, P, P]),
    "fem_apply_noalloc": (I, [P, P, P, P]),
    "fem_assemble_diagonal": (I, [P, P, I, P]),
    "fem_rhs": (I, [P, P, P, P]),
    "fem_qpoint_coords": (I, [P, P, P]),
    "fem_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
    "fem_solve": (I, [P, P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P]),
    "fem_lift_rhs": (I, [P, P, P, P, P]),
    "fem_compliance_grad": (I, [P, P, P, P]),
    "fem_compliance": (I, [P, P, P, P, P]),
    "fem_batch_create": (I, [P, I, I, P, C.POINTER(P)]),
    "fem_batch_destroy": (None, [P]),
    "fem_batch_info": (I, [P, C.POINTER(I64), P]),
    "fem_batch_apply": (I, [P, I, P, P, I, P]),
    "fem_batch_solve": (I, [P, P, P, C.POINTER(SolveOpts), P, P, P]),
    "fem_batch_tune": (I, [P, I, C.c_char_p, P]),
    "fem_batch_tiles": (I, [P, P]),
    "fem_mg_opts_default": (None, [C.POINTER(MgOpts)]),
    "fem_mg_create": (I, [P, C.POINTER(MgOpts), P, C.POINTER(P)]),
    "fem_mg_destroy": (None, [P]),
    "fem_mg_info": (I, [P, P, P, P, P]),
    "fem_mg_vcycle": (I, [P, P, P, P]),
    "fem_mg_level_form": (P, [P, I]),
    "fem_mg_prolong": (I, [P, I, P, P, P]),
    "fem_mg_restrict": (I, [P, I, P, P, P]),
    "fem_mg_solve": (I, [P, P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P]),
    "fem_partition_slabs": (I, [P, I, P]),
    "fem_shard_create": (I, [P, P, I, I, C.POINTER(P)]),
    "fem_shard_destroy": (None, [P]),
    "fem_shard_space": (P, [P]),
    "fem_shard_info": (I, [P, P, P, P, P, P, P]),
    "fem_shard_tables": (I, [P, P, P, P, P, P, P]),
    "fem_shard_combine_table": (I, [P, P, P, P, P, P]),
    "fem_shard_localize": (I, [P, P, I64, P]),
    "fem_shard_to_local": (I, [P, I, P, P, P]),
    "fem_shard_to_global": (I, [P, I, P, P, P]),
    "fem_shard_apply": (I, [P, P, P, P, I, P, P]),
    "fem_shard_diagonal": (I, [P, P, P, I, P, P]),
    "fem_shard_rhs": (I, [P, P, P, P, P, P]),
    "fem_shard_dot": (I, [P, I, P, P, P, P, P]),
    "fem_shard_solve": (I, [P, P, P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P, P]),
    "fem_probe_fma_peak": (I, [I, I, C.POINTER(C.c_double), P]),
}

_lib = None


def lib():
    """Load libfem.so once and declare every entry point's signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1911_09220_gb300.build` "
                "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH, mode=C.RTLD_GLOBAL)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != FEM_OK:
        raise FemError(status, lib().fem_last_error().decode())
    return status
