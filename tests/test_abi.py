"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; the Python binding declares a signature for each."""

import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fem_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1911_09220_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("fem_mesh_create", "fem_space_create", "fem_form_create", "fem_apply",
                 "fem_assemble_diagonal", "fem_solve", "fem_compliance_grad"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fem_[a-z0-9_]+)\b", out))
    missing = _declared() - exported
    assert not missing, missing


def test_binding_loads_and_declares_all(libpath):
    import paper_1911_09220_gb300 as P
    from paper_1911_09220_gb300 import _binding as B
    L = P.lib()
    for name in _declared():
        assert name in B.SIGNATURES, name
        assert hasattr(L, name)
    assert "sm_103a" in P.version()
    assert P.supported(4, 6) and P.supported(2, 4) and not P.supported(4, 9)


def test_error_path_without_gpu(libpath):
    # argument validation happens before any CUDA call
    import ctypes as C
    import paper_1911_09220_gb300 as P
    from paper_1911_09220_gb300 import _binding as B
    h = C.c_void_p()
    st = P.lib().fem_mesh_create(None, 0, None, 0, C.byref(h))
    assert st == B.FEM_EINVAL
    assert "empty mesh" in P.lib().fem_last_error().decode()


def test_solve_option_defaults(libpath):
    """fem_solve_opts_default leaves inner_rtol at 0: every solver then takes
    its mode's measured default (documented in include/fem.h); the other
    fields have their documented values."""
    import ctypes as C
    import paper_1911_09220_gb300 as P
    from paper_1911_09220_gb300 import _binding as B
    o = B.SolveOpts()
    P.lib().fem_solve_opts_default(C.byref(o))
    assert o.inner_rtol == 0.0
    assert o.rtol == 1e-10 and o.maxit == 20000 and o.max_outer == 30
    assert o.check_every == 16 and o.use_graph == 1 and o.precond == 0
    hdr = open(os.path.join(ROOT, "include", "fem.h")).read()
    for phrase in ("fem_solve 1e-4 (FEM_SOLVE_MIXED)", "(FEM_SOLVE_MIXED_RU); fem_mg_solve 3e-4",
                   "fem_batch_solve 1e-4"):
        assert phrase in " ".join(hdr.split()), phrase
