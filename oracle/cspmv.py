"""ctypes front end of oracle/spmv.c (test infrastructure only): the
oracle's assembled CSR operator applied by a plain C loop, OpenMP over rows,
for timing the CPU baseline on all host cores. `build()` compiles the
shared object next to the source (gcc -O2 -fopenmp -ffp-contract=off)."""

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmv.c")
LIB = os.path.join(HERE, "_spmv.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle spmv build failed: {' '.join(cmd)}\n{r.stderr}")
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        f = _lib.oracle_csr_spmv
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
    return _lib


class CSR:
    """A scipy CSR matrix in the C loop's index types (int64 row pointers,
    int32 column indices, float64 values)."""

    def __init__(self, K):
        self.n = K.shape[0]
        self.indptr = np.ascontiguousarray(K.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(K.indices, dtype=np.int32)
        self.data = np.ascontiguousarray(K.data, dtype=np.float64)

    def apply(self, x, threads, out=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n) if out is None else out
        st = _load().oracle_csr_spmv(self.n, self.indptr.ctypes.data, self.indices.ctypes.data,
                                     self.data.ctypes.data, x.ctypes.data, y.ctypes.data, int(threads))
        if st != 0:
            raise ValueError("oracle_csr_spmv: bad arguments")
        return y
