"""Build the sm_103a shared library `libfem.so` in-tree.

Each CUDA translation unit is compiled by nvcc for sm_103a only, host C++
by g++, in parallel, then linked with nvcc into
paper_1911_09220_gb300/libfem.so. Objects go to paper_1911_09220_gb300/_build
and are reused while newer than every source and header.

    python -m paper_1911_09220_gb300.build [--force] [--jobs N]
"""

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfem.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc):
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources():
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return [os.path.join(CSRC, s) for s in srcs], headers


def _defines():
    """Build options from the environment: FEM_NE_TABLE=large|small selects
    one candidate elements-per-block table for every element type (used to
    re-measure the choice); unset or `measured` gives the measured table.
    FEM_BATCH_MIN_BLOCKS=k compiles the batched FP32 element kernel for k
    resident 256-thread blocks per SM (its register budget). FEM_F32_TC=1
    runs the x-direction stages of the FP32 diffusion kernel (p >= 4) on the
    tensor cores (split-TF32 mma, k_tc.cuh); FEM_F32_TC=2 with single TF32
    products. FEM_F32_LANES=0 packs the short stages of the FP32 element
    kernels like the FP64 ones instead of giving each element whole warps
    (k_element.cuh, stage_lanes)."""
    t = os.environ.get("FEM_NE_TABLE", "measured")
    out = {"large": ["-DFEM_NE_TABLE=1"], "small": ["-DFEM_NE_TABLE=2"]}.get(t, [])
    mb = os.environ.get("FEM_BATCH_MIN_BLOCKS")
    if mb:
        out.append(f"-DFEM_BATCH_MIN_BLOCKS={int(mb)}")
    mb64 = os.environ.get("FEM_BATCH_MIN_BLOCKS64")
    if mb64:
        out.append(f"-DFEM_BATCH_MIN_BLOCKS64={int(mb64)}")
    if os.environ.get("FEM_F32_TC") in ("1", "2"):
        out.append(f"-DFEM_F32_TC={os.environ['FEM_F32_TC']}")
    if os.environ.get("FEM_F32_LANES") == "0":
        out.append("-DFEM_F32_LANES=0")
    return out


def _compile(src, obj, nvcc, cuda_home, verbose_ptxas):
    inc = ["-I", INCLUDE, "-I", CSRC, *_defines()]
    if src.endswith(".cu"):
        cmd = [nvcc, "-c", src, "-o", obj, "-std=c++17", "-O3", "-lineinfo", *ARCH,
               "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", *inc]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd = ["g++", "-c", src, "-o", obj, "-std=c++17", "-O2", "-fPIC", "-pthread", *inc,
               "-I", os.path.join(cuda_home, "include")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force=False, jobs=None, verbose_ptxas=False, quiet=True):
    nvcc = _nvcc()
    cuda_home = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    srcs, headers = _sources()
    hdr_mtime = max(os.path.getmtime(h) for h in headers)
    stamp = os.path.join(BUILD, "options")
    opts = " ".join(_defines())
    if not os.path.exists(stamp) or open(stamp).read() != opts:
        force = True
        with open(stamp, "w") as fh:
            fh.write(opts)
    todo = []
    objs = []
    for s in srcs:
        obj = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(obj)
        stale = (force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(s), hdr_mtime))
        if stale:
            todo.append((s, obj))
    jobs = jobs or min(len(todo) or 1, os.cpu_count() or 4)
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = [ex.submit(_compile, s, o, nvcc, cuda_home, verbose_ptxas) for s, o in todo]
            for f in futs:
                logs.append(f.result())
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        rpath = os.path.join(cuda_home, "lib64")
        cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread", "-Xlinker", "-rpath", "-Xlinker", rpath]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if not quiet:
        for l in logs:
            if l.strip():
                print(l)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--ptxas", action="store_true", help="print -Xptxas -v resource usage")
    a = ap.parse_args(argv)
    print(build(force=a.force, jobs=a.jobs, verbose_ptxas=a.ptxas, quiet=False))


if __name__ == "__main__":
    sys.exit(main())
