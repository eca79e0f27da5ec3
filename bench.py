"""Benchmark: FP64 partial-assembly diffusion apply (GDOF/s) and Jacobi-PCG
time to 1e-10 relative residual, FP64 vs FP32-inner iterative refinement.

Workload (one GPU): unit-cube hexahedral mesh N^3 (N = 68), vertices
perturbed by U[-0.15h, 0.15h] (tangentially on the boundary), order p = 4,
q = 6 Gauss points per direction, per-element lognormal kappa, 20,346,417
DOFs, x ~ U[-1, 1]. One step = one operator application y = A x (element
kernel + inverse-map scatter, through fem_apply). Inputs (D = 3.26 GB) are
far larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) the default is the sharded operator: one problem
partitioned into element slabs, one per rank, with a halo exchange over
NCCL after every apply (`--scaling weak`: about N^3 elements per rank;
`--scaling strong`: the N^3 problem split over the ranks); `value` is the
global DOFs over the slowest rank's apply time. `--parallel replicas` runs
one independent problem per rank instead (seed offset by rank; no
collective in the data path; aggregate DOFs/s).
The reference arm (`--impl reference`) times the CPU oracle (assembled CSR
SpMV, scipy, one core) on a bounded sample of the same workload.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_element_kernel.txt")
# FP64 FMA rate of a GB300 SM: 2 DFMA per clock per SM (derived from the
# nominal 1.25 TFLOP/s; a DFMA microbenchmark on the box measured 1.19 TFLOP/s
# at ~1.96 GHz). Peak = 152 SMs x 2 DFMA x 2 flop x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def alg_counts(p, q, E, n, kind="diffusion", fp=8, dim=3):
    """Algorithmic flops and bytes of one apply (stream D once, read the map
    once, read x and write y once)."""
    D1, Q = p + 1, q
    if dim == 2:
        if kind == "diffusion":
            flops_e = 2 * (4 * Q * D1 ** 2 + 4 * Q ** 2 * D1) + 6 * Q ** 2
            bytes_ = 3 * fp * Q ** 2 * E + 4 * D1 ** 2 * E + 2 * fp * n
        else:
            flops_e = 2 * (2 * Q * D1 ** 2 + 2 * Q ** 2 * D1) + Q ** 2
            bytes_ = fp * Q ** 2 * E + 4 * D1 ** 2 * E + 2 * fp * n
        return flops_e * E, bytes_
    if kind == "diffusion":
        flops_e = 2 * (4 * Q * D1 ** 3 + 6 * Q ** 2 * D1 ** 2 + 6 * Q ** 3 * D1) + 15 * Q ** 3
        bytes_ = 6 * fp * Q ** 3 * E + 4 * D1 ** 3 * E + 2 * fp * n
    else:
        flops_e = 4 * (Q * D1 ** 3 + Q ** 2 * D1 ** 2 + Q ** 3 * D1) + Q ** 3
        bytes_ = fp * Q ** 3 * E + 4 * D1 ** 3 * E + 2 * fp * n
    return flops_e * E, bytes_


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("k_apply_kernels.cuh", "k_common.cuh", "k_element.cuh", "k_tables.cuh", "k_df64.cuh", "k_tc.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1911_09220_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload_key):
    """dram bytes per launch of the element kernel from a committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    ent = t.get(workload_key)
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def time_events(fn, steps, warmup):
    """Average device time (ms) of fn() over `steps` calls after `warmup`
    calls, with CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def reduce_max(value, device=None):
    """Max of a per-rank float over all ranks (identity without a process
    group): the slowest rank's time sets the whole job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if dist.get_backend() != "nccl":
        device = None
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed_offset(rank):
    """Each rank applies the operator of its own independent problem."""
    return 1000 * int(rank)


def make_problem(p, N, seed_offset=0):
    from fem_inputs import hex_lattice, lognormal, x_uniform
    c, h = hex_lattice(N, 0.15, seed=10 + p + seed_offset)
    kappa = lognormal(20 + p + seed_offset, h.shape[0])
    return c, h, kappa, (lambda n: x_uniform(30 + p + seed_offset, n))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


_ORACLE_SAMPLES = {}


def cpu_oracle_problem(p, N_sample):
    """The oracle's assembled sub-problem of the same recipe (cached: the
    SpMV and PCG baselines share one assembly). Returns (problem, K,
    assembly seconds, x generator)."""
    key = (p, N_sample)
    if key not in _ORACLE_SAMPLES:
        from oracle import assemble
        c, h, kappa, xgen = make_problem(p, N_sample)
        t0 = time.perf_counter()
        prob = assemble.Problem(c, h, p, p + 2, kappa=kappa)
        K = prob.K
        _ORACLE_SAMPLES[key] = (prob, K, time.perf_counter() - t0, xgen)
    return _ORACLE_SAMPLES[key]


def cpu_oracle_spmv(p, N_sample, reps, deadline_s=30.0):
    """Time the oracle's apply (its assembled CSR matrix) on a sub-problem of
    the same recipe: scipy's product on one thread, and the oracle's C loop
    (OpenMP over rows) on every host core. Returns dict; `gdofs`, `times`
    and `cores` are the all-cores figures."""
    from oracle import cspmv
    prob, K, t_asm, xgen = cpu_oracle_problem(p, N_sample)
    h = prob.hexes
    x = xgen(prob.ndof)

    def timed(fn, budget):
        fn()
        ts = []
        t_start = time.perf_counter()
        for _ in range(reps):
            t1 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t1)
            if time.perf_counter() - t_start > budget:
                break
        return ts

    t1core = timed(lambda: K @ x, deadline_s / 2)
    A = cspmv.CSR(K)
    cores = host_cores()
    y = np.empty(prob.ndof)
    tall = timed(lambda: A.apply(x, cores, out=y), deadline_s / 2)
    t = statistics.median(tall)
    return {"ndof": prob.ndof, "E": h.shape[0], "t_spmv": t, "t_assembly": t_asm, "nnz": K.nnz,
            "gdofs": prob.ndof / t / 1e9, "reps": len(tall), "times": tall, "cores": cores,
            "single_core": {"gdofs": prob.ndof / statistics.median(t1core) / 1e9,
                            "t_spmv": statistics.median(t1core), "reps": len(t1core),
                            "kind": "scipy CSR product, one thread"}}


class _ThreadedCSR:
    """The oracle's assembled matrix with its product on `threads` host cores
    (the oracle's C loop): what the oracle's PCG multiplies by."""

    def __init__(self, K, threads):
        from oracle import cspmv
        self.K, self.C, self.threads, self.shape = K, cspmv.CSR(K), int(threads), K.shape

    def __matmul__(self, x):
        return self.C.apply(x, self.threads)

    def diagonal(self):
        return self.K.diagonal()


def cpu_oracle_pcg(p, N_sample, iters_full=None, ndof_full=None, one_core_iters=20):
    """The oracle's Jacobi-PCG to the 1e-10 true residual on a sub-problem of
    the same recipe (sin sin sin source, homogeneous Dirichlet boundary):
    all host cores for the C product, then `one_core_iters` iterations on one
    core (time per iteration). With iters_full / ndof_full, the all-cores and
    one-core solve times are extrapolated to the full problem as time per
    iteration per DOF x DOFs x iterations (labelled as extrapolated)."""
    from oracle import solve as osolve
    prob, K, t_asm0, _ = cpu_oracle_problem(p, N_sample)
    h = prob.hexes
    t0 = time.perf_counter()
    ess = prob.num["boundary_dofs"]
    f = lambda x: 3 * np.pi ** 2 * np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.sin(np.pi * x[..., 2])
    Ac = osolve.constrain(K, ess)
    bc = osolve.constrain_rhs(K, prob.load(f), ess)
    t_asm = t_asm0 + time.perf_counter() - t0
    cores = host_cores()
    A_all = _ThreadedCSR(Ac, cores)
    t0 = time.perf_counter()
    _, info = osolve.pcg(A_all, bc, rtol=1e-10, maxit=20000)
    t_all = time.perf_counter() - t0
    A_one = _ThreadedCSR(Ac, 1)
    t0 = time.perf_counter()
    osolve.pcg(A_one, bc, rtol=1e-30, maxit=one_core_iters)
    t_one_it = (time.perf_counter() - t0) / one_core_iters
    n, its = prob.ndof, info["iterations"]
    out = {"ndof": n, "elements": int(h.shape[0]), "iterations": its, "converged": bool(info["converged"]),
           "true_relres": float(info["true_relres"]), "solve_s": t_all, "cores": cores,
           "one_core_s_per_iteration": t_one_it, "one_core_solve_s_est": t_one_it * its,
           "assembly_s": t_asm, "kind": "oracle Jacobi-PCG (Saad Alg. 9.1), assembled CSR, C product"}
    if iters_full and ndof_full:
        scale = (ndof_full / n) * (iters_full / max(its, 1))
        out["extrapolated"] = {"ndof": ndof_full, "iterations": iters_full, "solve_s_all_cores": t_all * scale,
                               "solve_s_one_core": t_one_it * its * scale,
                               "how": "sample time per iteration per DOF x full DOFs x the full problem's "
                                      "iteration count (measured by the GPU FP64 solve)"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = args.p
    r = cpu_oracle_spmv(p, args.cpu_n, max(args.steps, 1), deadline_s=60.0)
    total = sum(r["times"][: args.steps]) if len(r["times"]) >= args.steps else sum(r["times"])
    pcg = None if args.no_solve else cpu_oracle_pcg(p, args.cpu_n, iters_full=FP64_PCG_ITERS.get((p, args.N)),
                                                    ndof_full=(p * args.N + 1) ** 3)
    value = r["gdofs"]
    line = {
        "impl": "reference", "metric": "PA diffusion apply GDOF/s", "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": len(r["times"]), "warmup": 1, "ms_per_step": r["t_spmv"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 diffusion y=Ax, p={p}, q={p + 2}, {args.cpu_n}^3 perturbed hex sample "
                               f"({r['ndof']} DOFs) of the N={args.N} workload", "p": p, "q1d": p + 2,
                   "ndof": r["ndof"]},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": r["cores"], "kind": "oracle",
                         "sample": f"the oracle's assembled CSR matrix applied by its C loop (OpenMP over rows, "
                                   f"{r['cores']} threads), {r['ndof']} DOFs (nnz {r['nnz']}), median of "
                                   f"{len(r['times'])}; assembly {r['t_assembly']:.1f} s untimed",
                         "single_core": r["single_core"], "pcg": pcg},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "total_s": total,
    }
    print(json.dumps(line))
    return 0


# FP64 Jacobi-PCG iterations of the GPU solve at full size (p, N), for the
# per-DOF extrapolation of the CPU oracle's solve time
FP64_PCG_ITERS = {(4, 68): 1870, (6, 45): 2256}

SWEEP_N = {"1e6": {1: 99, 2: 49, 3: 33, 4: 25, 5: 20, 6: 16, 7: 14, 8: 12},
           "4e6": {1: 158, 2: 79, 3: 53, 4: 39, 5: 32, 6: 26, 7: 23, 8: 20},
           "2e7": {1: 270, 2: 135, 3: 90, 4: 68, 5: 54, 6: 45, 7: 39, 8: 34},
           "3e7": {1: 310, 2: 155, 3: 103, 4: 77, 5: 62, 6: 52, 7: 44, 8: 39}}


def _sin_rhs(form, b):
    import torch
    xq = form.qpoint_coords()
    fq = (3 * np.pi ** 2 * torch.sin(np.pi * xq[..., 0]) * torch.sin(np.pi * xq[..., 1])
          * torch.sin(np.pi * xq[..., 2])).contiguous()
    del xq
    form.rhs(fq, b)


def run_sweep(args):
    """One JSON line per order p: FP64/FP32 mass and diffusion applies, setup,
    diagonal, load vector and FP64 / mixed Jacobi-PCG to 1e-10."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    orders = [int(v) for v in args.orders.split(",")]
    for p in orders:
        N = SWEEP_N[args.sweep_size][p]
        q = p + 2
        c, h, kappa, xgen = make_problem(p, N)
        t0 = time.perf_counter()
        space = F.Space(F.Mesh(c, h), p)
        t_space = time.perf_counter() - t0
        n, E = space.ndof, space.ne
        kap = torch.as_tensor(kappa, device="cuda")
        x = torch.as_tensor(xgen(n), device="cuda")
        y = torch.empty_like(x)
        out = {"p": p, "q1d": q, "N": N, "ndof": n, "elements": E, "space_host_s": t_space}
        for kind in ("diffusion", "mass"):
            form = F.Form(space, kind, q, coef=kap)
            tset = time_events(lambda: form.set_coef(kap), 2, 1)
            flops, bytes64 = alg_counts(p, q, E, n, kind=kind)
            _, bytes32 = alg_counts(p, q, E, n, kind=kind, fp=4)
            t64 = time_events(lambda: form.apply(x, y), args.steps, 3)
            x32 = x.float()
            y32 = torch.empty_like(x32)
            t32 = time_events(lambda: form.apply(x32, y32), args.steps, 3)
            ye = torch.empty((E, (p + 1) ** 3), dtype=torch.float64, device="cuda")
            ye32 = torch.empty((E, (p + 1) ** 3), dtype=torch.float32, device="cuda")
            te64 = time_events(lambda: form.apply_element(x, ye), args.steps, 3)
            te32 = time_events(lambda: form.apply_element(x32, ye32), args.steps, 3)
            tedf = time_events(lambda: form.apply_element(x, ye, arith="df64"), args.steps, 3)
            del ye, ye32
            d = torch.empty_like(x)
            tdiag = time_events(lambda: form.diagonal(d), 3, 1)
            out[kind] = {
                "f64_gdofs": n / t64 * 1e-6, "f64_ms": t64, "f64_tflops": flops / t64 * 1e-9,
                "f64_frac_fp64_peak": flops / t64 * 1e-9 / FP64_PEAK_TFLOPS,
                "f32_gdofs": n / t32 * 1e-6, "f32_ms": t32, "f32_alg_gbs": bytes32 / t32 * 1e-6,
                "f32_frac_hbm": bytes32 / t32 * 1e-6 / peaks().get("hbm_gbs", 6800.0),
                "setup_ms": tset, "diag_ms": tdiag,
                "element_ms": {"f64": te64, "f32": te32, "df64": tedf}}
            if kind == "diffusion":
                b = torch.empty_like(x)
                out["rhs_ms"] = time_events(lambda: _sin_rhs(form, b), 2, 1)
                if not args.no_solve:
                    form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
                    bc = torch.empty_like(b)
                    form.lift_rhs(b, torch.zeros_like(b), bc)
                    sol = {}
                    for prec in ("f64", "mixed", "mixed_ru"):
                        u = torch.zeros_like(b)
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        info = form.solve(bc, u, rtol=1e-10, maxit=args.solve_maxit, precision=prec,
                                          raise_on_error=False)
                        torch.cuda.synchronize()
                        sol[prec] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                     "outer": info["outer"], "relres": info["relres"],
                                     "converged": info["converged"]}
                    sol["speedup_mixed"] = sol["f64"]["seconds"] / sol["mixed"]["seconds"]
                    sol["speedup_mixed_ru"] = sol["f64"]["seconds"] / sol["mixed_ru"]["seconds"]
                    out["solve"] = sol
            del form, x32, y32, d
        # convection (beta . grad u, v) with beta = (1 + y, sin 2z, x y - 1/2)
        probe = F.Form(space, "mass", q)
        xq = probe.qpoint_coords()
        beta = torch.stack([1.0 + xq[..., 1], torch.sin(2.0 * xq[..., 2]), xq[..., 0] * xq[..., 1] - 0.5],
                           -1).contiguous()
        del xq, probe
        cform = F.Form.convection(space, beta, q1d=q, coef=kap)
        del beta
        D1 = p + 1
        cflops = 2.0 * (3 * q * D1 ** 3 + 4 * q ** 2 * D1 ** 2 + 4 * q ** 3 * D1 + 3 * q ** 3) * E
        ye = torch.empty((E, D1 ** 3), dtype=torch.float64, device="cuda")
        ye32 = torch.empty((E, D1 ** 3), dtype=torch.float32, device="cuda")
        x32 = x.float()
        tc = time_events(lambda: cform.apply(x, y), args.steps, 3)
        tc64 = time_events(lambda: cform.apply_element(x, ye), args.steps, 3)
        tc32 = time_events(lambda: cform.apply_element(x32, ye32), args.steps, 3)
        tcdf = time_events(lambda: cform.apply_element(x, ye, arith="df64"), args.steps, 3)
        out["convection"] = {"f64_ms": tc, "f64_gdofs": n / tc * 1e-6,
                             "f64_element_frac_fp64_peak": cflops / tc64 * 1e-9 / FP64_PEAK_TFLOPS,
                             "element_ms": {"f64": tc64, "f32": tc32, "df64": tcdf}}
        del cform, ye, ye32, x32
        print(json.dumps(out), flush=True)
        del space, x, y
        torch.cuda.empty_cache()
    return 0


# Lattice sizes of the elasticity workload: 3 * ndof ~ 4.1e6-4.3e6 vector entries.
ELAST_N = {1: 110, 2: 55, 3: 37, 4: 28, 5: 22, 6: 18, 7: 16, 8: 14}


def elasticity_flops(p, q, E):
    """Algorithmic flops of one elasticity apply: the diffusion sum
    factorization on three components (unfolded 1D operators, 2 flops per
    multiply-add) plus the stress map at every point (H = Ghat J^-1: 45,
    trace and lambda term: 3, stress: 15, F = S J^-T: 45; 108 flops)."""
    D1, Q = p + 1, q
    return (6 * (4 * Q * D1 ** 3 + 6 * Q ** 2 * D1 ** 2 + 6 * Q ** 3 * D1) + 108 * Q ** 3) * E


def run_elasticity(args):
    """Linear elasticity workload, one JSON line per order p: a 0.15h-perturbed
    lattice with 3 ndof ~ 4.2e6 vector entries, lognormal lambda and mu per
    element; setup, FP64 / double-float / FP32 apply, the diagonal, and
    Jacobi-PCG (FP64 and FP32-inner refinement) and p-multigrid flexible CG
    (FP32 V-cycle, double-float outer) to 1e-8 for a clamped body under
    gravity."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from fem_inputs import hex_lattice, lognormal, x_uniform
    for p in [int(v) for v in args.orders.split(",")]:
        N, q = ELAST_N[p], p + 2
        c, h = hex_lattice(N, 0.15, seed=60 + p)
        E = h.shape[0]
        lam = torch.as_tensor(lognormal(70 + p, E), device="cuda")
        mu = torch.as_tensor(lognormal(80 + p, E), device="cuda")
        space = F.Space(F.Mesh(c, h), p)
        form = F.Form.elasticity(space, lam, mu, q1d=q)
        n = form.n
        x = torch.as_tensor(x_uniform(90 + p, n), device="cuda")
        y = torch.empty_like(x)
        x32, y32 = x.float(), torch.empty(n, dtype=torch.float32, device="cuda")
        ye = torch.empty(3 * E * (p + 1) ** 3, dtype=torch.float64, device="cuda")
        ye32 = torch.empty(3 * E * (p + 1) ** 3, dtype=torch.float32, device="cuda")
        flops = elasticity_flops(p, q, E)
        bytes32 = 4 * (12 * q ** 3 * E + 2 * n) + 4 * (p + 1) ** 3 * E
        t64 = time_events(lambda: form.apply(x, y), args.steps, 3)
        tdf = time_events(lambda: form.apply(x, y, arith="df64"), args.steps, 3)
        t32 = time_events(lambda: form.apply(x32, y32), args.steps, 3)
        te64 = time_events(lambda: form.apply_element(x, ye), args.steps, 3)
        tedf = time_events(lambda: form.apply_element(x, ye, arith="df64"), args.steps, 3)
        te32 = time_events(lambda: form.apply_element(x32, ye32), args.steps, 3)
        del ye, ye32
        d = torch.empty_like(x)
        tdiag = time_events(lambda: form.diagonal(d), 3, 1)
        tset = time_events(lambda: form.set_lame(lam, mu), 3, 1)
        out = {"workload": f"elasticity p={p}, q={q}, {N}^3 hexes", "p": p, "q1d": q, "N": N, "elements": E,
               "ndof": space.ndof, "vector_len": n,
               "f64": {"ms": t64, "gdofs": n / t64 * 1e-6, "element_ms": te64,
                       "element_frac_fp64_peak": flops / te64 * 1e-9 / FP64_PEAK_TFLOPS},
               "df64": {"ms": tdf, "gdofs": n / tdf * 1e-6, "element_ms": tedf},
               "f32": {"ms": t32, "gdofs": n / t32 * 1e-6, "element_ms": te32,
                       "element_alg_gbs": bytes32 / te32 * 1e-6,
                       "element_frac_hbm": bytes32 / te32 * 1e-6 / peaks().get("hbm_gbs", 6800.0),
                       "element_tflops": flops / te32 * 1e-9},
               "alg_flops": flops, "diag_ms": tdiag, "setup_ms": tset}
        if not args.no_solve:
            ndof = space.ndof
            bd = torch.as_tensor(space.boundary_dofs(), device="cuda", dtype=torch.int64)
            form.set_essential(torch.cat([bd + k * ndof for k in range(3)]).to(torch.int32))
            fq = torch.zeros((3, E, q ** 3), dtype=torch.float64, device="cuda")
            fq[2] = -1.0
            b = torch.empty_like(x)
            form.rhs(fq, b)
            del fq
            bc = torch.empty_like(b)
            form.lift_rhs(b, torch.zeros_like(b), bc)
            sol = {}
            for prec in ("f64", "mixed"):
                u = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = form.solve(bc, u, rtol=1e-8, maxit=args.solve_maxit, precision=prec, raise_on_error=False)
                torch.cuda.synchronize()
                sol[prec] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                             "outer": info["outer"], "relres": info["relres"], "converged": info["converged"]}
            sol["speedup_mixed"] = sol["f64"]["seconds"] / sol["mixed"]["seconds"]
            # p-multigrid flexible CG: FP32 V-cycle, double-float outer operator
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # Chebyshev order 4 on [0.2, 1] * 1.1 lambda: the best of the measured
            # (order, interval, coarse iterations) choices for elasticity
            mg = F.Multigrid(form, precision="f32", cheb_order=4, cheb_lo=0.2)
            torch.cuda.synchronize()
            t_mg = time.perf_counter() - t0
            u = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = mg.solve(bc, u, rtol=1e-8, check_every=4, raise_on_error=False, arith="df64")
            torch.cuda.synchronize()
            sol["pmg_f32_df64"] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                   "relres": info["relres"], "converged": info["converged"],
                                   "hierarchy_setup_s": t_mg}
            sol["speedup_pmg"] = sol["f64"]["seconds"] / sol["pmg_f32_df64"]["seconds"]
            u = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = mg.solve(bc, u, rtol=1e-8, check_every=4, raise_on_error=False, arith="f32")
            torch.cuda.synchronize()
            sol["pmg_f32_f32"] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                  "outer": info["outer"], "relres": info["relres"], "converged": info["converged"]}
            sol["speedup_pmg_f32_outer"] = sol["f64"]["seconds"] / sol["pmg_f32_f32"]["seconds"]
            del mg
            out["solve_1e-8"] = sol
        print(json.dumps(out), flush=True)
        del form, space, x, y, x32, y32, d
        torch.cuda.empty_cache()
    return 0


def batch_config(seed=40, nprob=256):
    """Seeded sizes of the batching workload: N_i ~ U{2..24}, p_i ~ U{1..6}."""
    from fem_inputs import splitmix64
    d = splitmix64(seed, 2 * nprob)
    Ns = [2 + int(v % np.uint64(23)) for v in d[0::2]]
    ps = [1 + int(v % np.uint64(6)) for v in d[1::2]]
    return Ns, ps


def run_batch(args):
    """Batching workload: 256 independent diffusion problems, N_i^3 elements
    (N_i ~ U{2..24}), p_i ~ U{1..6}, q = p + 2, lognormal kappa, 8 right-hand
    sides each, x ~ U[-1, 1]; FP64 and FP32 batched applies (one persistent
    element launch + one persistent scatter launch, one CUDA graph), tile
    autotuning, and the mixed-precision batched solve."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from fem_inputs import hex_lattice, lognormal, x_uniform
    Ns, ps = batch_config(nprob=args.nprob)
    nrhs = args.nrhs
    forms, keep = [], []
    t0 = time.perf_counter()
    for i, (N, p) in enumerate(zip(Ns, ps)):
        c, h = hex_lattice(N, 0.15, seed=4000 + i)
        kappa = lognormal(5000 + i, h.shape[0])
        sp = F.Space(F.Mesh(c, h), p)
        fm = F.Form(sp, "diffusion", p + 2, coef=torch.as_tensor(kappa, device="cuda"))
        forms.append(fm)
        keep.append(sp)
    t_setup = time.perf_counter() - t0
    bt = F.Batch(forms, nrhs)
    ndof = int(bt.off[-1])
    E = sum(sp.ne for sp in keep)
    flops = sum(alg_counts(sp.p, sp.p + 2, sp.ne, sp.ndof)[0] for sp in keep) * nrhs
    bytes64 = sum(alg_counts(sp.p, sp.p + 2, sp.ne, sp.ndof)[1] - 16 * sp.ndof for sp in keep) + 16 * ndof * nrhs
    X = torch.as_tensor(x_uniform(41, bt.total_len), device="cuda")
    Y = torch.empty_like(X)
    out = {"workload": f"batch: {len(forms)} diffusion problems, N_i~U{{2..24}}, p_i~U{{1..6}}, {nrhs} RHS",
           "problems": len(forms), "nrhs": nrhs, "ndof_total": ndof, "unknowns": bt.total_len, "elements": E,
           "host_setup_s": t_setup}
    cache = os.path.join(tempfile.gettempdir(), "fem_batch_tiles.json")
    t0 = time.perf_counter()
    tiles32 = bt.tune("f32", cache)
    out["tune_f32_s"] = time.perf_counter() - t0
    out["tiles"] = {f"p{p}q{p + 2}": int(tiles32[2 * p + 1]) for p in sorted(set(ps))}
    for dt, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        Xd = X.to(tdt)
        Yd = torch.empty_like(Xd)
        t = time_events(lambda: bt.apply(Xd, Yd), args.steps, 2)
        rec = {"ms": t, "gdofs": bt.total_len / t * 1e-6}
        if dt == "f64":
            rec["tflops"] = flops / t * 1e-9
            rec["frac_fp64_peak"] = flops / t * 1e-9 / FP64_PEAK_TFLOPS
        else:
            b32 = bytes64 / 2
            rec["alg_gbs"] = b32 / t * 1e-6
        out[f"apply_{dt}"] = rec
        del Xd, Yd
    if not args.no_solve:
        for fm, sp in zip(forms, keep):
            fm.set_essential(torch.as_tensor(sp.boundary_dofs(), device="cuda"))
        Bc = torch.empty_like(X)
        for i, (fm, sp) in enumerate(zip(forms, keep)):
            zero = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
            for r in range(nrhs):
                fm.lift_rhs(bt.block(X, i, r).contiguous(), zero, bt.block(Bc, i, r))
        precs = ["mixed"] + (["f64"] if args.batch_f64_solve else [])
        for prec in precs:
            U = torch.zeros_like(Bc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = bt.solve(Bc, U, rtol=1e-10, precision=prec, maxit=args.solve_maxit, raise_on_error=False)
            torch.cuda.synchronize()
            out[f"solve_{prec}"] = {"seconds": time.perf_counter() - t0, "status": info["status"],
                                    "max_iterations": int(info["iterations"].max()),
                                    "mean_iterations": float(info["iterations"].mean()),
                                    "max_relres": float(info["relres"].max())}
    print(json.dumps(out), flush=True)
    return 0


# The 2D Example-1 workload of the paper's GPU table: about 1.3M DOFs for
# p = 1, 2, 4, 8 on an N x N quadrilateral mesh ((N p + 1)^2 DOFs).
PAPER2D_N = {1: 1140, 2: 570, 4: 285, 8: 143}
# Seconds for 200 CG iterations on one GV100 in the paper's table (context
# only: another GPU, another code): best GPU backend and the plain CUDA one.
PAPER2D_GV100_S = {1: (0.19, 0.36), 2: (0.15, 0.26), 4: (0.12, 0.17), 8: (0.12, 0.15)}


def run_paper2d(args):
    """2D Poisson (Example 1): -Laplace u = 1 on the unit square, perturbed
    (0.15h) quadrilateral mesh, homogeneous Dirichlet conditions, partial
    assembly, 200 CG iterations, p in {1, 2, 4, 8} at about 1.3M DOFs. One
    JSON line per order: 200 iterations of plain CG and of Jacobi-PCG (FP64
    and FP32 vectors), and the FP64 / FP32 / double-float apply."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from fem_inputs import quad_lattice
    orders = [int(v) for v in args.orders.split(",") if int(v) in PAPER2D_N] if args.orders != "1,2,3,4,5,6,7,8" \
        else [1, 2, 4, 8]
    for p in orders:
        N = PAPER2D_N[p]
        q = p + 2
        c, qd = quad_lattice(N, 0.15, seed=60 + p)
        space = F.Space(F.Mesh2D(c, qd), p)
        n, E = space.ndof, space.ne
        form = F.Form(space, "diffusion", q)
        form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        form.rhs(torch.ones((E, form.nq), dtype=torch.float64, device="cuda"), b)
        bc = torch.empty_like(b)
        form.lift_rhs(b, torch.zeros_like(b), bc)
        out = {"workload": f"2D Poisson Ex1, p={p}, q={q}, {N}^2 quads perturbed 0.15h, 200 CG iterations",
               "p": p, "q1d": q, "N": N, "ndof": n, "elements": E,
               "paper_gv100_s": {"best_gpu": PAPER2D_GV100_S[p][0], "cuda": PAPER2D_GV100_S[p][1]}}
        for name, prec, pc in (("cg_f64", "f64", "none"), ("pcg_f64", "f64", "jacobi"),
                               ("pcg_df64", "df64", "jacobi")):
            ts = []
            for rep in range(3):
                u = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = form.solve(bc, u, rtol=1e-30, maxit=200, precision=prec, precond=pc, raise_on_error=False,
                                  check_every=50)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            out[name] = {"seconds": min(ts), "iterations": info["iterations"], "relres": info["relres"]}
        x = torch.as_tensor(np.linspace(-1.0, 1.0, n), device="cuda")
        y = torch.empty_like(x)
        flops, _ = alg_counts(p, q, E, n, dim=2)
        _, bytes32 = alg_counts(p, q, E, n, fp=4, dim=2)
        t64 = time_events(lambda: form.apply(x, y), args.steps, 3)
        x32, y32 = x.float(), torch.empty(n, dtype=torch.float32, device="cuda")
        t32 = time_events(lambda: form.apply(x32, y32), args.steps, 3)
        ye = torch.empty((E, (p + 1) ** 2), dtype=torch.float64, device="cuda")
        te64 = time_events(lambda: form.apply_element(x, ye), args.steps, 3)
        tedf = time_events(lambda: form.apply_element(x, ye, arith="df64"), args.steps, 3)
        out["apply"] = {"f64_ms": t64, "f64_gdofs": n / t64 * 1e-6, "f64_element_ms": te64,
                        "f64_element_frac_fp64_peak": flops / te64 * 1e-9 / FP64_PEAK_TFLOPS,
                        "df64_element_ms": tedf, "f32_ms": t32, "f32_gdofs": n / t32 * 1e-6,
                        "f32_alg_gbs": bytes32 / t32 * 1e-6}
        print(json.dumps(out), flush=True)
        del form, space, x, y, x32, y32, ye, b, bc
        torch.cuda.empty_cache()
    return 0


MG_SWEEP = [(2, 0.25, 1.1, 20), (2, 0.25, 1.1, 30), (2, 0.25, 1.1, 40), (2, 0.25, 1.1, 60), (3, 0.2, 1.1, 30),
            (3, 0.2, 1.1, 40), (4, 0.2, 1.1, 30), (2, 0.3, 1.2, 30)]


def run_mgsweep(args):
    """Smoother and coarse-solve parameters of the p-multigrid solve: for each
    (Chebyshev order K, interval low end, cheb_hi, coarsest-level PCG
    iterations) of MG_SWEEP, flexible CG with an FP32 V-cycle and the
    double-float outer operator, best of two solves. --kind diffusion: the
    mg workload's problem (p, N, rtol 1e-10); --kind elasticity: the
    elasticity workload's problem for each p of --orders (rtol 1e-8). One
    JSON line per configuration."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from fem_inputs import hex_lattice, lognormal
    problems = []
    if args.kind == "diffusion":
        p, N = args.p, args.N
        c, h, kappa, _ = make_problem(p, N)
        space = F.Space(F.Mesh(c, h), p)
        form = F.Form(space, "diffusion", p + 2, coef=torch.as_tensor(kappa, device="cuda"))
        form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
        b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
        _sin_rhs(form, b)
        problems.append((p, N, form, b, 1e-10))
    else:
        for p in [int(v) for v in args.orders.split(",")]:
            N = ELAST_N[p]
            c, h = hex_lattice(N, 0.15, seed=60 + p)
            E = h.shape[0]
            space = F.Space(F.Mesh(c, h), p)
            form = F.Form.elasticity(space, torch.as_tensor(lognormal(70 + p, E), device="cuda"),
                                     torch.as_tensor(lognormal(80 + p, E), device="cuda"), q1d=p + 2)
            bd = torch.as_tensor(space.boundary_dofs(), device="cuda", dtype=torch.int64)
            form.set_essential(torch.cat([bd + k * space.ndof for k in range(3)]).to(torch.int32))
            fq = torch.zeros((3, E, (p + 2) ** 3), dtype=torch.float64, device="cuda")
            fq[2] = -1.0
            b = torch.empty(form.n, dtype=torch.float64, device="cuda")
            form.rhs(fq, b)
            problems.append((p, N, form, b, 1e-8))
    for p, N, form, b, rtol in problems:
        bc = torch.empty_like(b)
        form.lift_rhs(b, torch.zeros_like(b), bc)
        for K, lo, hi, cits in MG_SWEEP:
            mg = F.Multigrid(form, cheb_order=K, cheb_lo=lo, cheb_hi=hi, coarse_its=cits, precision="f32")
            best, it, conv = None, None, None
            for _ in range(2):
                u = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = mg.solve(bc, u, rtol=rtol, check_every=4, raise_on_error=False, arith="df64")
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                if best is None or t < best:
                    best, it, conv = t, info["iterations"], info["converged"]
            print(json.dumps({"kind": args.kind, "p": p, "N": N, "rtol": rtol, "cheb_order": K, "cheb_lo": lo,
                              "cheb_hi": hi, "coarse_its": cits, "iterations": it, "seconds": best,
                              "converged": conv}), flush=True)
            del mg
    return 0


def run_mg(args):
    """p-multigrid workload: the apply workload's problem (p, N; lognormal
    kappa, sin sin sin right-hand side, homogeneous Dirichlet conditions),
    solved to 1e-10 by flexible CG with one V-cycle per iteration (FP64 and
    FP32 V-cycles), beside Jacobi-PCG in FP64 and mixed precision. One JSON
    line."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    p, N = args.p, args.N
    c, h, kappa, _ = make_problem(p, N)
    space = F.Space(F.Mesh(c, h), p)
    form = F.Form(space, "diffusion", p + 2, coef=torch.as_tensor(kappa, device="cuda"))
    form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
    b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    _sin_rhs(form, b)
    bc = torch.empty_like(b)
    form.lift_rhs(b, torch.zeros_like(b), bc)
    out = {"workload": f"p-multigrid FCG, p={p}, q={p + 2}, {N}^3 hexes perturbed 0.15h, lognormal kappa, rtol 1e-10",
           "p": p, "N": N, "ndof": space.ndof}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    for prec in ("f32", "f64"):
        ts, mg = timed(lambda: F.Multigrid(form, precision=prec, coarse_its=args.mg_coarse_its))
        res = {"setup_s": ts, "levels": mg.info()}
        z = torch.empty_like(b)
        res["vcycle_ms"] = time_events(lambda: mg.vcycle(bc, z), 5, 2)
        for arith in ("f64", "df64", "f32"):
            best = None
            for _ in range(2):
                u = torch.zeros_like(b)
                t, info = timed(lambda: mg.solve(bc, u, rtol=1e-10, check_every=4, raise_on_error=False, arith=arith))
                if best is None or t < best[0]:
                    best = (t, info)
            res["outer_" + arith] = {"seconds": best[0], "iterations": best[1]["iterations"],
                                     "relres": best[1]["relres"], "converged": best[1]["converged"]}
        out["mg_" + prec] = res
        del mg
    if not args.no_solve:
        for prec in ("mixed", "f64"):
            u = torch.zeros_like(b)
            t, info = timed(lambda: form.solve(bc, u, rtol=1e-10, maxit=args.solve_maxit, precision=prec,
                                               raise_on_error=False))
            out["pcg_" + prec] = {"seconds": t, "iterations": info["iterations"], "relres": info["relres"]}
    print(json.dumps(out), flush=True)
    return 0


def run_curved(args):
    """Curved-geometry workload: the apply workload's mesh (p, N) with order-k
    nodal geometry (k = 2, 4; boundary-preserving bulge of amplitude 0.05):
    setup (D) time against the vertex geometry, FP64 apply, and the
    p-multigrid solve to 1e-10 on the curved mesh. One JSON line."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from fem_inputs import curved_nodes
    p, N = args.p, args.N
    c, h, kappa, xgen = make_problem(p, N)
    kap = torch.as_tensor(kappa, device="cuda")
    out = {"workload": f"curved geometry, p={p}, q={p + 2}, {N}^3 hexes, nodal order k = 2, 4", "p": p, "N": N}
    for k in (0, 2, 4):
        mesh = F.Mesh(c, h)
        t0 = time.perf_counter()
        if k:
            mesh.set_nodes(curved_nodes(c, h, k, amp=0.05), k)
        t_nodes = time.perf_counter() - t0
        space = F.Space(mesh, p)
        form = F.Form(space, "diffusion", p + 2, coef=kap)
        t_setup = time_events(lambda: form.set_coef(kap), 3, 1)
        x = torch.as_tensor(xgen(space.ndof), device="cuda")
        y = torch.empty_like(x)
        t_apply = time_events(lambda: form.apply(x, y), args.steps, 3)
        res = {"nodes_host_s": t_nodes, "setup_ms": t_setup, "apply_f64_ms": t_apply, "ndof": space.ndof}
        if not args.no_solve:
            form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
            b = torch.empty_like(x)
            _sin_rhs(form, b)
            bc = torch.empty_like(b)
            form.lift_rhs(b, torch.zeros_like(b), bc)
            mg = F.Multigrid(form, precision="f32")
            u = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = mg.solve(bc, u, rtol=1e-10, check_every=4, raise_on_error=False, arith="df64")
            torch.cuda.synchronize()
            res["pmg_solve"] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                "converged": info["converged"], "relres": info["relres"]}
            del mg
        out["k%d" % k if k else "vertex"] = res
        del form, space, mesh, x, y
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_grad(args):
    """Differentiation workload: 64^3 hexes, 0.1h, p = 2, kappa = 0.01 + rho^3,
    rho ~ U[0.2, 1], f = 1, homogeneous Dirichlet: compliance solve and the
    adjoint-kernel gradient through torch.autograd."""
    import torch
    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300.autograd import compliance
    from fem_inputs import hex_lattice, rho_uniform
    c, h = hex_lattice(64, 0.1, seed=50)
    E = h.shape[0]
    rho = torch.as_tensor(rho_uniform(50, E), device="cuda")
    space = F.Space(F.Mesh(c, h), 2)
    form = F.Form(space, "diffusion", 4, coef=0.01 + rho ** 3)
    form.set_essential(torch.as_tensor(space.boundary_dofs(), device="cuda"))
    fq = torch.ones((E, form.nq), dtype=torch.float64, device="cuda")
    b = torch.empty(space.ndof, dtype=torch.float64, device="cuda")
    form.rhs(fq, b)
    bc = torch.empty_like(b)
    form.lift_rhs(b, torch.zeros_like(b), bc)
    out = {"workload": "compliance gradient, 64^3 hexes, p=2, q=4", "ndof": space.ndof, "elements": E}
    for prec in ("f64", "mixed"):
        r = rho.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, u = compliance(0.01 + r ** 3, form, bc, rtol=1e-10, precision=prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out[prec] = {"forward_s": t1 - t0, "backward_s": t2 - t1, "J": J.item()}
    g = torch.empty(E, dtype=torch.float64, device="cuda")
    out["grad_kernel_ms"] = time_events(lambda: form.compliance_grad(u, g), args.steps, 2)
    print(json.dumps(out), flush=True)
    return 0


def run_sharded(args, world, rank, local, dev):
    """N > 1: one problem element-partitioned over the ranks (slab
    partition, owned + halo L-vector, one halo exchange per apply over NCCL;
    include/fem.h fem_shard_*). Weak scaling keeps ~N^3 elements per rank
    (global mesh round(N * world^(1/3))^3); strong scaling splits the N^3
    problem. One step = one sharded apply y = A x (element kernel, scatter,
    pack, exchange, combine); value = global DOFs / the slowest rank's step
    time."""
    import torch
    import torch.distributed as dist
    import paper_1911_09220_gb300 as F
    from paper_1911_09220_gb300 import shard as S
    from fem_inputs import hex_lattice, lognormal, x_uniform
    p, q = args.p, args.p + 2
    Ng = int(round(args.N * world ** (1.0 / 3.0))) if args.scaling == "weak" else args.N
    c, h = hex_lattice(Ng, 0.15, seed=10 + p)
    kappa = lognormal(20 + p, h.shape[0])
    t0 = time.perf_counter()
    gmesh = F.Mesh(c, h)
    gspace = F.Space(gmesh, p)
    part = S.partition_slabs(gmesh, world)
    sh = S.Shard(gspace, part, world, rank)
    tab = sh.tables()
    t_setup = time.perf_counter() - t0
    form = F.Form(sh.space, "diffusion", q, coef=torch.as_tensor(kappa[tab["elems"]], device=dev))
    comm = S.TorchComm()
    xg = x_uniform(30 + p, gspace.ndof)
    x_host = torch.as_tensor(np.ascontiguousarray(xg[tab["l2g"]])).pin_memory()
    x = x_host.to(dev)
    y = torch.empty_like(x)
    del xg
    stream = torch.cuda.current_stream()
    dist.barrier()
    for _ in range(args.warmup):
        sh.apply(form, x, y, comm)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sh.apply(form, x, y, comm)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms_step = reduce_max(e0.elapsed_time(e1) / args.steps, dev)
    value = gspace.ndof / (ms_step * 1e-3) / 1e9
    # the rank's element kernel alone (FP64 roofline of the local work)
    ye = torch.empty((sh.ne, (p + 1) ** 3), dtype=torch.float64, device=dev)
    t_el = time_events(lambda: form.apply_element(x, ye), args.steps, 2)
    flops, bytes_alg = alg_counts(p, q, sh.ne, sh.ndof)
    achieved = flops / (t_el * 1e-3) / 1e12
    # end to end: the rank's local input from pinned host memory, the sharded
    # apply, the result back to pinned host memory, every step
    y_host = torch.empty_like(x_host).pin_memory()
    xb = torch.empty_like(x)

    def e2e_step():
        xb.copy_(x_host, non_blocking=True)
        sh.apply(form, xb, y, comm)
        y_host.copy_(y, non_blocking=True)

    e2e_step()
    dist.barrier()
    torch.cuda.synchronize()
    t_e2e = reduce_max(time_events(e2e_step, args.steps, 1), dev)
    if rank == 0:
        line = {
            "metric": "PA diffusion apply GDOF/s", "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 PA diffusion apply y=Ax, p={p}, q={q}, {Ng}^3 hex mesh perturbed 0.15h, "
                                   f"lognormal kappa, {gspace.ndof} DOFs, element slabs over {world} ranks",
                       "p": p, "q1d": q, "N": Ng, "ndof": gspace.ndof, "elements": int(h.shape[0]),
                       "parallelism": f"element-partitioned x{world} (halo exchange over NCCL)",
                       "rank0_local_dofs": sh.ndof, "rank0_neighbours": sh.nnbr, "rank0_shared_slots": sh.nslots,
                       "l2": "inputs larger than L2; no flush"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "kernel": f"k_diffusion_apply<double,{p + 1},{q},NE> on rank 0's elements",
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz"},
            "cpu_baseline": None,
            "e2e": {"value": gspace.ndof / (t_e2e * 1e-3) / 1e9, "unit": "GDOF/s",
                    "h2d_bytes_per_step": 8 * sh.ndof * world, "d2h_bytes_per_step": 8 * sh.ndof * world,
                    "ms_per_step": t_e2e},
            "gpu_launches": 4 * args.steps, "clocks": clk, "setup_s": {"global_and_shard_host": t_setup},
        }
        print(json.dumps(line))
    dist.barrier()
    dist.destroy_process_group()
    return 0



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--N", type=int, default=68)
    ap.add_argument("--cpu-n", type=int, default=16, help="lattice size of the CPU oracle sample")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--solve-maxit", type=int, default=20000)
    ap.add_argument("--workload", default="apply", choices=["apply", "sweep", "batch", "grad", "paper2d", "mg", "curved",
                                                         "elasticity", "mgsweep"])
    ap.add_argument("--kind", default="diffusion", choices=["diffusion", "elasticity"])
    ap.add_argument("--sweep-size", default="4e6", choices=["1e6", "4e6", "2e7", "3e7"])
    ap.add_argument("--orders", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--nprob", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--batch-f64-solve", action="store_true")
    ap.add_argument("--mg-coarse-its", type=int, default=30)
    ap.add_argument("--parallel", default="shard", choices=["shard", "replicas"],
                    help="N > 1: one element-partitioned problem (shard) or independent problems per rank")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="shard mode: ~N^3 elements per rank (weak) or one N^3 problem split over the ranks")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "paper2d":
        return run_paper2d(args)
    if args.workload == "mg":
        return run_mg(args)
    if args.workload == "curved":
        return run_curved(args)
    if args.workload == "grad":
        return run_grad(args)
    if args.workload == "elasticity":
        return run_elasticity(args)
    if args.workload == "mgsweep":
        return run_mgsweep(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # FEM_BENCH_BACKEND=gloo runs the ranks' exchanges through host copies
        # (several ranks sharing one GPU in a test); NCCL otherwise
        dist.init_process_group(os.environ.get("FEM_BENCH_BACKEND", "nccl"))
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1911_09220_gb300 import build as fbuild
    fbuild.build()
    import paper_1911_09220_gb300 as F
    if world > 1 and args.parallel == "shard":
        return run_sharded(args, world, rank, local, dev)

    # measured FMA rates of this GPU (library probe kernel, ~20 ms each):
    # the cross-check of the derived FP64 peak that the roofline is quoted on
    probe = {"fp64_tflops": F.probe_fma_peak("f64"), "fp32_tflops": F.probe_fma_peak("f32"),
             "kernel": "k_fma_probe (fem_probe_fma_peak): 8 independent FMA chains per thread, every SM at "
                       "full occupancy, CUDA events"}
    p, N = args.p, args.N
    q = p + 2
    c, h, kappa, xgen = make_problem(p, N, seed_offset=rank_seed_offset(rank))
    t0 = time.perf_counter()
    mesh = F.Mesh(c, h)
    space = F.Space(mesh, p)
    t_space = time.perf_counter() - t0
    kap = torch.as_tensor(kappa, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    form = F.Form(space, "diffusion", q, coef=kap)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n, E = space.ndof, space.ne
    x_host = torch.as_tensor(xgen(n)).pin_memory()
    x = x_host.to(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    ye = torch.empty((E, (p + 1) ** 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        form.apply(x, y)
        form.apply_element(x, ye)
        form.scatter(ye, y)
    torch.cuda.synchronize()

    # Timed region: K steps of the public apply (fem_apply: element kernel and
    # scatter, the E-vector in DOF-sorted order at this size), then the same
    # K applies through the public halves (element-major E-vector), whose
    # per-kernel CUDA events give the element kernel's duration for the
    # roofline (the same arithmetic; only its output addresses differ).
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e_start, e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for k in range(args.steps):
        form.apply(x, y)
    e_stop.record(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        form.apply_element(x, ye)
        ev[k][1].record(stream)
        form.scatter(ye, y)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t_total_ms = e_start.elapsed_time(e_stop)
    t_elem = [a.elapsed_time(b) for a, b, _ in ev]
    t_scat = [b.elapsed_time(c_) for _, b, c_ in ev]
    ms_step = reduce_max(t_total_ms / args.steps, dev)
    value = world * n / (ms_step * 1e-3) / 1e9

    # end to end through the public API with host buffers: every step copies
    # its input from pinned host memory, applies, and copies the result back
    # to pinned host memory. Steps are pipelined the way a streaming caller
    # would run them: two device buffers, the input copy on one stream, the
    # result copy on another, so that step k's apply overlaps the input copy
    # of step k+1 and the result copy of step k-1. Timed from before the
    # first input copy to after the last result copy.
    y_host = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    xbuf = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    ybuf = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    def pipelined(K):
        e_in = [torch.cuda.Event() for _ in range(2)]
        e_ap = [torch.cuda.Event() for _ in range(2)]
        e_out = [torch.cuda.Event() for _ in range(2)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s_in)
        for k in range(K):
            b = k % 2
            if k >= 2:
                s_in.wait_event(e_ap[b])           # step k-2 has read xbuf[b]
            with torch.cuda.stream(s_in):
                xbuf[b].copy_(x_host, non_blocking=True)
            e_in[b].record(s_in)
            stream.wait_event(e_in[b])
            if k >= 2:
                stream.wait_event(e_out[b])        # step k-2's result has left ybuf[b]
            form.apply(xbuf[b], ybuf[b], stream=stream)
            e_ap[b].record(stream)
            s_out.wait_event(e_ap[b])
            with torch.cuda.stream(s_out):
                y_host[b].copy_(ybuf[b], non_blocking=True)
            e_out[b].record(s_out)
        t1.record(s_out)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    pipelined(2)
    e2e_ms = reduce_max(pipelined(args.steps) / args.steps, dev)
    e2e = {"value": world * n / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_ms,
           "pipelining": "double-buffered: H2D of step k+1 and D2H of step k-1 overlap the apply of step k"}

    flops, bytes_alg = alg_counts(p, q, E, n)
    t_el = statistics.mean(t_elem) * 1e-3
    achieved = flops / t_el / 1e12
    key = f"diffusion_f64_p{p}_N{N}"
    traffic_full = measured_traffic(key)
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_full,
            "kernel": f"k_diffusion_apply<double,{p + 1},{q},NE> (FP64 element kernel)",
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (headline)",
            "peak_measured": probe["fp64_tflops"], "frac_of_measured": achieved / probe["fp64_tflops"],
            "peak_measured_source": probe["kernel"],
            "alg_flops_per_launch": flops, "alg_bytes_per_launch": bytes_alg,
            "hbm_achieved_gbs": bytes_alg / (ms_step * 1e-3) / 1e9,
            "hbm_peak_gbs_measured": peaks().get("hbm_gbs"),
            "element_kernel_ms": statistics.mean(t_elem), "scatter_kernel_ms_element_major": statistics.mean(t_scat),
            "apply_ms": ms_step,
            "element_share": statistics.mean(t_elem) / ms_step}

    # FP32 apply of the same operator (the inner operator of the mixed solver)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    ye32 = torch.empty((E, (p + 1) ** 3), dtype=torch.float32, device=dev)
    form.apply(x32, y32)
    t32e = time_events(lambda: form.apply_element(x32, ye32), args.steps, 2)
    t32 = time_events(lambda: form.apply(x32, y32), args.steps, 2)
    _, bytes32 = alg_counts(p, q, E, n, fp=4)
    # bytes the atomic-free design moves on top of the algorithmic ones: the
    # inverse map (one int32 slot position per element slot and one offset
    # per DOF) and the E-vector written by the element kernel and read by the
    # scatter (counted separately, as implementation overheads)
    nd = (p + 1) ** 3
    impl32 = bytes32 + 4 * nd * E + 4 * (n + 1) + 2 * 4 * nd * E
    hbm = peaks().get("hbm_gbs", 6800.0)
    fp32 = {"gdofs": n / (t32 * 1e-3) / 1e9, "ms_per_apply": t32, "element_kernel_ms": t32e,
            "element_kernel_hbm_gbs": (bytes32 - 8 * n + 4 * n) / (t32e * 1e-3) / 1e9,
            "apply_alg_gbs": bytes32 / (t32 * 1e-3) / 1e9,
            "apply_frac_of_hbm": bytes32 / (t32 * 1e-3) / 1e9 / hbm,
            "alg_bytes_per_apply": bytes32,
            "impl_bytes_per_apply": impl32,
            "apply_frac_of_hbm_impl_bytes": impl32 / (t32 * 1e-3) / 1e9 / hbm}
    del x32, y32, ye32
    # double-float element arithmetic (FP64 vectors, FP32 pipe)
    form.apply(x, y, arith="df64")
    tdfe = time_events(lambda: form.apply_element(x, ye, arith="df64"), args.steps, 2)
    tdf = time_events(lambda: form.apply(x, y, arith="df64"), args.steps, 2)
    df64 = {"gdofs": n / (tdf * 1e-3) / 1e9, "ms_per_apply": tdf, "element_kernel_ms": tdfe,
            "alg_fp64_equiv_tflops": flops / (tdfe * 1e-3) / 1e12,
            "speedup_vs_fp64_element": statistics.mean(t_elem) / tdfe}
    # FP64 mass apply on the same mesh and coefficient
    mform = F.Form(space, "mass", q, coef=kap)
    tm = time_events(lambda: mform.apply(x, y), args.steps, 2)
    mflops, mbytes = alg_counts(p, q, E, n, kind="mass")
    mass = {"gdofs": n / (tm * 1e-3) / 1e9, "ms_per_apply": tm, "achieved_tflops": mflops / (tm * 1e-3) / 1e12,
            "frac_fp64_peak": mflops / (tm * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    del mform

    solve = None
    if not args.no_solve:
        solve = {}
        ess = torch.as_tensor(space.boundary_dofs(), device=dev)
        form.set_essential(ess)
        xq = form.qpoint_coords()
        fq = (3 * np.pi ** 2 * torch.sin(np.pi * xq[..., 0]) * torch.sin(np.pi * xq[..., 1])
              * torch.sin(np.pi * xq[..., 2])).contiguous()
        del xq
        b = torch.empty(n, dtype=torch.float64, device=dev)
        form.rhs(fq, b)
        del fq
        bc = torch.empty_like(b)
        form.lift_rhs(b, torch.zeros_like(b), bc)
        sols = {}
        for prec in ("f64", "mixed", "df64", "mixed_ru"):
            u = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = form.solve(bc, u, rtol=1e-10, maxit=args.solve_maxit, precision=prec, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            solve[prec] = {"seconds": dt, "iterations": info["iterations"], "outer": info["outer"],
                           "converged": info["converged"], "relres": info["relres"]}
            sols[prec] = u
        diff = (sols["mixed"] - sols["f64"]).abs().max().item() / sols["f64"].abs().max().item()
        solve["mixed_vs_f64_maxrel"] = diff
        solve["df64_vs_f64_maxrel"] = (sols["df64"] - sols["f64"]).abs().max().item() / sols["f64"].abs().max().item()
        solve["speedup_df64"] = solve["f64"]["seconds"] / solve["df64"]["seconds"]
        solve["mixed_ru_vs_f64_maxrel"] = (sols["mixed_ru"] - sols["f64"]).abs().max().item() / \
            sols["f64"].abs().max().item()
        solve["speedup_mixed_ru"] = solve["f64"]["seconds"] / solve["mixed_ru"]["seconds"]
        solve["speedup_mixed"] = solve["f64"]["seconds"] / solve["mixed"]["seconds"]
        # p-multigrid flexible CG: FP32 V-cycle, double-float outer operator
        t0 = time.perf_counter()
        mg = F.Multigrid(form, precision="f32")
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        u = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = mg.solve(bc, u, rtol=1e-10, check_every=4, raise_on_error=False, arith="df64")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        solve["pmg_f32_df64"] = {"seconds": dt, "setup_seconds": t_setup, "iterations": info["iterations"],
                                 "converged": info["converged"], "relres": info["relres"],
                                 "levels": mg.info()["orders"]}
        solve["pmg_vs_f64_maxrel"] = (u - sols["f64"]).abs().max().item() / sols["f64"].abs().max().item()
        solve["speedup_pmg"] = solve["f64"]["seconds"] / dt
        # the same with the FP32 outer operator inside FP64 refinement
        u = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = mg.solve(bc, u, rtol=1e-10, check_every=4, raise_on_error=False, arith="f32")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        solve["pmg_f32_f32"] = {"seconds": dt, "iterations": info["iterations"], "outer": info["outer"],
                                "converged": info["converged"], "relres": info["relres"],
                                "vs_f64_maxrel": (u - sols["f64"]).abs().max().item() / sols["f64"].abs().max().item()}
        solve["speedup_pmg_f32_outer"] = solve["f64"]["seconds"] / dt
        del mg
        solve["rtol"] = 1e-10

    cpu = None
    if rank == 0 and not args.no_cpu:
        its_full = solve["f64"]["iterations"] if solve else FP64_PCG_ITERS.get((p, N))
        pcg = None if args.no_solve else cpu_oracle_pcg(p, args.cpu_n, iters_full=its_full, ndof_full=n)
        r = cpu_oracle_spmv(p, args.cpu_n, 20, deadline_s=20.0)
        cpu = {"value": r["gdofs"], "unit": "GDOF/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"the oracle's assembled CSR matrix on a {args.cpu_n}^3-element sample of the same "
                         f"recipe ({r['ndof']} DOFs, nnz {r['nnz']}) applied by its C loop (OpenMP over rows, "
                         f"{r['cores']} threads), median of {r['reps']}; assembly {r['t_assembly']:.1f} s not timed",
               "single_core": r["single_core"], "host_cpus": os.cpu_count(), "pcg": pcg}

    if rank == 0:
        line = {
            "metric": "PA diffusion apply GDOF/s", "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 PA diffusion apply y=Ax, p={p}, q={q}, {N}^3 hex mesh perturbed 0.15h, "
                                   f"lognormal kappa, {n} DOFs per GPU", "p": p, "q1d": q, "N": N, "ndof": n,
                       "elements": E, "parallelism": f"replicas x{world} (independent problems)",
                       "l2": "inputs larger than L2 (D alone 3.26 GB); no flush"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 4 * args.steps,
            "fp32_apply": fp32, "mass_apply_f64": mass, "df64_apply": df64, "fma_probe": probe,
            "clocks": clk, "solve": solve,
            "setup_s": {"space_host": t_space, "form_setup": t_setup},
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
