"""bench.py's multi-rank path under torchrun: two ranks on the one GPU run
the sharded apply (element slabs, halo exchange after every apply) with the
exchange through gloo (FEM_BENCH_BACKEND=gloo; on a multi-GPU node the
default is NCCL), in weak and strong scaling modes. The JSON line must carry
the global problem, the whole-job throughput and the rank-0 roofline."""

import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("scaling,N,Ng", [("weak", 10, 13), ("strong", 12, 12)])
def test_bench_sharded_two_ranks(scaling, N, Ng):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FEM_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2",
           "--steps", "3", "--warmup", "1", "--p", "2", "--N", str(N), "--scaling", scaling]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == scaling
    assert d["config"]["N"] == Ng and d["config"]["ndof"] == (2 * Ng + 1) ** 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["value"] == pytest.approx(d["config"]["ndof"] / (d["ms_per_step"] * 1e-3) / 1e9)
    assert d["roofline"]["bound"] == "alu" and d["roofline"]["achieved"] > 0
    assert d["e2e"]["value"] > 0 and d["gpu_launches"] == 4 * 3
    assert d["config"]["rank0_neighbours"] == 1
