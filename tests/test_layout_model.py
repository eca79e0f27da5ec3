"""The FP32 element kernel's shared-memory layout (k_element.cuh): the
compile-time slab and buffer strides and lanes per element, printed by a
small host program built with nvcc, are run through a warp-by-warp model of
every stage's shared-memory accesses (32 four-byte banks; a warp access
costs as many wavefronts as the largest number of distinct words it touches
in one bank). Where each element gets its own warp in the short stages
(p = 4 at q = 6) the model must show no bank-conflict replays at all, for
the single-problem kernel's block and the batch's tile; where it gets a
half-warp (p = 2 at q = 4) fewer wavefronts than with packed lines;
elsewhere the layout must be the packed one (one lane per line)."""

import os
import shutil
import subprocess
import tempfile
from collections import defaultdict

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_09220_gb300", "csrc")

PRINTER = r"""
#include <cstdio>
#include "k_element.cuh"
template <int D1, int Q> void pr() {
  using L = ElemSmem<float, D1, Q>;
  printf("%d %d %d %d %d %d %d %d %d %d\n", D1, Q, L::XP, L::RB, L::RC, L::RT, L::RU, L::SE, L::L1, L::L2);
}
int main() {
  pr<2, 3>(); pr<3, 4>(); pr<4, 5>(); pr<5, 6>(); pr<6, 7>(); pr<7, 8>(); pr<8, 9>(); pr<9, 10>();
  return 0;
}
"""


@pytest.fixture(scope="module")
def layouts():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "p.cu"), os.path.join(d, "p")
    open(src, "w").write(PRINTER)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                        "-I", CSRC, src, "-o", exe, "-Xlinker", "--unresolved-symbols=ignore-all"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    shutil.rmtree(d, ignore_errors=True)
    res = {}
    for line in out.split("\n"):
        if line.strip():
            v = list(map(int, line.split()))
            res[(v[0], v[1])] = dict(zip(("XP", "RB", "RC", "RT", "RU", "SE", "L1", "L2"), v[2:]))
    return res


def _warp_cost(addrs):
    banks = defaultdict(set)
    for a in addrs:
        banks[a % 32].add(a)
    return max((len(s) for s in banks.values()), default=0)


def _wavefronts(L, D1, Q, NE):
    """(wavefronts, ideal) of one block of NE elements: the gather's stores
    and every stage's loads and stores, each pattern weighted by how many
    accesses of that shape a line makes."""
    QQ, N1, N2, ND = Q * Q, D1 * D1, D1 * Q, D1 ** 3
    NT = QQ * NE
    SE, XP, RB, RC, RT, RU = L["SE"], L["XP"], L["RB"], L["RC"], L["RT"], L["RU"]
    tot = ideal = 0

    def pattern(f, weight):
        nonlocal tot, ideal
        for w0 in range(0, NT, 32):
            a = [f(t) for t in range(w0, min(w0 + 32, NT))]
            a = [x for x in a if x is not None]
            if a:
                tot += weight * _warp_cost(a)
                ideal += weight

    def short(n, lanes, fn):
        return lambda tid: (tid // lanes) * SE + fn(tid % lanes) if tid // lanes < NE and tid % lanes < n else None

    for j in range((ND + QQ - 1) // QQ):
        pattern(lambda tid, j=j: None if (tid % QQ) + j * QQ >= ND else
                (tid // QQ) * SE + (((tid % QQ) + j * QQ) // D1) * XP + ((tid % QQ) + j * QQ) % D1, 1)
    pattern(short(N1, L["L1"], lambda t: t * XP), D1)                                   # S1 loads
    pattern(short(N1, L["L1"], lambda t: t), 2 * Q)                                     # S1 stores
    pattern(short(N2, L["L2"], lambda t: (t % Q) * RB + (t // Q) * D1), 2 * D1)        # S2 loads
    pattern(short(N2, L["L2"], lambda t: t), 3 * Q)                                     # S2 stores
    pattern(lambda tid: (tid // QQ) * SE + ((tid % QQ) // Q) * RC + (tid % QQ) % Q, 3 * D1)  # S3 loads
    pattern(lambda tid: (tid // QQ) * SE + tid % QQ, 3 * D1)                           # S3 stores
    pattern(short(N2, L["L2"], lambda t: (t // Q) * RT + t % Q), 3 * Q)                 # S4 loads
    pattern(short(N2, L["L2"], lambda t: t), 2 * D1)                                    # S4 stores
    pattern(short(N1, L["L1"], lambda t: (t % D1) * RU + (t // D1) * Q), 2 * Q)        # S5 loads
    return tot, ideal


@pytest.mark.parametrize("NE", [4, 7])
def test_p4_blocks_have_no_bank_replays(layouts, NE):
    """p = 4, q = 6: the single-problem FP32 block (4 elements) and the
    batch's tile (7 elements), one warp per element in the short stages."""
    L = layouts[(5, 6)]
    assert L["L1"] == 32 and L["L2"] == 32
    tot, ideal = _wavefronts(L, 5, 6, NE)
    assert tot == ideal, (tot, ideal)


def test_p2_half_warps_cut_the_replays(layouts):
    """p = 2, q = 4: a half-warp per element (two elements per warp) leaves
    some replays, but fewer wavefronts than the packed lines on the same
    slab stride."""
    L = layouts[(3, 4)]
    assert L["L1"] == 16 and L["L2"] == 16
    lanes, _ = _wavefronts(L, 3, 4, 16)
    packed, _ = _wavefronts(dict(L, L1=9, L2=12), 3, 4, 16)
    assert lanes <= 0.85 * packed, (lanes, packed)


@pytest.mark.parametrize("D1,Q", [(2, 3), (4, 5), (6, 7), (7, 8), (8, 9), (9, 10)])
def test_other_orders_keep_packed_lines(layouts, D1, Q):
    L = layouts[(D1, Q)]
    assert L["L1"] in (D1 * D1, 16) and L["L2"] in (D1 * Q,)
    assert L["L1"] == D1 * D1 or D1 * D1 == 16      # p = 3: 16 lines already fill a half-warp
