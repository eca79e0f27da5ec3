"""The C CSR product of the oracle (oracle/spmv.c, the timed all-cores CPU
baseline) against the oracle's own scipy product and a dense product: the
result is independent of the thread count (bit for bit) and agrees with
scipy and with the dense matrix to rounding."""

import os

import numpy as np
import pytest

from fem_inputs import hex_lattice, lognormal, x_uniform
from oracle import assemble, cspmv


@pytest.mark.parametrize("p", [1, 3])
def test_c_spmv_matches_scipy_and_dense(p):
    c, h = hex_lattice(3, 0.15, seed=3, shuffle=True)
    prob = assemble.Problem(c, h, p, p + 2, kappa=lognormal(4, h.shape[0]))
    K = prob.K
    x = x_uniform(5, prob.ndof)
    A = cspmv.CSR(K)
    y1 = A.apply(x, 1)
    nt = max(2, min(8, os.cpu_count() or 2))
    yn = A.apply(x, nt)
    assert np.array_equal(y1, yn)
    ys = K @ x
    scale = np.abs(ys).max()
    assert np.abs(y1 - ys).max() <= 1e-14 * scale
    yd = K.toarray() @ x
    assert np.abs(y1 - yd).max() <= 1e-13 * scale


def test_c_spmv_rejects_bad_thread_count():
    import scipy.sparse as sp
    A = cspmv.CSR(sp.identity(3, format="csr"))
    assert np.array_equal(A.apply(np.arange(3.0), 1), np.arange(3.0))
    with pytest.raises(ValueError):
        A.apply(np.arange(3.0), 0)
