"""The seeded input recipes against the paper's tables (host only).

Table 2 defines the XLATM1 modes for D = diag(d) with condition number kappa; Table 1 lists
the sixteen (MODE of D, MODE of Sigma) pairs (fixture `golden/table1_modes.txt`, typed from
Table 1)."""
import os

import numpy as np
import pytest

from paper_2209_04626_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("n", [2, 7, 64])
@pytest.mark.parametrize("kappa", [1e2, 1e12, 1e20])
def test_xlatm1_modes_table2(n, kappa):
    rng = np.random.default_rng(5)
    i = np.arange(1, n + 1, dtype=np.float64)
    d1 = inputs.xlatm1(rng, 1, n, kappa)  # clustered at 1/kappa: d(1) = 1, d(2:n) = 1/kappa
    assert d1[0] == 1.0 and np.all(d1[1:] == 1.0 / kappa)
    d2 = inputs.xlatm1(rng, 2, n, kappa)  # clustered at 1: d(1:n-1) = 1, d(n) = 1/kappa
    assert np.all(d2[:-1] == 1.0) and d2[-1] == 1.0 / kappa
    d3 = inputs.xlatm1(rng, 3, n, kappa)  # geometric: d(i) = kappa^(-(i-1)/(n-1))
    assert np.allclose(np.log(d3), -(i - 1) / (n - 1) * np.log(kappa), rtol=0, atol=1e-12)
    d4 = inputs.xlatm1(rng, 4, n, kappa)  # arithmetic: d(i) = 1 - (i-1)/(n-1) (1 - 1/kappa)
    assert np.allclose(d4, 1.0 - (i - 1) / (n - 1) * (1.0 - 1.0 / kappa), rtol=1e-15, atol=1e-15)
    assert np.all(np.diff(d4) < 0) or n < 2
    for d in (d1, d2, d3, d4):  # condition number kappa exactly (up to rounding)
        assert abs(d.max() / d.min() / kappa - 1.0) < 1e-12
    d5 = inputs.xlatm1(rng, 5, n, kappa)  # log-random in (1/kappa, 1)
    assert np.all(d5 > 1.0 / kappa) and np.all(d5 < 1.0)


def test_xlatm1_mode5_log_uniform():
    """Mode 5: the logarithms are uniform on (-log kappa, 0): mean and spread of many draws."""
    rng = np.random.default_rng(6)
    kappa, n = 1e8, 200000
    x = np.log(inputs.xlatm1(rng, 5, n, kappa)) / np.log(kappa)  # uniform on (-1, 0)
    assert abs(x.mean() + 0.5) < 5e-3 and abs(x.var() - 1.0 / 12.0) < 2e-3


def test_table1_pairs():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table1_modes.txt"))
            if l.strip() and not l.startswith("#")]
    assert [(int(r[1]), int(r[2])) for r in rows] == inputs.TABLE1
    assert [int(r[0]) for r in rows] == list(range(1, 17))


def test_table1_matrix_structure():
    """A = B D: the column norms of A are |B e_j| d_j with B = W1 diag(Sigma) W2^T; the singular
    values of B are Sigma (mode 3 of Sigma, kappa(B) = 1e4) and D has the requested extremes."""
    rng = np.random.default_rng(7)
    n = 40
    A = inputs.table1_pair(rng, n, 2, 3, 1e6, 1e4)
    rng2 = np.random.default_rng(7)
    d = inputs.xlatm1(rng2, 2, n, 1e6)
    s = inputs.xlatm1(rng2, 3, n, 1e4)
    B = A / d[None, :]
    sb = np.linalg.svd(B, compute_uv=False)
    assert np.allclose(sb, np.sort(s)[::-1], rtol=1e-12, atol=0)
