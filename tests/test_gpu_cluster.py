"""GPU parity of the binary64 sweeps with cluster-split visits (every visit of a block pair
split by rows over a thread-block cluster of 2, 4 or 8 CTAs) against the CPU oracle, and
against the single-CTA visits on the same matrices."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import (align_signs, check_factorization, check_sign_rule, elementwise_vs_oracle,
                            gpu_svd, sigma_gate)

pytestmark = pytest.mark.gpu


def _vs_oracle(A, mode, cs, **opts):
    U, S, V, st = gpu_svd(A, mode=mode, work_kernel="cluster", work_cluster=cs, **opts)
    assert st["status"] in (0, 8), st
    assert st["work_cluster"] >= cs and st["block_w_work"] == opts.get("block_w", 4), st
    oopts = {k: v for k, v in opts.items() if k in ("y_tol", "v_by_qr")}
    Uo, So, Vo, sto = oracle.svd(A, mode=mode, **oopts)
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    sigma_gate(A, S, So)
    gaps = np.minimum(np.r_[np.inf, -np.diff(So)], np.r_[-np.diff(So), np.inf]) / So
    sep = gaps >= 1e-3
    Ua, Va = align_signs(U, V, Uo, Vo)
    assert np.abs(Va[:, sep] - Vo[:, sep]).max(initial=0) <= 1e-8
    assert np.abs(Ua[:, sep] - Uo[:, sep]).max(initial=0) <= 1e-8
    return st, sto


@pytest.mark.parametrize("cs", [2, 4, 8])
@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_cluster_sweeps_against_oracle(mode, cs):
    """256 x 128 workload: 128 rows of Y split over 2, 4 or 8 CTAs (64, 32, 16 rows each)."""
    A, _ = inputs.plain_256x128()
    st, sto = _vs_oracle(A, mode, cs)
    assert st["sweeps_work"] <= sto["sweeps_work"] + 1


@pytest.mark.parametrize("w", [2, 8])
def test_cluster_block_widths(w):
    """Block widths 2 and 8 of the cluster form (16 and 4 rows per thread) against the oracle,
    on the 256 x 128 workload and on a ragged 200-column matrix."""
    A, _ = inputs.plain_256x128()
    st, _ = _vs_oracle(A, "mixed", 4, block_w=w)
    assert st["block_w_work"] == w
    rng = np.random.default_rng(320 + w)
    B = inputs.known_sigma(rng, 230, 200, np.logspace(0, -4, 200))
    st, _ = _vs_oracle(B, "mixed", 2, block_w=w)
    assert st["block_w_work"] == w


@pytest.mark.parametrize("n", [1, 2, 5, 7, 33, 130])
def test_cluster_ragged_shapes(n):
    """Column counts that leave phantom blocks and rows that split unevenly (n = 7 over 8 CTAs:
    one row each, one CTA without rows)."""
    rng = np.random.default_rng(300 + n)
    m = n + n // 3 + 1
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -4, n))
    _vs_oracle(A, "mixed", 8 if n == 7 else 2)


@pytest.mark.parametrize("opts", [dict(v_by_qr=1), dict(y_tol=1e-6)])
def test_cluster_refinement_variants(opts):
    """The V-free refinement with V from QR(X^T U_X), and the Y1/Y2 safeguard's filtered
    sweeps, on cluster-split visits, against the oracle with the same options."""
    A, _ = inputs.plain_256x128()
    st, sto = _vs_oracle(A, "mixed", 4, **opts)
    if opts.get("v_by_qr"):
        assert st["sweeps_v"] >= 1
    if opts.get("y_tol"):
        assert st["y2_cols"] > 0


@pytest.mark.parametrize("cs", [4, 8])
def test_cluster_large_recipe_against_oracle(cs):
    """The 8192 x 8192 workload's recipe at n = 768 on 4- and 8-CTA visits (192 and 96 rows
    each) against the binary64 oracle element by element (kappa(B) = 1e2: the binary64 floor
    is far below 1e-12)."""
    A = inputs.large_8192(n=768)
    Uo, So, Vo, sto = oracle.svd(A, mode="mixed")
    U, S, V, st = gpu_svd(A, mode="mixed", work_kernel="cluster", work_cluster=cs)
    assert st["status"] == 0 and st["work_cluster"] == cs, st
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    elementwise_vs_oracle(U, S, V, So, Uo, Vo)


@pytest.mark.parametrize("cs", [0, 4, 8])
def test_cluster_against_single_cta_visits(cs):
    """2304 x 2304 (large recipe): more rows than one CTA's registers hold at block width 4, so
    the automatic choice takes clusters (4 CTAs: at most 1024 rows each); 4 and 8 CTAs per
    visit against single-CTA visits (block width 2): the same singular values to 1e-12, the
    bars on both."""
    A = inputs.large_8192(n=2304)
    U0, S0, V0, st0 = gpu_svd(A, mode="mixed", work_kernel="cta")
    assert st0["status"] == 0 and st0["work_cluster"] == 1
    U1, S1, V1, st1 = gpu_svd(A, mode="mixed", work_kernel="auto" if cs == 0 else "cluster", work_cluster=cs)
    assert st1["status"] == 0
    assert st1["work_cluster"] == (4 if cs == 0 else cs) and st1["block_w_work"] == 4, st1
    check_factorization(A, U1, S1, V1)
    assert np.max(np.abs(S1 - S0) / S0) <= 1e-12
    assert st1["sweeps_work"] <= st0["sweeps_work"] + 1


def test_cluster_deterministic():
    """Two calls: bit-identical outputs (every cross-CTA sum is taken in rank order)."""
    A = inputs.large_8192(n=600)
    r0 = gpu_svd(A, mode="mixed", work_kernel="cluster", work_cluster=4)
    r1 = gpu_svd(A, mode="mixed", work_kernel="cluster", work_cluster=4)
    for a, b in zip(r0[:3], r1[:3]):
        assert np.array_equal(a, b)
