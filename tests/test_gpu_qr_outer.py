"""The two-level blocked Householder QR (256-column outer blocks, their trailing updates and the
applications of Q in the compact UT form with the binary64 products on the bf16 tensor cores):
against the oracle's Householder QR, against the one-level binary64 form, and the whole SVD
with it against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import (U64, check_factorization, check_sign_rule, elementwise_vs_oracle, gpu_svd,
                            sigma_gate)

pytestmark = pytest.mark.gpu


def _qr(A, mode):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(qr_update=mode)
    QR, tau = h.geqrf(torch.from_numpy(A).cuda())
    out = QR.cpu().numpy(), tau.cpu().numpy()
    h.close()
    return out


def _graded(rng, m, n, decades):
    A = rng.standard_normal((m, n))
    return A * 10.0 ** rng.uniform(-decades, 0, n)


@pytest.mark.parametrize("m,n", [(700, 600), (1030, 777), (600, 600)])
def test_geqrf_two_level_against_oracle(m, n):
    """R and the reflectors against the oracle's Householder QR, column by column relative to
    the column's norm (graded columns over 8 decades: the error must stay columnwise, as in
    binary64); tau to a few ulps."""
    rng = np.random.default_rng(m + 3 * n)
    A = _graded(rng, m, n, 8)
    QR, tau = _qr(A, "tc")
    QRo, tauo = oracle.geqrf(A)
    cn = np.linalg.norm(A, axis=0)
    R, Ro = np.triu(QR[:n]), np.triu(QRo[:n])
    assert np.max(np.abs(R - Ro) / cn[None, :]) <= 256 * m * U64
    assert np.max(np.abs(tau - tauo)) <= 16 * m * U64
    Vt, Vo = np.tril(QR, -1), np.tril(QRo, -1)
    assert np.max(np.abs(Vt - Vo)) <= 1e-10


@pytest.mark.parametrize("m,n", [(900, 700), (600, 520)])
def test_apply_q_two_level(m, n):
    """Q (formed by applying Q to the identity) orthogonal to binary64 precision and Q R = A,
    against the one-level form on the same reflectors."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    rng = np.random.default_rng(11 + m)
    A = _graded(rng, m, n, 6)
    QR, tau = _qr(A, "tc")
    I = np.eye(m, n)
    outs = {}
    for mode in ("tc", "f64"):
        h = mpjsvd.Handle(qr_update=mode)
        outs[mode] = h.apply_q(torch.from_numpy(QR).cuda(), torch.from_numpy(tau).cuda(),
                               torch.from_numpy(I).cuda()).cpu().numpy()
        h.close()
    Q = outs["tc"]
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 32 * m * U64
    R = np.triu(QR[:n])
    # column by column: the backward error of each column relative to its own norm
    assert np.all(np.linalg.norm(Q @ R - A, axis=0) <= 64 * m * U64 * np.linalg.norm(A, axis=0))
    assert np.max(np.abs(Q - outs["f64"])) <= 1e-12


@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_svd_with_two_level_qr_against_oracle(mode):
    """420 x 300 (an outer block of 256 columns and a ragged one of 44), sigma over 5 decades:
    every QR and application of Q in the pipeline (the preconditioner's, the switch's, U) in
    the two-level form."""
    rng = np.random.default_rng(21)
    A = inputs.known_sigma(rng, 420, 300, np.logspace(0, -5, 300))
    U, S, V, st = gpu_svd(A, mode=mode, qr_update="tc")
    assert st["status"] == 0, st
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    Uo, So, Vo, _ = oracle.svd(A, mode=mode)
    sigma_gate(A, S, So)


def test_large_recipe_two_level_qr_against_oracle():
    """The 8192 x 8192 workload's recipe at n = 1024 (graded columns over 10 decades) with the
    two-level QRs against the binary64 oracle element by element."""
    A = inputs.large_8192(n=1024)
    Uo, So, Vo, sto = oracle.svd(A, mode="mixed")
    U, S, V, st = gpu_svd(A, mode="mixed", qr_update="tc")
    assert st["status"] == 0, st
    check_factorization(A, U, S, V)
    elementwise_vs_oracle(U, S, V, So, Uo, Vo)


def test_precision_workload_two_level_qr_against_oracle():
    A = inputs.precision_2048x1024()
    Uo, So, Vo, sto = oracle.svd(A, mode="mixed")
    U, S, V, st = gpu_svd(A, mode="mixed", qr_update="tc")
    assert st["status"] == 0, st
    check_factorization(A, U, S, V)
    elementwise_vs_oracle(U, S, V, So, Uo, Vo)
