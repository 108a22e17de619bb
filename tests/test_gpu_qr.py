"""Blocked Householder QR (mpjsvd_geqrf) and the compact-WY application of Q (mpjsvd_apply_q)
against the oracle's unblocked Householder QR (Section 3.1 preconditioning; Section 3.3 QR of
the switch), through the C ABI.

The reflectors are unique given the sign convention (beta = -sign(alpha)|x|), so R, tau and the
reflector tails are compared element by element; Q is checked through Q R = A and Q^T Q = I.
Sizes cover one and many panels, ragged last panels and row chunks, square and tall shapes,
the 2048 x 1024 workload's size and a tall case that takes 16-column panels.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import U64

pytestmark = pytest.mark.gpu

CASES = [(40, 7), (64, 64), (256, 128), (300, 300), (1000, 333), (2048, 1024), (6400, 70)]


def _gpu_qr(A):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.default_handle()
    QR, tau = h.geqrf(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    return h, QR, tau


@pytest.mark.parametrize("m,n", CASES)
def test_geqrf_matches_oracle(m, n):
    rng = np.random.default_rng(m * 7919 + n)
    A = rng.standard_normal((m, n))
    _, QR, tau = _gpu_qr(A)
    QRg, taug = QR.cpu().numpy(), tau.cpu().numpy()
    QRo, tauo = oracle.geqrf(A)
    scale = np.abs(A).max() * np.sqrt(m)
    R_g, R_o = np.triu(QRg[:n]), np.triu(QRo[:n])
    assert np.abs(R_g - R_o).max() <= 1e-13 * scale
    assert np.abs(taug - tauo).max() <= 1e-13
    tail = np.tril(np.ones((m, n)), -1).astype(bool)
    assert np.abs(QRg[tail] - QRo[tail]).max() <= 1e-12


@pytest.mark.parametrize("m,n", [(256, 128), (1000, 333), (2048, 1024)])
def test_apply_q_reconstructs_and_is_orthogonal(m, n):
    import torch
    rng = np.random.default_rng(m + 3 * n)
    A = rng.standard_normal((m, n))
    h, QR, tau = _gpu_qr(A)
    R0 = np.zeros((m, n))
    R0[:n] = np.triu(QR.cpu().numpy()[:n])
    QRv = QR.cpu().numpy()
    # Q [R; 0] = A
    QRr = h.apply_q(QR, tau, torch.from_numpy(R0).cuda()).cpu().numpy()
    assert np.linalg.norm(QRr - A) / np.linalg.norm(A) <= 1e-14
    # thin Q = Q I(:, :n): orthonormal columns, and equal to the oracle's Q
    I = np.eye(m, n)
    Qg = h.apply_q(QR, tau, torch.from_numpy(I).cuda()).cpu().numpy()
    assert np.abs(Qg.T @ Qg - np.eye(n)).max() <= 64 * n * U64
    Qo = oracle.apply_q(QRv, tau.cpu().numpy(), I)
    assert np.abs(Qg - Qo).max() <= 1e-13


def test_apply_q_on_a_wide_block_with_fewer_reflectors():
    import torch
    rng = np.random.default_rng(5)
    m, k, nc = 700, 90, 257
    A = rng.standard_normal((m, k))
    h, QR, tau = _gpu_qr(A)
    C = rng.standard_normal((m, nc))
    Cg = h.apply_q(QR, tau, torch.from_numpy(C).cuda()).cpu().numpy()
    Co = oracle.apply_q(QR.cpu().numpy(), tau.cpu().numpy(), C)
    assert np.abs(Cg - Co).max() <= 1e-13 * np.abs(C).max() * np.sqrt(m)


def test_geqrf_zero_column_and_rank_deficiency():
    # a zero column gives tau = 0 and v = e_j; a last column equal to an earlier one leaves
    # only rounding noise on R's last diagonal entry
    rng = np.random.default_rng(9)
    A = rng.standard_normal((200, 40))
    A[:, 5] = 0.0
    A[:, 39] = A[:, 3]
    _, QR, tau = _gpu_qr(A)
    QRg = QR.cpu().numpy()
    QRo, tauo = oracle.geqrf(A)
    assert tau.cpu().numpy()[5] == 0.0 and tauo[5] == 0.0
    scale = np.abs(A).max() * np.sqrt(200)
    Rg, Ro = np.triu(QRg[:40]), np.triu(QRo[:40])
    assert abs(Rg[39, 39]) <= 1e-13 * scale and abs(Ro[39, 39]) <= 1e-13 * scale
    Rg[39, 39] = Ro[39, 39] = 0.0
    assert np.abs(Rg - Ro).max() <= 1e-13 * scale
