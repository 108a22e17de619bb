"""The rank-revealing QR of the preconditioning on the GPU (mpjsvd_geqp3): the mixed-precision
RRQR of Alg. 5 (binary32 pivot search, binary64 QR of A P) and the binary64 Businger-Golub
kernel, against the oracle.

Pivots are compared exactly where the order is decided by margins far above binary32
rounding (strongly graded columns); elsewhere binary32 rounding order may pick a different
column among near-ties, so the test checks what is unique: the permutation is valid, every
pivot had the largest remaining norm up to binary32 rounding, and R equals the oracle's
binary64 QR of A P for the GPU's own P, element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu_geqp3(A, qrcp):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(qrcp=qrcp)
    QR, jpvt, tau = h.geqp3(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    st = h.stats()
    out = QR.cpu().numpy(), jpvt.cpu().numpy(), tau.cpu().numpy(), st
    h.close()
    return out


def _graded(rng, m, n, ratio):
    return rng.standard_normal((m, n)) * (ratio ** -np.arange(n))[rng.permutation(n)]


@pytest.mark.parametrize("qrcp,m,n", [(q, m, n) for q in ("mixed", "f64")
                                      for m, n in [(60, 30), (300, 200), (2048, 1024)]] +
                         [("mixed", 10300, 610)])
def test_pivots_exact_on_graded_columns(qrcp, m, n):
    """(10300, 610): columns too long for the register- and shared-memory-resident binary32
    search, so Alg. 5 keeps them in global memory."""
    rng = np.random.default_rng(m + n)
    A = _graded(rng, m, n, 10.0 ** (min(30, 200) / n * 0.6 + 0.02)) if n > 30 else _graded(rng, m, n, 10.0)
    QR, jpvt, tau, st = _gpu_geqp3(A, qrcp)
    assert st["qrcp"] == (0 if qrcp == "mixed" else 1)
    jo = oracle.qrcp_pivots_f32(A) if qrcp == "mixed" else oracle.geqp3(A)[1]
    assert np.array_equal(jpvt, jo)


@pytest.mark.parametrize("qrcp,m,n", [(q, m, n) for q in ("mixed", "f64")
                                      for m, n in [(200, 120), (1000, 333), (2048, 1024)]] +
                         [("mixed", 10300, 610)])
def test_rrqr_property_and_r_parity(qrcp, m, n):
    rng = np.random.default_rng(7 * m + n)
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -5, n)) * rng.uniform(0.1, 10.0, n)
    QR, jpvt, tau, st = _gpu_geqp3(A, qrcp)
    assert sorted(jpvt.tolist()) == list(range(n))
    R = np.triu(QR[:n])
    # every pivot had the largest remaining norm, up to the accuracy of the norms the search
    # compares: the downdated norms are recomputed only once a downdate has lost about sqrt(u)
    # (2^-12 in binary32, 2^-26.5 in binary64), so the choice is exact to about 2 sqrt(u)
    # relative; and the remaining columns themselves carry the search precision's rounding of
    # m-term dot products, about m u |a_k| absolute (binary32: what Alg. 5 trades for speed)
    slack = 2 * 2.0 ** -12 if qrcp == "mixed" else 2 * 2.0 ** -26.5
    u_s = 2.0 ** -24 if qrcp == "mixed" else 2.0 ** -53
    absl = m * u_s * np.linalg.norm(A, axis=0).max()
    rem = np.sqrt(np.cumsum((R ** 2)[::-1], axis=0)[::-1])  # rem[j, k] = |R(j:, k)|
    for j in range(n):
        assert abs(R[j, j]) >= (1 - slack) * rem[j, j:].max() - absl, j
    # R and the reflectors equal the oracle's binary64 QR of A P for the GPU's P
    QRo, tauo = oracle.geqrf(A[:, jpvt])
    scale = np.abs(A).max() * np.sqrt(m)
    assert np.abs(R - np.triu(QRo[:n])).max() <= 1e-12 * scale
    assert np.abs(tau - tauo).max() <= 1e-10  # tau in [1, 2]; inputs with kappa up to ~1e7


def test_mixed_rrqr_extreme_scales_and_zero_columns():
    rng = np.random.default_rng(3)
    A = _graded(rng, 200, 60, 3.0)
    A[:, 7] = 0.0
    # far outside binary32's range, inside the range where binary64 squares stay finite
    for s in (2.0 ** 400, 2.0 ** -400):
        QR, jpvt, tau, st = _gpu_geqp3(A * s, "mixed")
        assert st["qrcp"] == 0
        assert np.array_equal(jpvt, oracle.qrcp_pivots_f32(A * s))
        assert jpvt[-1] == 7 and tau[-1] == 0.0
