"""GPU parity at the full sizes the bench times: the 2048 x 1024 precision workload (single
matrix, the bench's launch configuration) and the 4096-matrix uneven batch (one persistent
launch). The oracle cannot run the whole workloads in a test's time, so these check properties
that hold at any size (orthogonality, backward error, mixed vs plain binary64 path, the leading
singular values against LAPACK where LAPACK is relatively accurate) and compare a seeded
sample of the batch's matrices with the oracle one by one."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import check_factorization, check_sign_rule, gpu_svd, sigma_gate

pytestmark = pytest.mark.gpu


def test_precision_2048x1024_full():
    A = inputs.precision_2048x1024()
    U, S, V, st = gpu_svd(A, "mixed")
    assert st["status"] == 0 and st["branch"] == 0, st
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    Up, Sp, Vp, stp = gpu_svd(A, "plain")
    assert stp["status"] == 0
    assert np.max(np.abs(S - Sp) / Sp) <= 1e-12
    # LAPACK's singular values are accurate to a modest multiple of u sigma_max absolutely:
    # compare the leading ones (89 values >= 0.1 sigma_max, LAPACK's relative error there a
    # small multiple of 1e-15)
    s_lapack = np.linalg.svd(A, compute_uv=False)
    lead = s_lapack >= 0.1 * s_lapack[0]
    assert lead.sum() > 10
    U64 = 2.0 ** -53
    assert np.all(np.abs(S[lead] - s_lapack[lead]) <= 1e-12 * s_lapack[lead] + 64 * U64 * s_lapack[0])


def test_batched_4096_full():
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    mats, sigmas, m, n, kappa = inputs.batch_matrices()
    h = mpjsvd.Handle(mode="mixed")
    dmats = [mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")) for A in mats]
    Us, Ss, Vs, info = h.svd_batched(dmats)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert np.all(info == 0), np.nonzero(info)
    # every matrix: the factorization bars; a seeded sample well inside the sigma bar's domain
    # (kappa <= 1e4, where the binary64 floor is far below 1e-12) and small enough for the
    # extended-precision oracle: one by one against it
    for i in range(len(mats)):
        check_factorization(mats[i], Us[i].cpu().numpy(), Ss[i].cpu().numpy(), Vs[i].cpu().numpy())
    eligible = [i for i in range(len(mats)) if n[i] <= 96 and kappa[i] <= 1e4]
    rng = np.random.default_rng(77)
    for i in rng.choice(eligible, size=12, replace=False):
        A = mats[i]
        U, S, V = Us[i].cpu().numpy(), Ss[i].cpu().numpy(), Vs[i].cpu().numpy()
        check_factorization(A, U, S, V)
        check_sign_rule(V)
        _, So, _, _ = oracle.svd(A, mode="mixed", qrcp=0)
        sigma_gate(A, S, So)
    h.close()
