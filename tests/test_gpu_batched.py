"""GPU parity of the batched path (one persistent launch, one CTA per matrix) against the
CPU oracle and against the single-matrix GPU path, on seeded uneven batches."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import (U64, align_signs, check_factorization, check_sign_rule, gpu_svd,
                            sigma_gate)

pytestmark = pytest.mark.gpu


def _run_batched(mats, mode):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(mode=mode)
    dmats = [mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")) for A in mats]
    Us, Ss, Vs, info = h.svd_batched(dmats)
    torch.cuda.synchronize()
    out = ([u.cpu().numpy() for u in Us], [s.cpu().numpy() for s in Ss],
           [v.cpu().numpy() for v in Vs], info.cpu().numpy())
    h.close()
    return out


def _small_batch(seed, count, nmax):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count):
        n = int(rng.integers(1, nmax + 1))
        m = n + int(rng.integers(0, n + 1))
        kappa = 10.0 ** rng.uniform(1, 6)
        mats.append(inputs.known_sigma(rng, m, n, np.logspace(0, -np.log10(kappa), n)))
    return mats


@pytest.mark.parametrize("mode", ["mixed", "plain", "auto"])
def test_batched_against_oracle(mode):
    mats = _small_batch(40, 24, 48)
    Us, Ss, Vs, info = _run_batched(mats, mode)
    assert np.all(info == 0), info
    for A, U, S, V in zip(mats, Us, Ss, Vs):
        check_factorization(A, U, S, V)
        check_sign_rule(V)
        Uo, So, Vo, _ = oracle.svd(A, mode=mode)
        sigma_gate(A, S, So)
        gaps = np.minimum(np.r_[np.inf, -np.diff(So)], np.r_[-np.diff(So), np.inf]) / So
        sep = gaps >= 1e-3
        Ua, Va = align_signs(U, V, Uo, Vo)
        assert np.abs(Va[:, sep] - Vo[:, sep]).max(initial=0) <= 1e-8
        assert np.abs(Ua[:, sep] - Uo[:, sep]).max(initial=0) <= 1e-8


def test_batched_agrees_with_single_matrix_path():
    """Matrices of the uneven-batch recipe (n up to 256): batched vs single-matrix GPU path,
    both with the binary64 QRCP (the batched kernel's); Alg. 5's pivots give a different R and
    hence different rounding, which the accuracy tests bound against the extended oracle."""
    mats_all, sig_all, m, n, kappa = inputs.batch_matrices(count=12)
    mats = [A for A, k in zip(mats_all, kappa)]
    Us, Ss, Vs, info = _run_batched(mats, "mixed")
    assert np.all(info == 0)
    for A, U, S, V in zip(mats, Us, Ss, Vs):
        check_factorization(A, U, S, V)
        U1, S1, V1, st = gpu_svd(A, mode="mixed", qrcp="f64")
        assert np.max(np.abs(S - S1) / S1) <= 1e-12
        gaps = np.minimum(np.r_[np.inf, -np.diff(S1)], np.r_[-np.diff(S1), np.inf]) / S1
        sep = gaps >= 1e-3
        Ua, Va = align_signs(U, V, U1, V1)
        assert np.abs(Va[:, sep] - V1[:, sep]).max(initial=0) <= 1e-8


def test_batched_edge_cases():
    rng = np.random.default_rng(41)
    mats = [np.array([[3.0], [4.0]]),                         # n = 1
            np.diag([2.0, -1.0, 0.5]),                          # diagonal, m = n
            inputs.orthonormal(rng, 20, 10) * 2.0,             # cond_R = 1
            rng.standard_normal((8, 8))]
    mats[3][:, 2] = 0.0                                         # zero column
    Us, Ss, Vs, info = _run_batched(mats, "auto")
    assert np.allclose(Ss[0], [5.0], rtol=4 * U64)
    assert np.allclose(Ss[1], [2.0, 1.0, 0.5], rtol=4 * U64)
    assert info[3] & 8 and Ss[3][-1] == 0.0
    for A, U, S, V in zip(mats[:3], Us[:3], Ss[:3], Vs[:3]):
        check_factorization(A, U, S, V)
    bad = [np.ones((4, 3))]
    bad[0][1, 1] = np.inf
    _, Sb, _, infob = _run_batched(bad + [mats[2]], "auto")
    assert infob[0] & 2 and infob[1] == 0
