"""Binary64 products on the bf16 tensor cores by error-free operand splitting (the Ozaki
scheme), standalone against numpy's binary64 product and inside the SVD (the precision switch
of Section 3.3 and the n x n products of Section 3.4) against the FP64-pipe path and the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import check_factorization, check_sign_rule, gpu_svd, sigma_gate

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def _dgemm_tc(A, B, transA):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    dev = torch.device("cuda")
    Ad = mpjsvd.colmajor(torch.from_numpy(A), dev)
    Bd = mpjsvd.colmajor(torch.from_numpy(B), dev)
    M = A.shape[1] if transA else A.shape[0]
    K, N = B.shape
    C = mpjsvd.empty_colmajor(M, N, dev)
    h = mpjsvd.Handle()
    rc = mpjsvd.mpjsvd_dgemm_tc(h.h, M, N, K, Ad.data_ptr(), Ad.stride(1), 1 if transA else 0, Bd.data_ptr(),
                                Bd.stride(1), C.data_ptr(), C.stride(1))
    assert rc == 0, mpjsvd.mpjsvd_last_error()
    st = h.stats()
    assert st["status"] == 0, st
    out = C.cpu().numpy()
    h.close()
    return out


@pytest.mark.parametrize("M,N,K,transA", [(128, 64, 16, False), (300, 70, 1000, False), (1, 1, 1, False),
                                          (257, 129, 513, True), (1024, 1024, 1024, True),
                                          (2048, 96, 4100, False)])
def test_dgemm_tc_against_binary64(M, N, K, transA):
    """Each entry within 8 K 2^-53 max_k |op(A)_ik| max_k |B_kj| of numpy's binary64 product
    (the splitting keeps 56 bits of every row and column relative to its maximum; entries
    graded over 10 decades, ragged tiles, k ranges spanning several exact 512-k chunks)."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    opA = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-5, 5, (M, 1)) * 10.0 ** rng.uniform(-3, 0, (1, K))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-5, 5, (1, N))
    A = np.asfortranarray(opA.T) if transA else np.asfortranarray(opA)
    C = _dgemm_tc(A, np.asfortranarray(B), transA)
    ref = opA @ B
    bound = 8 * K * U64 * np.outer(np.abs(opA).max(axis=1), np.abs(B).max(axis=0))
    err = np.abs(C - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and as accurate as binary64 itself where the entries are balanced: relative error of the
    # well-conditioned entries near the unit roundoff
    bal = np.abs(ref) > 0.1 * np.sqrt(K) * np.outer(np.abs(opA).max(axis=1), np.abs(B).max(axis=0))
    if bal.any():
        assert np.max(err[bal] / np.abs(ref[bal])) <= 64 * U64


def test_dgemm_tc_exact_on_integers():
    """Integer operands whose products and sums are exact in binary64: the split product is
    exact too (every slice product and every partial sum of the exact classes is exact)."""
    rng = np.random.default_rng(90)
    A = rng.integers(-2 ** 20, 2 ** 20, (200, 700)).astype(np.float64)
    B = rng.integers(-2 ** 20, 2 ** 20, (700, 90)).astype(np.float64)
    C = _dgemm_tc(np.asfortranarray(A), np.asfortranarray(B), False)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("n", [200, 1024])
def test_switch_on_tensor_cores_against_fp64_pipe_and_oracle(n):
    """The mixed SVD with the switch's products on the tensor cores and on the FP64 pipe: the
    same singular values to 1e-12, both meeting every bar, the tensor-core one against the
    oracle."""
    if n == 1024:
        A = inputs.precision_2048x1024()
    else:
        A = inputs.known_sigma(np.random.default_rng(91), n + 40, n, np.logspace(0, -5, n))
    U, S, V, st = gpu_svd(A, "mixed", gemm_kernel="tc")
    U2, S2, V2, st2 = gpu_svd(A, "mixed", gemm_kernel="f64")
    assert st["status"] == 0 and st2["status"] == 0
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    assert np.max(np.abs(S - S2) / S2) <= 1e-12
    assert st["sweeps_work"] <= st2["sweeps_work"] + 1
    if n <= 256:
        _, So, _, _ = oracle.svd(A, mode="mixed")
        sigma_gate(A, S, So)


@pytest.mark.parametrize("opts", [dict(v_by_qr=1), dict(y_tol=1e-6)])
def test_refinement_variants_on_tensor_cores(opts):
    A, _ = inputs.plain_256x128()
    U, S, V, st = gpu_svd(A, "mixed", gemm_kernel="tc", **opts)
    _, So, _, _ = oracle.svd(A, mode="mixed", **opts)
    assert st["status"] == 0
    check_factorization(A, U, S, V)
    sigma_gate(A, S, So)
