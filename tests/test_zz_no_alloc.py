"""The allocation-free entry point (mpjsvd_svd_noalloc) against the handle-based
mpjsvd_svd and the oracle, through the C ABI.

mpjsvd_svd_noalloc serves callers that cannot allocate device memory (an allocator that owns
the GPU's memory up front, loops where an allocation's implicit synchronization is not
acceptable): its scratch is a static device array shared by every call, so it takes no
handle and never calls cudaMalloc.
This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test. It must pass in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import U64, align_signs, check_factorization, sigma_gate

pytestmark = pytest.mark.gpu


def _noalloc(A, stream=None, with_status=True):
    """One call through the C ABI; returns (U, S, V, status) on the host."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    m, n = A.shape
    Ad = mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda"))
    U = mpjsvd.empty_colmajor(m, n, Ad.device)
    S = torch.empty(n, dtype=torch.float64, device=Ad.device)
    V = mpjsvd.empty_colmajor(n, n, Ad.device)
    status = torch.full((1,), -1, dtype=torch.int32, device=Ad.device)
    torch.cuda.synchronize()
    sptr = status.data_ptr() if with_status else None
    rc = mpjsvd.mpjsvd_svd_noalloc(m, n, Ad.data_ptr(), m, U.data_ptr(), S.data_ptr(),
                                   V.data_ptr(), 0.0, sptr,
                                   stream.cuda_stream if stream is not None else None)
    assert rc == 0, mpjsvd.mpjsvd_last_error()
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), int(status.item())


def _handle(A):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(mode="auto")
    Ad = mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda"))
    U, S, V = [t.cpu().numpy() for t in h.svd(Ad)]
    st = h.stats()
    h.close()
    assert st["status"] == 0
    return U, S, V


def test_noalloc_at_its_maximum_size():
    rng = np.random.default_rng(32)
    A = inputs.known_sigma(rng, 512, 256, np.logspace(0, -4, 256))
    U, S, V, status = _noalloc(A)
    assert status == 0
    Ur, Sr, Vr = _handle(A)
    check_factorization(A, U, S, V)
    assert np.max(np.abs(S - Sr) / Sr) <= 1e-12


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    rng = np.random.default_rng(31)
    cases = [inputs.known_sigma(rng, 300, 200, np.logspace(0, -5, 200)),
             inputs.known_sigma(rng, 96, 64, np.logspace(0, -2, 64))]
    for A in cases:  # two calls in a row on the shared scratch, different shapes
        U, S, V, status = _noalloc(A)
        assert status == 0
        Ur, Sr, Vr = _handle(A)
        n = A.shape[1]
        check_factorization(A, U, S, V)
        assert np.max(np.abs(S - Sr) / Sr) <= 1e-12
        Ua, Va = align_signs(U, V, Ur, Vr)
        assert np.abs(Va - Vr).max() <= 1e-8
        assert np.abs(Ua - Ur).max() <= 1e-8
        assert np.abs(U.T @ U - np.eye(n)).max() <= 64 * n * U64


def test_noalloc_against_the_oracle():
    rng = np.random.default_rng(33)
    A = inputs.known_sigma(rng, 200, 120, np.logspace(0, -4, 120))
    U, S, V, status = _noalloc(A)
    assert status == 0
    Uo, So, Vo, _ = oracle.svd(A, mode="auto")
    check_factorization(A, U, S, V)
    sigma_gate(A, S, So)
    Ua, Va = align_signs(U, V, Uo, Vo)
    assert np.abs(Va - Vo).max() <= 1e-8
    assert np.abs(Ua - Uo).max() <= 1e-8


def test_noalloc_allocates_no_device_memory_and_honours_the_stream():
    import torch
    rng = np.random.default_rng(34)
    A = inputs.known_sigma(rng, 160, 96, np.logspace(0, -3, 96))
    U0, S0, V0, st0 = _noalloc(A)  # warm call (first-use set-up done)
    assert st0 == 0
    # device memory the driver reports free, around a call whose buffers already exist
    from paper_2209_04626_gb300 import mpjsvd
    m, n = A.shape
    Ad = mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda"))
    U = mpjsvd.empty_colmajor(m, n, Ad.device)
    S = torch.empty(n, dtype=torch.float64, device=Ad.device)
    V = mpjsvd.empty_colmajor(n, n, Ad.device)
    status = torch.full((1,), -1, dtype=torch.int32, device=Ad.device)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with torch.cuda.stream(side):
        rc = mpjsvd.mpjsvd_svd_noalloc(m, n, Ad.data_ptr(), m, U.data_ptr(), S.data_ptr(),
                                       V.data_ptr(), 0.0, status.data_ptr(), side.cuda_stream)
    assert rc == 0, mpjsvd.mpjsvd_last_error()
    side.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(status.item()) == 0
    # the call on a non-default stream gives the default-stream result bit for bit
    assert np.array_equal(S.cpu().numpy(), S0)
    assert np.array_equal(U.cpu().numpy(), U0)
    assert np.array_equal(V.cpu().numpy(), V0)


def test_noalloc_reports_a_nonfinite_input():
    rng = np.random.default_rng(35)
    A = inputs.known_sigma(rng, 64, 32, np.logspace(0, -2, 32))
    A[5, 7] = np.nan
    U, S, V, status = _noalloc(A)
    assert status & 2  # MPJSVD_STATUS_NONFINITE
    assert np.all(np.isnan(S))
    # the shared scratch is usable again at once
    B = inputs.known_sigma(rng, 64, 32, np.logspace(0, -2, 32))
    U, S, V, status = _noalloc(B)
    assert status == 0
    check_factorization(B, U, S, V)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    from paper_2209_04626_gb300 import mpjsvd
    rc = mpjsvd.mpjsvd_svd_noalloc(1024, 8, 1, 1024, 1, 1, 1, 0.0)
    assert rc == -1 and "512" in mpjsvd.mpjsvd_last_error()
    rc = mpjsvd.mpjsvd_svd_noalloc(512, 300, 1, 512, 1, 1, 1, 0.0)
    assert rc == -2 and "256" in mpjsvd.mpjsvd_last_error()
