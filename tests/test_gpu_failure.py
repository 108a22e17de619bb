"""Failure detection on the GPU without a fault: a bounded device wait is made to run out on
purpose (a counter that nothing releases, a grid barrier one CTA never reaches) with a short
limit; the call must report MPJSVD_STATUS_TIMEOUT in a bounded time, and the same handle must
then run a normal SVD correctly (the context stays usable)."""
import time

import numpy as np
import pytest

from paper_2209_04626_gb300 import inputs
from tests.gpu_util import check_factorization

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_handle_survives():
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(wait_limit_ms=20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = mpjsvd.mpjsvd_selftest_timeout(h.h)
    assert rc == 0, mpjsvd.mpjsvd_last_error()
    st = h.stats()  # synchronizes the stream
    dt = time.perf_counter() - t0
    assert st["status"] & mpjsvd.STATUS_TIMEOUT
    assert dt < 5.0, dt
    # the next call on the same handle resets the status and computes normally
    h.set(wait_limit_ms=4000, mode="mixed")
    rng = np.random.default_rng(70)
    A = inputs.known_sigma(rng, 300, 200, np.logspace(0, -4, 200))
    U, S, V = [t.cpu().numpy() for t in h.svd(mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")))]
    st = h.stats()
    assert st["status"] == 0, st
    check_factorization(A, U, S, V)
    h.close()


def test_wait_limit_parameter_is_validated():
    from paper_2209_04626_gb300 import mpjsvd
    with pytest.raises(RuntimeError):
        mpjsvd.Handle(wait_limit_ms=0)
