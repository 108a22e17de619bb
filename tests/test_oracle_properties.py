"""Property tests of the oracle's options on random small matrices (host only): every
combination of mode, Jacobi input, switch, V construction, safeguard and stopping rule returns
an SVD that meets the factorization bars and the LAPACK singular values to u sigma_max."""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

U64 = 2.0 ** -53


@hyp.settings(max_examples=60, deadline=None)
@hyp.given(seed=st.integers(0, 2 ** 31 - 1), n=st.integers(1, 10), extra=st.integers(0, 6),
           mode=st.sampled_from(["auto", "mixed", "plain"]), precond=st.sampled_from(["rt", "r", "l", "auto"]),
           switch_method=st.sampled_from([0, 1]), v_by_qr=st.sampled_from([0, 1]),
           y_tol=st.sampled_from([0.0, 1e-12]), stop=st.sampled_from([0, 1]),
           decades=st.integers(0, 10))
def test_oracle_options_give_the_svd(seed, n, extra, mode, precond, switch_method, v_by_qr, y_tol, stop,
                                     decades):
    rng = np.random.default_rng(seed)
    m = n + extra
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-decades, 0, n)[None, :]
    U, S, V, stt = oracle.svd(A, mode=mode, precond=precond, switch_method=switch_method,
                              v_by_qr=v_by_qr, y_tol=y_tol, stop=stop)
    assert stt["status"] == 0
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(S)) and np.all(np.isfinite(V))
    assert np.all(np.diff(S) <= 0)
    assert np.abs(U.T @ U - np.eye(n)).max() <= 64 * max(n, 4) * U64
    assert np.abs(V.T @ V - np.eye(n)).max() <= 64 * max(n, 4) * U64
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - (U * S) @ V.T) <= 1e-13 * nA
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.abs(S - s_ref) <= 64 * n * U64 * s_ref[0])
    for k in range(n):  # sign rule: the largest-magnitude entry of v_k is positive
        r = int(np.argmax(np.abs(V[:, k])))
        assert V[r, k] >= 0.0
