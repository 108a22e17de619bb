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


def test_block_reflector_ut_form_matches_the_product_of_householder_reflectors():
    """The compact form the two-level QR applies (Joffrain, Low, Quintana-Orti, van de Geijn):
    for reflectors H_j = I - tau_j v_j v_j^T (the oracle's Householder QR, geqrf layout, one
    zero reflector included), Q = H_1 ... H_k = I - V T V^T with T^{-1} = S = striu(V^T V) +
    diag(1 / tau). Checked against the oracle's own application of the reflectors: Q^T C =
    C - V X with S^T X = V^T C by forward substitution, Q C = C - V X with S X = V^T C by back
    substitution, each x_i multiplied by tau_i (so tau = 0 contributes nothing)."""
    rng = np.random.default_rng(71)
    m, k = 40, 12
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-6, 0, k)
    A[:, 5] = 0.0  # stays zero under the earlier reflectors: its own reflector has tau = 0
    QR, tau = oracle.geqrf(A)
    assert tau[5] == 0.0 and np.all(tau[np.arange(k) != 5] != 0.0)
    V = np.tril(QR[:, :k], -1) + np.eye(m, k)
    G = V.T @ V
    C = rng.standard_normal((m, 7))

    def subst(W, upper):
        X = W.copy()
        order = range(k - 1, -1, -1) if upper else range(k)
        for i in order:
            if upper:
                acc = X[i] - G[i, i + 1:] @ X[i + 1:]
            else:
                acc = X[i] - G[:i, i] @ X[:i]
            X[i] = acc * tau[i]
        return X

    QtC = C - V @ subst(V.T @ C, upper=False)
    QC = C - V @ subst(V.T @ C, upper=True)
    assert np.abs(QtC - oracle.apply_q(QR, tau, C, trans=True)).max() < 1e-13
    assert np.abs(QC - oracle.apply_q(QR, tau, C, trans=False)).max() < 1e-13
