"""Helpers for the GPU parity tests: run the library through the binding and compare
with the oracle on the same stored matrix."""
import numpy as np
import torch

U64 = 2.0 ** -53


def gpu_svd(A, mode="auto", precond="rt", qr_first=0, block_w=0, tol=0.0, maxsweep=30, stats=True,
            qrcp="mixed", stop="xgesvj", low_kernel="auto", **params):
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(mode=mode, precond=precond, qr_first=qr_first, block_w=block_w,
                      maxsweep=maxsweep, qrcp=qrcp, stop=stop, low_kernel=low_kernel, **params)
    Ad = mpjsvd.colmajor(torch.from_numpy(np.asarray(A, dtype=np.float64)), torch.device("cuda"))
    U, S, V = h.svd(Ad, tol=tol)
    st = h.stats() if stats else None
    out = (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), st)
    h.close()
    return out


def align_signs(U, V, Uref, Vref):
    """Flip (u_k, v_k) to match the reference's orientation (V decides)."""
    sg = np.sign(np.sum(V * Vref, axis=0))
    sg[sg == 0] = 1.0
    return U * sg, V * sg


def check_factorization(A, U, S, V, n_tol=64):
    m, n = A.shape
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(S)) and np.all(np.isfinite(V))
    assert np.all(np.diff(S) <= 0)
    assert np.abs(U.T @ U - np.eye(n)).max() <= n_tol * n * U64
    assert np.abs(V.T @ V - np.eye(n)).max() <= n_tol * n * U64
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - (U * S) @ V.T) / nA <= 1e-13


def check_sign_rule(V):
    for k in range(V.shape[1]):
        a = np.abs(V[:, k])
        r = int(np.argmax(a))  # first maximum = lowest row on exact ties
        assert V[r, k] >= 0.0


def sigma_gate(A, S_gpu, S_orc):
    """Singular values: GPU error vs the extended-precision oracle must be within
    max(1e-12, 2 x the binary64 oracle's own error). Returns (e_gpu, e_orc)."""
    import oracle
    _, Se, _, _ = oracle.svd(A, mode="plain", ext=True)
    Se = np.asarray(Se, dtype=np.longdouble)
    e_g = float(np.max(np.abs(np.asarray(S_gpu, dtype=np.longdouble) - Se) / Se))
    e_o = float(np.max(np.abs(np.asarray(S_orc, dtype=np.longdouble) - Se) / Se))
    assert e_g <= max(1e-12, 2.0 * e_o), (e_g, e_o)
    return e_g, e_o


def elementwise_vs_oracle(U, S, V, So, Uo, Vo, sig_tol=1e-12, vec_tol=1e-8):
    """Element-wise parity with a binary64 oracle SVD of the same stored A: singular values to
    sig_tol relative, singular vectors (after sign alignment) where the singular values are
    separated by >= 1e-3."""
    assert np.max(np.abs(S - So) / So) <= sig_tol, np.max(np.abs(S - So) / So)
    gaps = np.minimum(np.r_[np.inf, -np.diff(So)], np.r_[-np.diff(So), np.inf]) / So
    sep = gaps >= 1e-3
    assert sep.sum() > len(So) // 2
    Ua, Va = align_signs(U, V, Uo, Vo)
    assert np.abs(Va[:, sep] - Vo[:, sep]).max() <= vec_tol
    assert np.abs(Ua[:, sep] - Uo[:, sep]).max() <= vec_tol
