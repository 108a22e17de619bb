"""The tensor-core (tcgen05, TF32 with a 3-term split) form of the binary32 stage: its two
GEMM steps against binary64 products of the same binary32 data, and the whole SVD with the
stage forced onto the tensor cores against the oracle, across sizes that span several
64-column blocks, a ragged last block and a phantom block, up to the 2048 x 1024 workload."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import (align_signs, check_factorization, check_sign_rule, gpu_svd,
                            sigma_gate)

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _block(Z, W=None, gram=True):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    dev = torch.device("cuda")
    m = Z.shape[0]
    Zd = torch.from_numpy(np.asfortranarray(Z, dtype=np.float32).T.copy()).to(dev).t()  # column-major
    G = torch.zeros((128, 128), dtype=torch.float32, device=dev) if gram else None
    # W column-major: the row-major buffer of W^T
    Wd = torch.from_numpy(np.ascontiguousarray(np.asarray(W, dtype=np.float32).T)).to(dev) \
        if W is not None else None
    h = mpjsvd.Handle()
    rc = mpjsvd.mpjsvd_tc_block_f32(h.h, m, Zd.data_ptr(), m, G.data_ptr() if gram else None,
                                    Wd.data_ptr() if W is not None else None)
    assert rc == 0, mpjsvd.mpjsvd_last_error()
    st = h.stats()
    assert st["status"] == 0, st
    Gh = G.cpu().numpy().T if gram else None  # written column-major
    out = Zd.cpu().numpy()
    h.close()
    return Gh, out


@pytest.mark.parametrize("m", [1, 31, 128, 300, 1024, 4099, 4100, 8202])
def test_tc_gram_tf32x3(m):
    """G = Z^T Z: within the binary32 error bound of a dot product, 2 m u_32 |z_i| |z_j| (the
    3-term split drops only lo lo', about 2^-22 of each product), against the binary64
    product of the same binary32 data; graded columns (norms over 8 decades) included."""
    rng = np.random.default_rng(80 + m)
    Z = (rng.standard_normal((m, 128)) * 10.0 ** rng.uniform(-8, 0, 128)).astype(np.float32)
    G, _ = _block(Z)
    Zd = Z.astype(np.float64)
    Gr = Zd.T @ Zd
    nrm = np.sqrt(np.diag(Gr))
    bound = (2 * m + 8) * U32 * np.outer(nrm, nrm)
    assert np.all(np.abs(G - Gr) <= bound), np.max(np.abs(G - Gr) / np.outer(nrm, nrm))
    assert np.allclose(G, G.T, rtol=0, atol=0) or np.max(np.abs(G - G.T) / np.outer(nrm, nrm)) < 1e-6


@pytest.mark.parametrize("m", [5, 128, 257, 2048])
def test_tc_apply_tf32x3(m):
    """Z <- Z W for an orthogonal W (a rotation accumulation of the stage): each entry within
    (128 + 8) u_32 sum_k |z_ik| |w_kj| of the binary64 product of the same data."""
    rng = np.random.default_rng(90 + m)
    Z = (rng.standard_normal((m, 128)) * 10.0 ** rng.uniform(-6, 0, 128)).astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((128, 128)))
    W = Q.astype(np.float32)
    _, out = _block(Z, W, gram=False)
    ref = Z.astype(np.float64) @ W.astype(np.float64)
    bound = (128 + 8) * U32 * (np.abs(Z.astype(np.float64)) @ np.abs(W.astype(np.float64)))
    assert np.all(np.abs(out - ref) <= bound + 1e-30), np.max(np.abs(out - ref) / (bound + 1e-30))


def _compare_tc(A, mode="mixed", vec_tol=1e-8):
    U, S, V, st = gpu_svd(A, mode=mode, low_kernel="tc")
    Uo, So, Vo, sto = oracle.svd(A, mode=mode)
    assert st["status"] == 0, st
    if mode == "mixed":
        assert st["branch"] == 0 and st["block_w_low"] == 64 and st["sweeps_low"] > 0, st
    check_factorization(A, U, S, V)
    check_sign_rule(V)
    sigma_gate(A, S, So)
    gaps = np.minimum(np.r_[np.inf, -np.diff(So)], np.r_[-np.diff(So), np.inf]) / So
    sep = gaps >= 1e-3
    Ua, Va = align_signs(U, V, Uo, Vo)
    assert np.abs(Va[:, sep] - Vo[:, sep]).max(initial=0) <= vec_tol
    assert np.abs(Ua[:, sep] - Uo[:, sep]).max(initial=0) <= vec_tol
    return st, sto


@pytest.mark.parametrize("n", [64, 130, 200, 320])
def test_tc_stage_small_sizes(n):
    """One block, a ragged block and phantom blocks (k padded to even)."""
    rng = np.random.default_rng(110 + n)
    A = inputs.known_sigma(rng, n + 17, n, np.logspace(0, -4, n))
    _compare_tc(A)


def test_tc_stage_graded():
    rng = np.random.default_rng(120)
    A = inputs.graded(rng, 300, 256, np.logspace(0, -3, 256), 10.0 ** rng.uniform(-8, 0, 256))
    st, sto = _compare_tc(A, vec_tol=1e-7)
    # the refinement after the tensor-core stage needs no more sweeps than after the oracle's
    # binary32 stage, plus one
    assert st["sweeps_work"] <= sto["sweeps_work"] + 1, (st["sweeps_work"], sto["sweeps_work"])


def test_tc_stage_precision_2048x1024():
    """The 2048 x 1024 workload with the tensor-core binary32 stage, against the oracle."""
    A = inputs.precision_2048x1024()
    Uo, So, Vo, sto = oracle.svd(A, mode="mixed")
    U, S, V, st = gpu_svd(A, mode="mixed", low_kernel="tc")
    assert st["status"] == 0 and st["branch"] == 0, st
    check_factorization(A, U, S, V)
    assert np.max(np.abs(S - So) / So) <= 1e-12
    assert st["sweeps_work"] <= sto["sweeps_work"] + 1, (st["sweeps_work"], sto["sweeps_work"])
