"""GPU parity of the batched path (one persistent launch, one CTA per matrix) against the
CPU oracle and against the single-matrix GPU path, on seeded uneven batches."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import (U64, align_signs, check_factorization, check_sign_rule, gpu_svd,
                            sigma_gate)

pytestmark = pytest.mark.gpu


def _run_batched(mats, mode, **params):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    h = mpjsvd.Handle(mode=mode, **params)
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


@pytest.mark.parametrize("qrcp", ["mixed", "f64"])
@pytest.mark.parametrize("mode", ["mixed", "plain", "auto"])
def test_batched_against_oracle(mode, qrcp):
    """Both RRQRs of the batched path (Alg. 5 by default, binary64 Businger-Golub) against the
    oracle run with the same one."""
    mats = _small_batch(40, 24, 48)
    Us, Ss, Vs, info = _run_batched(mats, mode, qrcp=qrcp)
    assert np.all(info == 0), info
    for A, U, S, V in zip(mats, Us, Ss, Vs):
        check_factorization(A, U, S, V)
        check_sign_rule(V)
        Uo, So, Vo, _ = oracle.svd(A, mode=mode, qrcp=1 if qrcp == "mixed" else 0)
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
    Us, Ss, Vs, info = _run_batched(mats, "mixed", qrcp="f64")
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


def _device_batch(mats):
    """Device copies of the matrices, their pointer arrays and device size arrays."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    dev = torch.device("cuda")
    A = [mpjsvd.colmajor(torch.from_numpy(X), dev) for X in mats]
    U = [mpjsvd.empty_colmajor(X.shape[0], X.shape[1], dev) for X in mats]
    S = [torch.empty(X.shape[1], dtype=torch.float64, device=dev) for X in mats]
    V = [mpjsvd.empty_colmajor(X.shape[1], X.shape[1], dev) for X in mats]
    ptr = lambda ts: torch.tensor([t.data_ptr() for t in ts], dtype=torch.int64, device=dev)
    m = torch.tensor([X.shape[0] for X in mats], dtype=torch.int32, device=dev)
    n = torch.tensor([X.shape[1] for X in mats], dtype=torch.int32, device=dev)
    info = torch.full((len(mats),), 99, dtype=torch.int32, device=dev)
    return dict(A=A, U=U, S=S, V=V, pA=ptr(A), pU=ptr(U), pS=ptr(S), pV=ptr(V), m=m, n=n, lda=m.clone(),
                info=info)


def test_batched_device_sizes_in_a_cuda_graph():
    """The device-array call captured in a CUDA graph: two replays give bit-identical outputs,
    equal to an uncaptured call's, every matrix meets the bars and a sample matches the oracle;
    a matrix whose sizes exceed the stated bounds is reported with info = -1."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    mats = _small_batch(50, 40, 96)
    big = inputs.known_sigma(np.random.default_rng(51), 200, 150, np.logspace(0, -3, 150))
    mats.append(big)  # exceeds max_n = 128 below
    maxm = max(X.shape[0] for X in mats[:-1])
    d = _device_batch(mats)
    h = mpjsvd.Handle(mode="mixed")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    mpjsvd.mpjsvd_set_stream(h.h, side.cuda_stream)

    def call():
        return mpjsvd.mpjsvd_svd_batched_dev(h.h, len(mats), maxm, 128, d["m"].data_ptr(), d["n"].data_ptr(),
                                             d["lda"].data_ptr(), d["pA"].data_ptr(), d["pU"].data_ptr(),
                                             d["pS"].data_ptr(), d["pV"].data_ptr(), 0.0, d["info"].data_ptr())
    with torch.cuda.stream(side):
        assert call() == 0, mpjsvd.mpjsvd_last_error()  # the workspace is allocated here
    torch.cuda.synchronize()
    ref = [s.cpu().numpy().copy() for s in d["S"]], [v.cpu().numpy().copy() for v in d["V"]]
    info0 = d["info"].cpu().numpy().copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        assert call() == 0, mpjsvd.mpjsvd_last_error()
    outs = []
    for _ in range(2):
        for t in d["S"]:
            t.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        outs.append(([s.cpu().numpy().copy() for s in d["S"]], [v.cpu().numpy().copy() for v in d["V"]],
                     d["info"].cpu().numpy().copy()))
    h.close()
    assert info0[-1] == -1 and np.all(info0[:-1] == 0), info0
    for (S1, V1, i1) in outs:
        assert np.array_equal(i1, info0)
        for k in range(len(mats) - 1):
            assert np.array_equal(S1[k], ref[0][k]) and np.array_equal(V1[k], ref[1][k]), k
    for k in range(0, len(mats) - 1, 7):
        A = mats[k]
        U = d["U"][k].cpu().numpy()
        S, V = ref[0][k], ref[1][k]
        check_factorization(A, U, S, V)
        _, So, _, _ = oracle.svd(A, mode="mixed", qrcp=1)
        sigma_gate(A, S, So)


def test_batched_autotuner_picks_per_size_class():
    """The first batched call of a handle tunes every size class present (each kernel variant
    timed on a sample); the picks are valid block widths, and the tuned call meets the bars."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    rng = np.random.default_rng(52)
    mats = []
    for n in [20] * 30 + [60] * 30 + [120] * 20 + [200] * 10:
        mats.append(inputs.known_sigma(rng, n + 8, n, np.logspace(0, -3, n)))
    h = mpjsvd.Handle(mode="mixed")
    assert all(t == (0, 0, 0.0) for t in mpjsvd.mpjsvd_get_batched_tuning(h.h))
    dmats = [mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")) for A in mats]
    Us, Ss, Vs, info = h.svd_batched(dmats)
    torch.cuda.synchronize()
    tun = mpjsvd.mpjsvd_get_batched_tuning(h.h)
    for c, (wl, ww, ms) in enumerate(tun):
        if c <= 3:
            assert wl in (8, 16) and ww in (4, 8) and ms > 0.0, (c, tun)
        else:
            assert (wl, ww) == (0, 0)
    assert np.all(info.cpu().numpy() == 0)
    for i in range(0, len(mats), 9):
        check_factorization(mats[i], Us[i].cpu().numpy(), Ss[i].cpu().numpy(), Vs[i].cpu().numpy())
    h.close()
