"""GPU parity of the SVD adjoint: against the oracle's adjoint on the same (U, S, V,
cotangents), against central finite differences of the GPU forward (h = 1e-6), and the
near-degenerate flag count."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu_backward(U, S, V, gU, gS, gV, gap_tol=1e-3):
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    dev = torch.device("cuda")
    h = mpjsvd.Handle()
    t = lambda x: mpjsvd.colmajor(torch.from_numpy(np.ascontiguousarray(x)), dev)
    gA, nf = h.backward(t(U), torch.from_numpy(np.ascontiguousarray(S)).to(dev), t(V),
                        t(gU) if gU is not None else None,
                        torch.from_numpy(gS).to(dev) if gS is not None else None,
                        t(gV) if gV is not None else None, gap_tol=gap_tol)
    out = gA.cpu().numpy()
    h.close()
    return out, nf


@pytest.mark.parametrize("shape", [(64, 32), (33, 33), (200, 120)])
def test_adjoint_matches_oracle(shape):
    rng = np.random.default_rng(50 + shape[0])
    m, n = shape
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -2, n))
    U, S, V, _ = oracle.svd(A)
    w = rng.standard_normal(n)
    GU = rng.standard_normal((m, n))
    GV = rng.standard_normal((n, n))
    gA_o, nf_o = oracle.svd_backward(U, S, V, GU, w, GV)
    gA, nf = _gpu_backward(U, S, V, GU, w, GV)
    assert nf == nf_o
    assert np.abs(gA - gA_o).max() <= 1e-11 * np.abs(gA_o).max()
    # partial cotangents (None = zero)
    gA_o2, _ = oracle.svd_backward(U, S, V, None, w, None)
    gA2, _ = _gpu_backward(U, S, V, None, w, None)
    assert np.abs(gA2 - gA_o2).max() <= 1e-12 * np.abs(gA_o2).max()


def test_autograd_against_central_differences():
    """loss = sum w_i s_i + <G_U, U> + <G_V, V> through SVDFunction; central FD of the GPU
    forward along random directions (h = 1e-6)."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    rng = np.random.default_rng(60)
    m, n = 64, 32
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -2, n))
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    GU = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    GV = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    Ad = mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")).requires_grad_(True)

    def loss(X):
        U, S, V = mpjsvd.SVDFunction.apply(X, "mixed")
        return (w * S).sum() + (GU * U).sum() + (GV * V).sum()

    L = loss(Ad)
    L.backward()
    g = Ad.grad.detach().cpu().numpy()
    h = 1e-6
    L0 = abs(L.item())
    for k in range(6):
        E = rng.standard_normal((m, n))
        Et = mpjsvd.colmajor(torch.from_numpy(E), torch.device("cuda"))
        with torch.no_grad():
            fd = [(loss(Ad.detach() + s * Et).item() - loss(Ad.detach() - s * Et).item()) / (2 * s)
                  for s in (h, 2 * h)]
        an = float(np.sum(g * E))
        # central differences err by c h^2: estimate it from the 2h value (Richardson), plus
        # the rounding of the loss divided by h
        trunc = abs(fd[1] - fd[0]) / 3.0
        rounding = 1e3 * 2.0 ** -53 * max(1.0, L0) / h
        assert abs(fd[0] - an) <= 3.0 * trunc + rounding + 1e-9 * abs(an), (k, fd, an)
        richardson = (4.0 * fd[0] - fd[1]) / 3.0
        assert abs(richardson - an) <= abs(fd[0] - an) + rounding, (k, richardson, an)


def test_differentiation_workload_large_member():
    """The 1024 x 512 member of the differentiation workload: GPU adjoint vs oracle adjoint
    on the same factors."""
    items = inputs.differentiation(batch=1, large=(1024, 512))
    A, s, w, GU, GV = items[-1]
    U, S, V, _ = oracle.svd(A)
    gA_o, nf_o = oracle.svd_backward(U, S, V, GU, w, GV)
    gA, nf = _gpu_backward(U, S, V, GU, w, GV)
    assert nf == nf_o == 0
    assert np.abs(gA - gA_o).max() <= 1e-10 * np.abs(gA_o).max()


def test_near_degenerate_pairs_flagged_not_clamped():
    rng = np.random.default_rng(61)
    s = np.array([1.0, 0.5, 0.5 * (1 + 1e-9), 0.1])
    A = inputs.known_sigma(rng, 6, 4, s)
    U, S, V, _ = oracle.svd(A)
    gA, nf = _gpu_backward(U, S, V, None, np.ones(4), None, gap_tol=1e-6)
    assert nf == 1
    assert np.all(np.isfinite(gA))


def test_batched_adjoint_differentiation_workload():
    """The differentiation workload's 512 matrices of 64 x 32 in one batched SVD and one batched
    adjoint launch: every member's gA against the oracle's adjoint on the GPU's own factors,
    one member with a zero cotangent entry, and central differences of the batched forward
    along a random direction for a few members."""
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    items = inputs.differentiation(batch=512)[:512]
    dev = torch.device("cuda")
    mats = [mpjsvd.colmajor(torch.from_numpy(A), dev) for A, *_ in items]
    h = mpjsvd.Handle(mode="mixed")
    Us, Ss, Vs, info = h.svd_batched(mats)
    assert int((info != 0).sum()) == 0
    gUs = [mpjsvd.colmajor(torch.from_numpy(GU), dev) for _, _, _, GU, _ in items]
    gSs = [torch.from_numpy(w).to(dev) for _, _, w, _, _ in items]
    gVs = [mpjsvd.colmajor(torch.from_numpy(GV), dev) for *_, GV in items]
    gVs[7] = None  # a zero cotangent for one member
    gAs, flags = h.backward_batched(Us, Ss, Vs, gUs, gSs, gVs)
    torch.cuda.synchronize()
    assert int(flags.sum()) == 0
    for b in range(512):
        U, S, V = Us[b].cpu().numpy(), Ss[b].cpu().numpy(), Vs[b].cpu().numpy()
        _, _, w, GU, GV = items[b]
        gA_o, nf_o = oracle.svd_backward(U, S, V, GU, w, None if b == 7 else GV)
        assert nf_o == 0
        gA = gAs[b].cpu().numpy()
        assert np.abs(gA - gA_o).max() <= 1e-11 * np.abs(gA_o).max(), b
    # central differences of the loss of member b through the batched forward
    rng = np.random.default_rng(62)
    hstep = 1e-6
    for b in (0, 255, 511):
        A, _, w, GU, GV = items[b]
        E = rng.standard_normal(A.shape)

        Vref = Vs[b]

        def loss(X):
            # the sign rule (largest |v_ik| positive) is discontinuous where two entries tie in
            # magnitude; the derivative is that of the branch through A, so the perturbed
            # factors are oriented like A's before the loss is taken
            U, S, V, _ = h.svd_batched([mpjsvd.colmajor(torch.from_numpy(X), dev)])
            sg = torch.sign((V[0] * Vref).sum(0))
            return float((torch.from_numpy(w).to(dev) * S[0]).sum() +
                         (torch.from_numpy(GU).to(dev) * (U[0] * sg)).sum() +
                         (torch.from_numpy(GV).to(dev) * (V[0] * sg)).sum())
        fd = [(loss(A + s * E) - loss(A - s * E)) / (2 * s) for s in (hstep, 2 * hstep)]
        an = float(np.sum(gAs[b].cpu().numpy() * E))
        trunc = abs(fd[1] - fd[0]) / 3.0
        rounding = 1e3 * 2.0 ** -53 * max(1.0, abs(loss(A))) / hstep
        assert abs(fd[0] - an) <= 3.0 * trunc + rounding + 1e-9 * abs(an), (b, fd, an)
    h.close()


def test_autograd_reports_near_degenerate_flags():
    """Through torch.autograd: the adjoint of a matrix with a near-degenerate pair warns with
    the count, which stays readable after .backward() (last_backward_flags, handle stats)."""
    import warnings
    import torch
    from paper_2209_04626_gb300 import mpjsvd
    rng = np.random.default_rng(63)
    s = np.array([1.0, 0.5, 0.5 * (1 + 1e-6), 0.1, 0.05])
    A = inputs.known_sigma(rng, 8, 5, s)
    Ad = mpjsvd.colmajor(torch.from_numpy(A), torch.device("cuda")).requires_grad_(True)
    with warnings.catch_warnings(record=True) as rec:
        warnings.simplefilter("always")
        U, S, V = mpjsvd.svd(Ad, mode="plain")  # requires grad: goes through SVDFunction
        S.sum().backward()
    assert any("near-degenerate" in str(r.message) for r in rec)
    assert mpjsvd.last_backward_flags() == 1
    assert mpjsvd.default_handle().stats()["n_flagged"] == 1
    # d(sum s)/dA = sum_i u_i v_i^T = U V^T, finite for a near-degenerate pair
    g = Ad.grad.detach().cpu().numpy()
    Un, Vn = U.detach().cpu().numpy(), V.detach().cpu().numpy()
    assert np.abs(g - Un @ Vn.T).max() <= 1e-12
