"""Pins for the CPU oracle: each test checks the oracle against something other than
itself -- a closed form, an exact special case, a library routine (LAPACK through
numpy/scipy), high-precision arithmetic (mpmath) or finite differences -- so that a
dropped term, a wrong sign or index, or a transposed operand fails at least one test."""
import os

import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs

U64 = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fro(a):
    return float(np.linalg.norm(a))


# ---------------------------------------------------------------- rotation (Section 2.1)

def test_rotation_tangent_matches_angle_closed_form():
    """t = tan(theta) with tan(2 theta) = 2 gamma / (alpha - beta)... in the J convention
    x_p' = c x_p - s x_q; the minimal rotation has |theta| <= pi/4."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        x = rng.standard_normal((7, 2)) * rng.uniform(0.1, 10, 2)
        a, b, g = x[:, 0] @ x[:, 0], x[:, 1] @ x[:, 1], x[:, 0] @ x[:, 1]
        t = oracle.rot_tangent(a, b, g)
        # J = [c s; -s c]: x_p'^T x_q' = 0  <=>  tan(2 theta) = 2 g / (b - a) with t = tan(theta)
        theta = 0.5 * np.arctan2(2 * g, b - a)
        if theta > np.pi / 4:
            theta -= np.pi / 2
        if theta < -np.pi / 4:
            theta += np.pi / 2
        assert abs(t) <= 1.0
        assert t == pytest.approx(np.tan(theta), rel=1e-12, abs=1e-15)
        c = 1 / np.sqrt(1 + t * t)
        s = c * t
        xp = c * x[:, 0] - s * x[:, 1]
        xq = s * x[:, 0] + c * x[:, 1]
        assert abs(xp @ xq) <= 8 * U64 * np.linalg.norm(xp) * np.linalg.norm(xq) * 7
        # alpha' = alpha - t gamma, beta' = beta + t gamma
        assert xp @ xp == pytest.approx(a - t * g, rel=1e-13)
        assert xq @ xq == pytest.approx(b + t * g, rel=1e-13)


def test_golden_2x2():
    """Worked example in tests/golden/svd_2x2.txt (closed form of Section 2.1)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "svd_2x2.txt"))
            if l.strip() and not l.startswith("#")]
    vals = [r for r in rows if all(_isnum(t) for t in r)]
    A = np.array([float(v) for v in vals[0]]).reshape(2, 2)
    s1sq, s2sq = (float(v) for v in vals[1])
    t_expect = float(vals[2][0])
    x1, x2 = A[:, 0], A[:, 1]
    assert oracle.rot_tangent(x1 @ x1, x2 @ x2, x1 @ x2) == t_expect
    U, S, V, st = oracle.svd(A, mode="plain")
    assert S[0] ** 2 == pytest.approx(s1sq, rel=4 * U64)
    assert S[1] ** 2 == pytest.approx(s2sq, rel=8 * U64)
    assert np.allclose(np.abs(V), np.full((2, 2), np.sqrt(0.5)), atol=4 * U64)


def _isnum(t):
    try:
        float(t)
        return True
    except ValueError:
        return False


def test_2x2_closed_form_singular_values():
    rng = np.random.default_rng(5)
    for _ in range(50):
        A = rng.standard_normal((2, 2))
        _, S, _, _ = oracle.svd(A, mode="plain")
        a, b, g = A[:, 0] @ A[:, 0], A[:, 1] @ A[:, 1], A[:, 0] @ A[:, 1]
        r = np.sqrt(((a - b) / 2) ** 2 + g * g)
        s_closed = np.sqrt([(a + b) / 2 + r, (a + b) / 2 - r])
        assert S[0] == pytest.approx(s_closed[0], rel=1e-14)
        assert S[0] * S[1] == pytest.approx(abs(np.linalg.det(A)), rel=1e-13)
        assert S @ S == pytest.approx(_fro(A) ** 2, rel=1e-14)


# ---------------------------------------------------------------- exact special cases

@pytest.mark.parametrize("mode", ["plain", "mixed", "auto"])
def test_diagonal_input_exact(mode):
    rng = np.random.default_rng(2)
    d = rng.permutation(np.logspace(0, -9, 12)) * rng.choice([-1.0, 1.0], 12)
    A = np.diag(d)
    U, S, V, st = oracle.svd(A, mode=mode)
    assert np.array_equal(S, np.sort(np.abs(d))[::-1])
    assert st["rot_work"] == 0
    # U, V are signed permutations with U diag(S) V^T = A exactly
    assert np.array_equal(np.abs(V), np.abs(V).round())
    assert np.array_equal((U * S) @ V.T, A)


def test_permuted_diagonal_rectangular_exact():
    rng = np.random.default_rng(3)
    m, n = 9, 6
    d = rng.uniform(0.5, 3.0, n) * rng.choice([-1.0, 1.0], n)
    D = np.zeros((m, n))
    D[:n, :n] = np.diag(d)
    A = D[rng.permutation(m)][:, rng.permutation(n)]
    U, S, V, st = oracle.svd(A, mode="plain")
    assert np.array_equal(S, np.sort(np.abs(d))[::-1])
    assert np.allclose((U * S) @ V.T, A, atol=0, rtol=0) or np.abs((U * S) @ V.T - A).max() < 4 * U64 * 3


# ---------------------------------------------------------------- known sigma, invariants

@pytest.mark.parametrize("mode", ["plain", "mixed", "auto"])
def test_known_sigma_and_invariants(mode):
    rng = np.random.default_rng(7)
    m, n = 80, 48
    sigma = np.logspace(0, -6, n)
    A = inputs.known_sigma(rng, m, n, sigma)
    U, S, V, st = oracle.svd(A, mode=mode)
    assert st["status"] == 0
    # the stored A is sigma's matrix up to rounding: compare against LAPACK on the same A
    s_lapack = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(S - s_lapack) / s_lapack) < 1e-9  # LAPACK gesdd is not relatively accurate
    assert np.max(np.abs(S - sigma) / sigma) < 1e-8
    assert S @ S == pytest.approx(_fro(A) ** 2, rel=n * U64 * 4)
    assert np.abs(U.T @ U - np.eye(n)).max() <= 64 * n * U64
    assert np.abs(V.T @ V - np.eye(n)).max() <= 64 * n * U64
    assert _fro(A - (U * S) @ V.T) / _fro(A) <= 1e-13
    colerr = np.linalg.norm(A - (U * S) @ V.T, axis=0) / np.linalg.norm(A, axis=0)
    assert colerr.max() <= 1e-13
    assert np.all(np.diff(S) <= 0)


def test_matches_lapack_well_conditioned():
    """Well-conditioned input: every accurate SVD agrees to ~u; LAPACK (numpy) pins sigma
    and the singular subspaces."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((60, 40))
    U, S, V, _ = oracle.svd(A)
    Ul, Sl, Vlt = np.linalg.svd(A, full_matrices=False)
    assert np.max(np.abs(S - Sl) / Sl) < 1e-13
    # singular vectors agree up to sign (simple, well separated singular values)
    sgn = np.sign(np.sum(V * Vlt.T, axis=0))
    assert np.abs(V - Vlt.T * sgn).max() < 1e-11
    assert np.abs(U - Ul * sgn).max() < 1e-11


def test_high_precision_reference_tiny():
    """mpmath at 40 digits as an independent reference on a graded 6 x 4 matrix."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(9)
    A = rng.standard_normal((6, 4)) * np.array([1.0, 1e-3, 1e-6, 1e-9])
    _, S, _, _ = oracle.svd(A, mode="plain")
    M = mpmath.matrix(A.tolist())
    s_hp = mpmath.svd_r(M, compute_uv=False)
    s_hp = sorted([float(x) for x in s_hp], reverse=True)
    assert np.max(np.abs(S - s_hp) / np.array(s_hp)) < 1e-14


def test_scaling_invariance_columns_exact():
    """Scaling a column by a power of two scales nothing but that column's data: the
    oracle's sigma of A D (D = powers of two) equals that of the un-graded matrix only
    through the SVD -- so compare against the permutation-invariance instead: permuting
    the columns of A leaves sigma unchanged (the QRCP pivots see the same norms)."""
    rng = np.random.default_rng(10)
    A = rng.standard_normal((30, 20))
    _, S1, _, _ = oracle.svd(A)
    _, S2, _, _ = oracle.svd(A[:, rng.permutation(20)])
    assert np.max(np.abs(S1 - S2) / S1) < 1e-13


# ---------------------------------------------------------------- QR and QRCP

def test_geqrf_matches_lapack():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((50, 30))
    QR, tau = oracle.geqrf(A)
    R = np.triu(QR[:30])
    R_lapack = np.linalg.qr(A, mode="r")
    assert np.abs(R - R_lapack).max() < 1e-13 * np.abs(R).max()
    Q = oracle.apply_q(QR, tau, np.eye(50)[:, :30])
    assert np.abs(Q.T @ Q - np.eye(30)).max() < 30 * U64 * 8
    assert np.abs(Q @ R - A).max() < 1e-14 * 50
    # Q^T applied after Q gives back the identity columns
    back = oracle.apply_q(QR, tau, Q, trans=True)
    assert np.abs(back - np.eye(50)[:, :30]).max() < 1e-14


def test_geqp3_matches_lapack_pivots():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(13)
    A = rng.standard_normal((40, 25)) * np.logspace(0, -4, 25)[rng.permutation(25)]
    QR, jpvt, tau = oracle.geqp3(A)
    R = np.triu(QR[:25])
    Rl, piv = scipy_linalg.qr(A, mode="r", pivoting=True)
    assert np.array_equal(jpvt, piv)
    assert np.abs(R - Rl[:25]).max() < 1e-12 * np.abs(R).max()
    assert np.all(np.abs(np.diag(R))[:-1] >= np.abs(np.diag(R))[1:])
    Q = oracle.apply_q(QR, tau, np.eye(40)[:, :25])
    err = np.linalg.norm(Q @ R - A[:, jpvt], axis=0) / np.linalg.norm(A[:, jpvt], axis=0)
    assert err.max() < 25 * U64 * 16


# ---------------------------------------------------------------- Alg. 5 (mixed-precision RRQR)

def test_mixed_rrqr_pivots_match_binary64_when_unambiguous():
    # strongly graded columns (ratio 10 between neighbours in norm): the pivot order is decided
    # by margins far above binary32 rounding, so Alg. 5's pivots equal the binary64 QRCP's
    rng = np.random.default_rng(41)
    n = 30
    A = rng.standard_normal((60, n)) * (10.0 ** -np.arange(n))[rng.permutation(n)]
    jp32 = oracle.qrcp_pivots_f32(A)
    _, jp64, _ = oracle.geqp3(A)
    assert np.array_equal(jp32, jp64)
    QRm, jpm, taum = oracle.geqp3_mixed(A)
    QR64, _, tau64 = oracle.geqp3(A)
    assert np.array_equal(jpm, jp64)
    scale = np.abs(np.diag(QR64[:n]))
    assert np.all(np.abs(np.triu(QRm[:n]) - np.triu(QR64[:n])).max(axis=1) <= 1e-13 * np.abs(A).max() * 8)


def test_mixed_rrqr_is_rank_revealing_to_binary32_accuracy():
    # at every step the chosen column had the largest remaining norm, up to the accuracy of
    # the downdated binary32 norms (recomputed once a downdate has lost about sqrt(2^-24)):
    # |R_jj| >= (1 - 2^-11) max_{k >= j} |R(j:, k)| with R the binary64 QR of A P
    rng = np.random.default_rng(42)
    m, n = 120, 70
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -6, n)) * rng.uniform(0.2, 5.0, n)
    QR, jpvt, tau = oracle.geqp3_mixed(A)
    assert sorted(jpvt.tolist()) == list(range(n))
    R = np.triu(QR[:n])
    for j in range(n):
        rem = np.linalg.norm(R[j:, j:], axis=0)
        assert abs(R[j, j]) >= (1 - 2.0 ** -11) * rem.max()
    # the factorization is of A P
    Q = oracle.apply_q(QR, tau, np.eye(m)[:, :n])
    assert np.abs(Q @ R - A[:, jpvt]).max() <= 1e-14 * np.abs(A).max() * 16


def test_mixed_rrqr_ties_keep_the_first_column_and_scaling_is_exact():
    # exactly equal norms at every step (scaled unit columns: each reflector is the identity):
    # the first maximum wins every time
    E = 3.0 * np.eye(40)[:, :12]
    assert np.array_equal(oracle.qrcp_pivots_f32(E), np.arange(12))
    # two identical columns of the largest norm: the lower index goes first
    rng = np.random.default_rng(43)
    B = rng.standard_normal((40, 6)) * np.array([1.0, 0.5, 0.25, 0.1, 0.05, 0.01])
    B = np.column_stack([B[:, 1:4], B[:, 0], B[:, 4:], B[:, 0]])  # copies of column 0 at 3 and 6
    assert oracle.qrcp_pivots_f32(B)[0] == 3
    # the power-of-two scaling of lower(A) keeps binary32 in range: huge and tiny matrices
    # pivot exactly like the unscaled one
    rng = np.random.default_rng(44)
    A = rng.standard_normal((50, 20)) * np.logspace(0, -3, 20)
    jp = oracle.qrcp_pivots_f32(A)
    assert np.array_equal(oracle.qrcp_pivots_f32(A * 2.0 ** 900), jp)
    assert np.array_equal(oracle.qrcp_pivots_f32(A * 2.0 ** -1000), jp)


def test_svd_with_mixed_rrqr_matches_lapack():
    rng = np.random.default_rng(45)
    m, n = 90, 60
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -3, n))
    for mode in ("mixed", "plain"):
        U, S, V, st = oracle.svd(A, mode=mode, qrcp=1)
        assert st["status"] == 0
        s_lapack = np.linalg.svd(A, compute_uv=False)
        assert np.max(np.abs(S - s_lapack) / s_lapack) < 1e-12
        assert np.abs((U * S) @ V.T - A).max() < 1e-13 * np.abs(A).max() * 10


# ---------------------------------------------------------------- Alg. 1 in both precisions

def test_jacobi_f64_and_f32_converge_to_svd():
    rng = np.random.default_rng(14)
    n = 24
    X = inputs.known_sigma(rng, n, n, np.logspace(0, -3, n))
    Xi, V, sw, rot, rc = oracle.jacobi(X, np.eye(n))
    assert rc == 0
    S = np.linalg.norm(Xi, axis=0)
    Sl = np.linalg.svd(X, compute_uv=False)
    assert np.max(np.abs(np.sort(S)[::-1] - Sl) / Sl) < 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() < 64 * n * U64
    assert np.abs(X @ V - Xi).max() < 1e-13  # X V = X_inf: V accumulated every rotation
    Xf, swf, rotf, rcf = oracle.jacobi_f32(X)
    assert rcf == 0
    Sf = np.sort(np.linalg.norm(Xf.astype(np.float64), axis=0))[::-1]
    assert np.max(np.abs(Sf - Sl) / Sl) < 2e-4  # u_low * kappa(B_c) scale
    Xn = Xf.astype(np.float64) / np.linalg.norm(Xf.astype(np.float64), axis=0)
    assert np.abs(Xn.T @ Xn - np.eye(n)).max() < 1e-5


def test_derijk_pivoting_converges_to_the_svd_with_sorted_columns():
    """Alg. 1 with de Rijk's pivoting (Section 2.1): the same singular values as LAPACK, X V = X_inf
    with V orthogonal and V P the accumulated permutation, and (by construction: the last sweep
    rotates nothing and moves the largest remaining column forward in every subsweep) columns
    in descending norm order."""
    rng = np.random.default_rng(15)
    n = 24
    X = inputs.known_sigma(rng, 30, n, np.logspace(0, -3, n))
    Xi, V, perm, sw, rot, rc = oracle.jacobi_derijk(X, np.eye(n))
    assert rc == 0 and sorted(perm.tolist()) == list(range(n))
    S = np.linalg.norm(Xi, axis=0)
    assert np.all(np.diff(S) <= 0.0)
    Sl = np.linalg.svd(X, compute_uv=False)
    assert np.max(np.abs(S - Sl) / Sl) < 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() < 64 * n * U64
    assert np.abs(X @ V - Xi).max() < 1e-13


def test_derijk_pivoting_on_a_permuted_diagonal():
    """Orthogonal columns of distinct norms: no rotation, one sweep, and the columns come out
    in descending norm order (perm = the order of decreasing norms)."""
    d = np.array([0.5, 3.0, 1e-3, 2.0, 7.0])
    X = np.zeros((7, 5))
    X[[4, 0, 6, 2, 1], np.arange(5)] = d
    Xi, V, perm, sw, rot, rc = oracle.jacobi_derijk(X, np.eye(5))
    assert rc == 0 and rot == 0 and sw == 1
    assert perm.tolist() == list(np.argsort(-d))
    assert np.array_equal(np.linalg.norm(Xi, axis=0), np.sort(d)[::-1])


@pytest.mark.parametrize("seed", [16, 17, 18])
def test_derijk_pivoting_accelerates_convergence(seed):
    """The paper's remark that de Rijk's pivoting accelerates Alg. 1, on seeded graded inputs
    (sigma over 6 decades, columns scaled over 4 decades): no more sweeps than the cyclic order,
    the same singular values."""
    rng = np.random.default_rng(seed)
    n = 40
    X = inputs.known_sigma(rng, 50, n, np.logspace(0, -6, n)) * 10.0 ** rng.uniform(-4, 0, n)
    _, _, sw_c, rot_c, rc_c = oracle.jacobi(X)
    Xd, _, _, sw_d, rot_d, rc_d = oracle.jacobi_derijk(X)
    assert rc_c == 0 and rc_d == 0
    assert sw_d <= sw_c, (sw_d, sw_c)
    Xc, _, _, _, _ = oracle.jacobi(X)
    Sc = np.sort(np.linalg.norm(Xc, axis=0))[::-1]
    assert np.max(np.abs(np.linalg.norm(Xd, axis=0) - Sc) / Sc) < 1e-10


def _max_cos(X):
    Xn = X / np.linalg.norm(X, axis=0)
    G = np.abs(Xn.T @ Xn)
    np.fill_diagonal(G, 0.0)
    return G.max()


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_negligible_sweep_stop(seed):
    """The stopping rule of the paper's experiments (stop = 0): it ends no later than Alg. 1 as
    printed (stop = 1), gives the same singular values, and at exit no column pair is more
    than sqrt(n) tol from orthogonal (the rule's premise: the last sweep rotated only pairs
    below sqrt(n) tol, by angles too small to move the others)."""
    rng = np.random.default_rng(seed)
    m, n = 80, 48
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -6, n))
    tol = np.sqrt(m) * U64
    X0, V0, sw0, rot0, rc0 = oracle.jacobi(A, np.eye(n), stop=0)
    X1, V1, sw1, rot1, rc1 = oracle.jacobi(A, np.eye(n), stop=1)
    assert rc0 == 0 and rc1 == 0
    assert sw0 <= sw1 and rot0 <= rot1
    s0 = np.sort(np.linalg.norm(X0, axis=0))[::-1]
    s1 = np.sort(np.linalg.norm(X1, axis=0))[::-1]
    assert np.max(np.abs(s0 - s1) / s1) < 1e-13
    assert _max_cos(X0) <= 2 * np.sqrt(n) * tol
    assert np.abs(V0.T @ V0 - np.eye(n)).max() < 64 * n * U64
    # binary32 stage, same rule
    Xf0, swf0, _, rcf0 = oracle.jacobi_f32(A, stop=0)
    Xf1, swf1, _, rcf1 = oracle.jacobi_f32(A, stop=1)
    assert rcf0 == 0 and rcf1 == 0 and swf0 <= swf1
    assert _max_cos(Xf0.astype(np.float64)) <= 2 * np.sqrt(n) * np.sqrt(m) * 2.0 ** -24


def test_negligible_sweep_needs_two_sweeps():
    """A sweep that rotates nothing ends Alg. 1 under both rules, and the first sweep never
    ends it early: a pair that starts above the threshold takes two sweeps either way."""
    n = 6
    X = np.eye(n)
    X[0, 1] = 1e-10  # columns 0 and 1 at cosine 1e-10, far above tol = sqrt(6) u
    _, _, sw0, rot0, _ = oracle.jacobi(X, stop=0)
    _, _, sw1, rot1, _ = oracle.jacobi(X, stop=1)
    assert (sw0, rot0) == (2, 1) and (sw1, rot1) == (2, 1)
    _, _, sw, rot, _ = oracle.jacobi(np.eye(n), stop=0)
    assert (sw, rot) == (1, 0)


@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_lq_preconditioning(mode):
    """Alg. 2's else branch, X = L from R = L Q2: the same SVD as X = R^T (the singular values
    of R and of L = R Q2^T are the same; V = P Q2^T V_X), orthogonal factors, A = U S V^T."""
    rng = np.random.default_rng(41)
    A = inputs.known_sigma(rng, 70, 48, np.logspace(0, -4, 48))
    Ur, Sr, Vr, str_ = oracle.svd(A, mode=mode, precond="rt")
    Ul, Sl, Vl, stl = oracle.svd(A, mode=mode, precond="l")
    assert str_["precond"] == 0 and stl["precond"] == 2 and stl["status"] == 0
    assert np.max(np.abs(Sl - Sr) / Sr) < 1e-13
    n = A.shape[1]
    assert np.abs(Ul.T @ Ul - np.eye(n)).max() < 64 * n * U64
    assert np.abs(Vl.T @ Vl - np.eye(n)).max() < 64 * n * U64
    assert np.linalg.norm(A - (Ul * Sl) @ Vl.T) / np.linalg.norm(A) < 1e-14
    # well separated singular values: the vectors agree up to sign (sign rule: same choice)
    assert np.abs(Vl - Vr).max() < 1e-10 and np.abs(Ul - Ur).max() < 1e-10


def test_lq_choice_diagonal_dominance():
    """Alg. 2's choice: X = R when every column of R is diagonally dominant, else X = L."""
    rng = np.random.default_rng(42)
    n = 32
    # nearly orthogonal columns of graded norms: R = diag + O(1e-3) per entry, dominant
    A = (np.eye(n) + 1e-3 * rng.standard_normal((n, n))) @ np.diag(np.logspace(0, -3, n))
    _, S1, _, st1 = oracle.svd(A, mode="plain", precond="auto")
    assert st1["precond"] == 1
    # dense with a flat spectrum: the columns of R are not dominant
    B = inputs.known_sigma(rng, n, n, np.linspace(1.0, 0.5, n))
    _, S2, _, st2 = oracle.svd(B, mode="plain", precond="auto")
    assert st2["precond"] == 2
    for M, S in ((A, S1), (B, S2)):
        s_ref = np.linalg.svd(M, compute_uv=False)
        assert np.max(np.abs(S - s_ref) / s_ref) < 1e-13


@pytest.mark.parametrize("seed", [0, 51, 52])
def test_switch_methods(seed):
    """The two ways to switch precisions compared in the paper's section on the switch's
    efficiency: Y1 = X Q1 from the QR of B = X^T U_low (the default) has more orthogonal
    columns than Y2 = X Q2 from the QR of the binary32-accumulated V_low; both refine to
    the same singular values."""
    if seed == 0:
        A, _ = inputs.plain_256x128()
    else:
        rng = np.random.default_rng(seed)
        B = inputs.known_sigma(rng, 120, 80, np.logspace(0, -2, 80))
        A = B * 10.0 ** rng.uniform(-8, 0, 80)
    _, S1, _, st1 = oracle.svd(A, mode="mixed", switch_method=0)
    _, S2, _, st2 = oracle.svd(A, mode="mixed", switch_method=1)
    assert st1["switch_off"] < st2["switch_off"] < 1e-4
    assert np.max(np.abs(S1 - S2) / S2) < 1e-13


@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_v_by_qr(mode):
    """Section 3.4's cheaper V: the refinement without V, then V_X from the QR of X^T U_X as
    the start of one more Alg. 1 with V accumulated, which converges after one sweep of
    rotations (a second confirms); the same SVD as accumulating V throughout."""
    A, _ = inputs.plain_256x128()
    U0, S0, V0, s0 = oracle.svd(A, mode=mode)
    U1, S1, V1, s1 = oracle.svd(A, mode=mode, v_by_qr=1)
    assert s1["status"] == 0 and s1["sweeps_v"] <= 2
    n = A.shape[1]
    assert np.max(np.abs(S1 - S0) / S0) < 1e-13
    assert np.abs(V1.T @ V1 - np.eye(n)).max() < 64 * n * U64
    assert np.abs(U1.T @ U1 - np.eye(n)).max() < 64 * n * U64
    assert np.linalg.norm(A - (U1 * S1) @ V1.T) / np.linalg.norm(A) < 1e-14
    assert np.abs(V1 - V0).max() < 1e-10 and np.abs(U1 - U0).max() < 1e-10


def test_y1_y2_safeguard():
    """Section 3.4's safeguard: at the paper's orthogonality level (1e-5) the switch leaves Y
    orthogonal enough that Y2 is empty (\"rarely activated\"), and the result is the default's
    bit for bit; forced on with a tiny threshold it rotates inside Y2 and between Y1 and Y2
    first, and the refinement reaches the same SVD."""
    A, _ = inputs.plain_256x128()
    U0, S0, V0, s0 = oracle.svd(A, mode="mixed")
    U1, S1, V1, s1 = oracle.svd(A, mode="mixed", y_tol=1e-5)
    assert s1["y2_cols"] == 0 and np.array_equal(S1, S0) and np.array_equal(V1, V0)
    U2, S2, V2, s2 = oracle.svd(A, mode="mixed", y_tol=1e-12)
    assert s2["y2_cols"] > 0 and s2["status"] == 0 and s2["rot_work"] > 0
    n = A.shape[1]
    assert np.max(np.abs(S2 - S0) / S0) < 1e-13
    assert np.abs(V2.T @ V2 - np.eye(n)).max() < 64 * n * U64
    assert np.abs(V2 - V0).max() < 1e-10


def test_mixed_and_plain_agree():
    rng = np.random.default_rng(15)
    A = inputs.known_sigma(rng, 90, 64, np.logspace(0, -5, 64))
    Um, Sm, Vm, stm = oracle.svd(A, mode="mixed")
    Up, Sp, Vp, stp = oracle.svd(A, mode="plain")
    assert stm["branch"] == 0 and stp["branch"] == 4
    assert np.max(np.abs(Sm - Sp) / Sp) < 1e-13
    assert np.abs(Vm - Vp).max() < 1e-9  # gaps >= 17% -> vectors well determined
    assert stm["sweeps_work"] <= 4 < stp["sweeps_work"]  # "typically three sweeps" (Section 3.4)
    assert stm["switch_off"] < 1e-4  # orthogonal to O(u_low) after the switch (Section 4)


# ---------------------------------------------------------------- branch tests (Section 3.5)

def test_branch_cond_small():
    rng = np.random.default_rng(16)
    A = inputs.orthonormal(rng, 40, 32) * 3.0  # kappa(R) = 1
    _, _, _, st = oracle.svd(A)
    assert st["branch_name"] == "skip_cond"


def test_branch_trailing_small():
    rng = np.random.default_rng(17)
    n = 40
    d = np.ones(n)
    d[-n // 3:] = 1e-7
    A = rng.standard_normal((n, n)) * d
    _, _, _, st = oracle.svd(A)
    assert st["branch_name"] == "skip_trailing"


def test_branch_orth():
    rng = np.random.default_rng(18)
    n = 40
    A = inputs.orthonormal(rng, n, n) * np.logspace(0, -3, n)  # orthogonal, graded columns
    _, _, _, st = oracle.svd(A)
    assert st["branch_name"] == "skip_orth"
    assert st["orth"] <= 1e-5


def test_branch_runs_low_precision():
    rng = np.random.default_rng(24)
    A = inputs.known_sigma(rng, 64, 32, np.logspace(0, -2, 32))
    _, _, _, st = oracle.svd(A)
    assert st["branch_name"] == "mixed"


def test_precond_r_and_rt_agree():
    """X = R (Q2 = I) and X = R^T give the same SVD (roles of U and V exchanged)."""
    rng = np.random.default_rng(25)
    A = inputs.known_sigma(rng, 70, 40, np.logspace(0, -4, 40))
    U1, S1, V1, st1 = oracle.svd(A, mode="mixed", precond="rt")
    U2, S2, V2, st2 = oracle.svd(A, mode="mixed", precond="r")
    assert np.max(np.abs(S1 - S2) / S2) < 1e-13
    assert np.abs(U1 - U2).max() < 1e-9 and np.abs(V1 - V2).max() < 1e-9


# ---------------------------------------------------------------- adjoint

def _loss(A, w, GU, GV):
    U, S, V, _ = oracle.svd(A, mode="plain")
    return w @ S + np.sum(GU * U) + np.sum(GV * V)


def test_adjoint_sigma_only_closed_form():
    """d sigma_i / dA = u_i v_i^T, so for L = sum w_i sigma_i, gA = U diag(w) V^T."""
    rng = np.random.default_rng(19)
    A = inputs.known_sigma(rng, 12, 7, np.logspace(0, -1, 7))
    U, S, V, _ = oracle.svd(A)
    w = rng.standard_normal(7)
    gA, nf = oracle.svd_backward(U, S, V, gS=w)
    assert np.abs(gA - (U * w) @ V.T).max() < 1e-14
    assert nf == 0


@pytest.mark.parametrize("shape", [(9, 5), (6, 6)])
def test_adjoint_central_differences(shape):
    rng = np.random.default_rng(20 + shape[0])
    m, n = shape
    A = inputs.known_sigma(rng, m, n, np.logspace(0, -1, n))
    U, S, V, _ = oracle.svd(A, mode="plain")
    w = rng.standard_normal(n)
    GU = rng.standard_normal((m, n))
    GV = rng.standard_normal((n, n))
    gA, nf = oracle.svd_backward(U, S, V, GU, w, GV)
    h = 1e-6
    fd = np.zeros_like(A)
    for i in range(m):
        for j in range(n):
            E = np.zeros_like(A)
            E[i, j] = h
            fd[i, j] = (_loss(A + E, w, GU, GV) - _loss(A - E, w, GU, GV)) / (2 * h)
    assert np.abs(fd - gA).max() < 1e-6 * max(1.0, np.abs(gA).max())
    assert nf == 0


def test_adjoint_flags_near_degenerate():
    rng = np.random.default_rng(23)
    s = np.array([1.0, 0.5, 0.5 * (1 + 1e-9), 0.1])
    A = inputs.known_sigma(rng, 6, 4, s)
    U, S, V, _ = oracle.svd(A)
    _, nf = oracle.svd_backward(U, S, V, gS=np.ones(4), gap_tol=1e-6)
    assert nf == 1


# ---------------------------------------------------------------- extended-precision build

def test_extended_oracle_against_mpmath():
    """The long double build of the same oracle is the extended reference; pin it to
    mpmath at 40 digits (its error must be far below binary64's)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(26)
    A = inputs.known_sigma(rng, 7, 5, np.logspace(0, -6, 5))
    _, Se, _, st = oracle.svd(A, mode="plain", ext=True)
    _, Sd, _, _ = oracle.svd(A, mode="plain")
    s_hp = sorted(mpmath.svd_r(mpmath.matrix(A.tolist()), compute_uv=False), reverse=True)
    rel_e = max(float(abs(mpmath.mpf(str(se)) - sh) / sh) for se, sh in zip(Se, s_hp))
    rel_d = max(float(abs(mpmath.mpf(float(sd)) - sh) / sh) for sd, sh in zip(Sd, s_hp))
    # relative perturbation bound of Jacobi: O(u kappa(B_c)), B_c = A with unit columns
    kappa_bc = np.linalg.cond(A / np.linalg.norm(A, axis=0))
    assert rel_e <= 64 * oracle.unit_roundoff(ext=True) * kappa_bc
    assert rel_d <= 64 * 2.0 ** -53 * kappa_bc
    assert rel_e * 100 < rel_d  # the extended build really is the more accurate reference


def test_binary64_oracle_error_is_attributed_to_precision():
    """On a column-scaled condition ~1e6 input, the binary64 oracle differs from the
    extended build by more than binary64 rounding of sigma but far below u * kappa."""
    A, _ = inputs.plain_256x128(m=64, n=32)
    _, S, _, _ = oracle.svd(A, mode="plain")
    _, Se, _, _ = oracle.svd(A, mode="plain", ext=True)
    e = float(np.max(np.abs(np.asarray(S, dtype=np.longdouble) - Se) / Se))
    Bc = A / np.linalg.norm(A, axis=0)
    assert e < 2.0 ** -53 * np.linalg.cond(Bc) * 64
