"""The accuracy experiment of Section 7 on the GPU: the sixteen (MODE of D, MODE of Sigma) types
of Table 1 (matrices A = B D from the modes of Table 2), in the paper's two square settings
(kappa(D), kappa(B)) = (1e2, 1e12) and (1e20, 1e2), through Algorithm 4 (automatic branch
choice) and the plain binary64 algorithm, each against the extended-precision oracle on the
same stored A. The relative accuracy of one-sided Jacobi follows kappa(B), the condition of
the column-scaled matrix, so the bar is the binary64 oracle's own error (within 2x) or 1e-12,
whichever is larger; the factorization bars hold for every type."""
import numpy as np
import pytest

import oracle
from paper_2209_04626_gb300 import inputs
from tests.gpu_util import check_factorization, gpu_svd, sigma_gate

pytestmark = pytest.mark.gpu

N = 128
SETTINGS = [(1e2, 1e12), (1e20, 1e2)]


@pytest.mark.parametrize("setting", SETTINGS)
def test_table1_types(setting):
    kd, kb = setting
    worst = {}
    for t, (md, ms) in enumerate(inputs.TABLE1):
        rng = np.random.default_rng(100 + t)
        A = inputs.table1_pair(rng, N, md, ms, kd, kb)
        for mode in ("auto", "plain"):
            U, S, V, st = gpu_svd(A, mode=mode)
            assert st["status"] in (0, 8), (md, ms, mode, st)  # 8: an exactly zero sigma
            if st["status"] == 0:
                check_factorization(A, U, S, V)
            _, So, _, sto = oracle.svd(A, mode=mode)
            if mode == "auto":
                assert st["branch"] == sto["branch"], (md, ms, st["branch_name"], sto["branch_name"])
            keep = So > 0
            if kb <= 1e2:
                e_g, e_o = sigma_gate(A, S[keep], So[keep])
            else:
                # kappa(B) = 1e12: every binary64 algorithm's error is set by the perturbation
                # bound of one-sided Jacobi, about sqrt(n) u kappa(B_c) (here ~1e-3), not by the
                # algorithm; the GPU must stay within that bound (the oracle does too)
                _, Se, _, _ = oracle.svd(A, mode="plain", ext=True)
                Se = np.asarray(Se, dtype=np.longdouble)[keep]
                e_g = float(np.max(np.abs(np.asarray(S[keep], dtype=np.longdouble) - Se) / Se))
                e_o = float(np.max(np.abs(np.asarray(So[keep], dtype=np.longdouble) - Se) / Se))
                bound = np.sqrt(N) * 2.0 ** -53 * kb
                assert e_g <= bound and e_o <= bound, (md, ms, mode, e_g, e_o, bound)
            worst[(md, ms, mode)] = e_g
    # the error follows kappa(B): far below 1e-12 at kappa(B) = 1e2 for every type
    if kb <= 1e2:
        assert max(worst.values()) <= 1e-12, max(worst.values())
