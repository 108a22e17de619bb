/*
 * mpjsvd_oracle.h -- plain CPU oracle for the mixed-precision one-sided Jacobi SVD
 * (Gao, Ma, Shao, "A mixed precision Jacobi SVD algorithm", arXiv 2209.04626).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers. The GPU library neither links nor calls
 * this code, and this code includes nothing from the GPU library.
 *
 * All matrices are column-major (LAPACK convention): element (i, j) of a matrix
 * with leading dimension ld lives at a[j * ld + i]. Arithmetic is IEEE binary64
 * (orc_real, see below) unless a function name ends in _f32 (binary32 loops, used for
 * the paper's lower-precision stage). Nothing is blocked, fused or reordered beyond what the
 * paper's algorithms state.
 */
#ifndef MPJSVD_ORACLE_H
#define MPJSVD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Working precision. The default build is IEEE binary64, the precision of the method.
 * The same source compiled with -DORC_LONG_DOUBLE uses long double (x86-64: 64-bit
 * significand; aarch64: IEEE binary128) as an extended-precision reference that
 * attributes rounding error; the binary32 stage stays binary32 in both builds. */
#ifdef ORC_LONG_DOUBLE
typedef long double orc_real;
#else
typedef double orc_real;
#endif

/* Tunables of Algorithm 4 (Section 3, values used in Section 7.1). */
typedef struct {
    orc_real tol_alg;        /* Jacobi vs QR-SVD choice threshold (Alg. 4), default 1e-2 */
    orc_real tol_orth;       /* orthogonality skip threshold (Section 3.5), default 1e-5 */
    orc_real tol_cond_coef;  /* tol_cond = coef * n^(1/4) (Section 7.1), default 1.5 */
    orc_real trailing_frac;  /* fraction of trailing columns tested (Section 3.5), default 0.25 */
    orc_real tol;            /* Alg. 1 threshold in working precision; <= 0 -> sqrt(n) * 2^-53 */
    int maxsweep;          /* Alg. 1 maxiter, default 30 */
    int mode;              /* 0 auto (Alg. 4 branch tests), 1 force the low-precision stage,
                              2 never run it (plain FP64 preconditioned Jacobi, Alg. 2) */
    int precond;           /* Jacobi input after the QRCP A1 P = Q1 R: 0 -> X = R^T (lower
                              triangular; SVD of R with the roles of U and V exchanged),
                              1 -> X = R (Alg. 4 with Q2 = I), 2 -> X = L from the LQ
                              factorization R = L Q2 (Alg. 2's else branch), 3 -> Alg. 2's
                              choice: X = R when every column of R is diagonally dominant,
                              else X = L */
    int qrcp;              /* the RRQR of the preconditioning: 0 -> Businger-Golub in working
                              precision (orc_geqp3), 1 -> the mixed-precision RRQR of Alg. 5
                              (orc_geqp3_mixed) */
    int switch_method;     /* precision switch (Section 3.3 and the section on its efficiency):
                              0 -> B = X^T U_low, B = Q1 R1, Y = X Q1 (the paper's choice);
                              1 -> V_low accumulated by the binary32 stage, V_low = Q2 R2,
                              Y = X Q2 (the alternative it compares against) */
    int v_by_qr;           /* right singular vectors (Section 3.4): 0 -> accumulated through the
                              refinement sweeps; 1 -> refinement without V, then V_X from the
                              QR of X^T U_X and one more Alg. 1 with V from that start */
    int stop;              /* when Alg. 1 stops: 0 -> after a sweep without rotations, or after
                              a sweep (not the first) whose rotations were all negligible, as
                              the paper's experiments run it (LAPACK's xGESVJ, Section 7.1);
                              1 -> only after a sweep without rotations (Alg. 1 as printed) */
    orc_real y_tol;          /* > 0: the Y1/Y2 safeguard of Section 3.4 before the refinement:
                              Y2 = the columns from the first one (in the switch's order) whose
                              largest cosine with an earlier column exceeds y_tol; Alg. 1 on Y2,
                              then one sweep of the pairs between Y1 and Y2. 0: off (default) */
} orc_params;

/* What the driver did (per call). */
typedef struct {
    int branch;            /* 0 low-precision stage ran; 1 skipped: cond_R small;
                              2 skipped: trailing columns small; 3 skipped: orth <= tol_orth;
                              4 skipped: mode 2 */
    int sweeps_low;        /* FP32 Alg. 1 sweeps (0 if skipped) */
    int sweeps_work;       /* FP64 Alg. 1 sweeps */
    long long rot_low;     /* rotations applied in FP32 */
    long long rot_work;    /* rotations applied in FP64 */
    orc_real cond_r;         /* |R(0,0)| / |R(n-1,n-1)| */
    orc_real orth;           /* max |Xt^T Xt - I| of the column-scaled low(X), FP32 */
    orc_real switch_off;     /* max_{i!=j} |y_i^T y_j| / (|y_i||y_j|) right after the switch */
    int status;            /* 0 ok, 1 FP64 sweeps hit maxsweep, 2 non-finite input, <0 bad argument */
    int precond;           /* the Jacobi input that ran: 0 R^T, 1 R, 2 L */
    int sweeps_v;          /* v_by_qr = 1: sweeps of the final Alg. 1 with V */
    int y2_cols;           /* columns in the Y2 block of the safeguard (0: not activated) */
} orc_stats;

void orc_default_params(orc_params* p);

/* Householder reflector (Section 3.1): overwrite x[0..len-1] (stride 1) so that
 * x[0] = beta and x[1..] = v[1..] with v[0] = 1 implicit and H = I - tau v v^T,
 * H * x_in = beta * e_1. */
void orc_house(int len, orc_real* x, orc_real* tau);

/* Plain Householder QR, A = Q R (Alg. 4, the m > n preprocessing). In place: R in
 * the upper triangle, reflectors below it, tau[min(m,n)]. */
int orc_geqrf(int m, int n, orc_real* A, int lda, orc_real* tau);

/* Businger-Golub QR with column pivoting, A P = Q R (Section 3.1, Alg. 5 step 2).
 * jpvt[i] = original index of the column in position i (0-based). Column norms are
 * downdated after each step and recomputed when cancellation is severe. */
int orc_geqp3(int m, int n, orc_real* A, int lda, int* jpvt, orc_real* tau);

/* Mixed-precision RRQR (Alg. 5): the column permutation of a Businger-Golub QRCP of lower(A)
 * computed in binary32 (lower(A) = A scaled by the power of two that brings max |a_ij| into
 * [1, 2), so that binary32 neither overflows nor loses the small columns to underflow first),
 * then the Householder QR of A P in working precision. On return A holds that QR of A P
 * (orc_geqrf layout, columns in pivot order), jpvt[j] = the column of A in position j. */
int orc_geqp3_mixed(int m, int n, orc_real* A, int lda, int* jpvt, orc_real* tau);

/* Only the binary32 pivot search of Alg. 5 (step 2): jpvt from the scaled lower(A). A is not
 * modified. */
int orc_qrcp_pivots_f32(int m, int n, const orc_real* A, int lda, int* jpvt);

/* C <- Q C (trans = 0) or Q^T C (trans = 1), Q = H_0 H_1 ... H_{k-1} from orc_geqrf /
 * orc_geqp3 output (V, ldv, tau). C is m x ncols. */
void orc_apply_q(int trans, int m, int ncols, int k, const orc_real* V, int ldv,
                 const orc_real* tau, orc_real* C, int ldc);

/* Alg. 1 in binary64: cyclic one-sided Jacobi on X (m x n). If V != NULL, every rotation
 * is also applied to the columns of V (nv x n). Returns 0 if converged, 1 if maxsweep
 * sweeps ran without converging. */
int orc_jacobi(int m, int n, orc_real* X, int ldx, orc_real* V, int ldv, int nv, orc_real tol,
               int maxsweep, int stop, int* sweeps, long long* rotations);

/* Alg. 1 with de Rijk's pivoting (Section 2.1): subsweep p first moves the column of largest
 * norm among p .. n - 1 to position p (and the same column of V), then rotates the pairs
 * (p, q), q > p. perm (optional): perm[j] = the input column in position j at the end. Same
 * test, rotation, stopping rules and return value as orc_jacobi. */
int orc_jacobi_derijk(int m, int n, orc_real* X, int ldx, orc_real* V, int ldv, int nv, orc_real tol,
                      int maxsweep, int stop, int* perm, int* sweeps, long long* rotations);

/* Alg. 1 in binary32 (Alg. 4: "without generating V explicitly"; V (nv x n, binary32) is
 * accumulated only when not NULL, for the alternative switch). */
int orc_jacobi_f32(int m, int n, float* X, int ldx, float* V, int ldv, int nv, float tol, int maxsweep,
                   int stop, int* sweeps, long long* rotations);

/* Jacobi rotation for one column pair (Section 2.1): given alpha = |x_p|^2,
 * beta = |x_q|^2, gamma = x_p^T x_q (gamma != 0), the tangent t of the rotation closest
 * to the identity that makes [x_p, x_q] J orthogonal, J = [c s; -s c], s = c t. */
orc_real orc_rot_tangent(orc_real alpha, orc_real beta, orc_real gamma);

/* Algorithm 4 (with Algorithm 2 as its mode-2 special case): thin SVD of A (m x n,
 * m >= n). U m x n (ldu = m), S n (descending), V n x n (ldv = n), A = U diag(S) V^T.
 * Sign convention: each (u_i, v_i) is flipped so that the entry of v_i with the largest
 * magnitude (lowest row index on ties) is positive. */
int orc_svd(int m, int n, const orc_real* A, int lda, orc_real* U, orc_real* S, orc_real* V,
            const orc_params* p, orc_stats* st);

/* Adjoint of the thin SVD (not in the paper; published SVD-derivative formula).
 * Given U (m x n), S (n), V (n x n) and the cotangents gU (m x n), gS (n), gV (n x n)
 * (each may be NULL = zero), writes gA (m x n). Pairs with
 * |s_i - s_j| <= gap_tol * max(s_i, s_j) and singular values s_i <= 2^-53 * s_0 are
 * counted in *n_flagged; nothing is clamped. */
int orc_svd_backward(int m, int n, const orc_real* U, const orc_real* S, const orc_real* V,
                     const orc_real* gU, const orc_real* gS, const orc_real* gV, orc_real* gA,
                     orc_real gap_tol, int* n_flagged);

#ifdef __cplusplus
}
#endif
#endif
