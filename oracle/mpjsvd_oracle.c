/*
 * mpjsvd_oracle.c -- plain CPU oracle for the mixed-precision one-sided Jacobi SVD
 * (Gao, Ma, Shao, arXiv 2209.04626).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
 * leg are its only callers; the GPU library never links or calls it, and it shares no
 * code, header or table with the GPU library.
 *
 * Every routine is the textbook loop nest of the algorithm it cites, in the working
 * precision orc_real (binary64 by default; binary32 for the *_f32 routine and the
 * orthogonality test), column-major, unblocked, single-threaded.
 */
#include "mpjsvd_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(a, i, j, ld) ((a)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

#ifdef ORC_LONG_DOUBLE
#define RSQRT sqrtl
#define RFABS fabsl
static const orc_real U_WORK = LDBL_EPSILON / 2;      /* unit round-off of long double */
#else
#define RSQRT sqrt
#define RFABS fabs
static const orc_real U_WORK = 1.1102230246251565e-16; /* 2^-53, unit round-off of binary64 */
#endif
static const orc_real U_LOW = 5.9604644775390625e-08;  /* 2^-24, unit round-off of binary32 */

void orc_default_params(orc_params* p)
{
    p->tol_alg = 1e-2;        /* Section 7.1 */
    p->tol_orth = 1e-5;       /* Section 7.1 and the footnote of Section 3.5 */
    p->tol_cond_coef = 1.5;   /* Section 7.1: tol_cond = 1.5 n^(1/4) */
    p->trailing_frac = 0.25;  /* Section 3.5 footnote: check 1/4 to 1/3 of the columns */
    p->tol = 0.0;             /* -> RSQRT(n) * 2^-53 */
    p->maxsweep = 30;
    p->mode = 0;
    p->precond = 0;
    p->qrcp = 0;
    p->switch_method = 0;
    p->v_by_qr = 0;
    p->stop = 0;
    p->y_tol = 0.0;
}

static orc_real nrm2(int len, const orc_real* x)
{
    orc_real s = 0.0;
    for (int i = 0; i < len; ++i) s += x[i] * x[i];
    return RSQRT(s);
}

/* ---------------------------------------------------------------------------------
 * Householder reflector (used by the QR preconditioning of Section 3.1 and the QR of
 * the switch, Section 3.3). H = I - tau v v^T, v[0] = 1, H x = beta e_1 with
 * beta = -sign(x_0) |x|, the choice that avoids cancellation in x_0 - beta.
 * ------------------------------------------------------------------------------- */
void orc_house(int len, orc_real* x, orc_real* tau)
{
    if (len <= 1) { *tau = 0.0; return; }
    orc_real alpha = x[0];
    orc_real s = 0.0;
    for (int i = 1; i < len; ++i) s += x[i] * x[i];
    if (s == 0.0) { *tau = 0.0; return; } /* already a multiple of e_1: H = I */
    orc_real norm = RSQRT(alpha * alpha + s);
    orc_real beta = (alpha >= 0.0) ? -norm : norm;
    *tau = (beta - alpha) / beta;
    orc_real den = alpha - beta;
    for (int i = 1; i < len; ++i) x[i] /= den; /* divide: a lone nonzero maps to +-1 exactly */
    x[0] = beta;
}

/* Apply H = I - tau v v^T (v[0] = 1 implicit, v[1..len-1] = vtail) to column c (len). */
static void house_apply(int len, const orc_real* vtail, orc_real tau, orc_real* c)
{
    if (tau == 0.0) return;
    orc_real w = c[0];
    for (int i = 1; i < len; ++i) w += vtail[i] * c[i];
    w *= tau;
    c[0] -= w;
    for (int i = 1; i < len; ++i) c[i] -= w * vtail[i];
}

/* Plain QR, A = Q0 R1 (Alg. 4 preprocessing for m > n; Section 3.1). */
int orc_geqrf(int m, int n, orc_real* A, int lda, orc_real* tau)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    int k = m < n ? m : n;
    for (int j = 0; j < k; ++j) {
        orc_real* colj = &AT(A, j, j, lda);
        orc_house(m - j, colj, &tau[j]);
        for (int c = j + 1; c < n; ++c) house_apply(m - j, colj, tau[j], &AT(A, j, c, lda));
    }
    return 0;
}

/* Businger-Golub QR with column pivoting (the RRQR of Section 3.1 / Alg. 5, step 2):
 * at step j the remaining column of largest norm is swapped into position j, then
 * eliminated by a Householder reflector. Column norms are downdated by the new row-j
 * entry and recomputed from scratch when the downdate has lost more than half the
 * digits (ratio test against the norm recorded at the last recomputation). */
int orc_geqp3(int m, int n, orc_real* A, int lda, int* jpvt, orc_real* tau)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    const orc_real tol3z = RSQRT(U_WORK);
    orc_real* vn1 = (orc_real*)malloc(sizeof(orc_real) * (size_t)(n > 0 ? n : 1));
    orc_real* vn2 = (orc_real*)malloc(sizeof(orc_real) * (size_t)(n > 0 ? n : 1));
    if (!vn1 || !vn2) { free(vn1); free(vn2); return -9; }
    for (int c = 0; c < n; ++c) {
        jpvt[c] = c;
        vn1[c] = nrm2(m, &AT(A, 0, c, lda));
        vn2[c] = vn1[c];
    }
    int k = m < n ? m : n;
    for (int j = 0; j < k; ++j) {
        int p = j;
        for (int c = j + 1; c < n; ++c)
            if (vn1[c] > vn1[p]) p = c; /* first maximum wins ties */
        if (p != j) {
            for (int i = 0; i < m; ++i) {
                orc_real t = AT(A, i, j, lda);
                AT(A, i, j, lda) = AT(A, i, p, lda);
                AT(A, i, p, lda) = t;
            }
            int ti = jpvt[j]; jpvt[j] = jpvt[p]; jpvt[p] = ti;
            vn1[p] = vn1[j];
            vn2[p] = vn2[j];
        }
        orc_real* colj = &AT(A, j, j, lda);
        orc_house(m - j, colj, &tau[j]);
        for (int c = j + 1; c < n; ++c) {
            house_apply(m - j, colj, tau[j], &AT(A, j, c, lda));
            if (vn1[c] != 0.0) {
                orc_real r = RFABS(AT(A, j, c, lda)) / vn1[c];
                orc_real t = 1.0 - r * r;
                if (t < 0.0) t = 0.0;
                orc_real q = vn1[c] / vn2[c];
                if (t * q * q <= tol3z) {
                    vn1[c] = (j + 1 < m) ? nrm2(m - j - 1, &AT(A, j + 1, c, lda)) : 0.0;
                    vn2[c] = vn1[c];
                } else {
                    vn1[c] *= RSQRT(t);
                }
            }
        }
    }
    free(vn1);
    free(vn2);
    return 0;
}

/* |x| in binary32 without underflow or overflow of the squares: the entries are first scaled
 * by the power of two that brings max |x_i| into [1, 2) (exact), as single-precision LAPACK
 * norms avoid underflow. */
static float nrm2_f32(int len, const float* x)
{
    float amax = 0.0f;
    for (int i = 0; i < len; ++i) {
        float a = fabsf(x[i]);
        if (a > amax) amax = a;
    }
    if (amax == 0.0f) return 0.0f;
    int e;
    frexpf(amax, &e);
    const float sc = ldexpf(1.0f, 1 - e);
    float s = 0.0f;
    for (int i = 0; i < len; ++i) {
        float y = x[i] * sc;
        s += y * y;
    }
    return sqrtf(s) / sc;
}

/* Alg. 5, step 2 in binary32: the same Businger-Golub steps as orc_geqp3 (first maximum on
 * ties, norm downdating with recomputation when the downdate keeps less than half of the
 * binary32 digits), on lower(A); only the permutation is kept. Norms use nrm2_f32. */
int orc_qrcp_pivots_f32(int m, int n, const orc_real* A, int lda, int* jpvt)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    /* lower(A): scale by 2^-e, e the binary exponent of max |a_ij| (exact in binary64) */
    orc_real amax = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) {
            orc_real a = RFABS(AT(A, i, j, lda));
            if (a > amax) amax = a;
        }
    int e = 0;
    if (amax > 0.0) frexp((double)amax, &e); /* amax = f 2^e, f in [0.5, 1) */
    const double scale = ldexp(1.0, 1 - e);   /* amax * scale in [1, 2) */
    float* L = (float*)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
    float* vn1 = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* vn2 = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* v = (float*)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
    if (!L || !vn1 || !vn2 || !v) { free(L); free(vn1); free(vn2); free(v); return -9; }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) L[(size_t)j * m + i] = (float)((double)AT(A, i, j, lda) * scale);
    const float tol3z = sqrtf(5.9604644775390625e-08f); /* sqrt(2^-24) */
    for (int c = 0; c < n; ++c) {
        jpvt[c] = c;
        vn1[c] = nrm2_f32(m, &L[(size_t)c * m]);
        vn2[c] = vn1[c];
    }
    int k = m < n ? m : n;
    for (int j = 0; j < k; ++j) {
        int p = j;
        for (int c = j + 1; c < n; ++c)
            if (vn1[c] > vn1[p]) p = c;
        if (p != j) {
            for (int i = 0; i < m; ++i) {
                float t = L[(size_t)j * m + i];
                L[(size_t)j * m + i] = L[(size_t)p * m + i];
                L[(size_t)p * m + i] = t;
            }
            int ti = jpvt[j]; jpvt[j] = jpvt[p]; jpvt[p] = ti;
            vn1[p] = vn1[j];
            vn2[p] = vn2[j];
        }
        /* Householder reflector of L(j:m, j), the same convention as orc_house */
        float* colj = &L[(size_t)j * m];
        float alpha = colj[j], tj = 0.0f;
        const float tailn = (j + 1 < m) ? nrm2_f32(m - j - 1, &colj[j + 1]) : 0.0f;
        if (tailn != 0.0f) {
            float nrm = nrm2_f32(m - j, &colj[j]);
            float beta = (alpha >= 0.0f) ? -nrm : nrm;
            tj = (beta - alpha) / beta;
            float den = alpha - beta;
            v[j] = 1.0f;
            for (int i = j + 1; i < m; ++i) v[i] = colj[i] / den;
            colj[j] = beta;
            for (int i = j + 1; i < m; ++i) colj[i] = v[i];
        }
        for (int c = j + 1; c < n; ++c) {
            float* col = &L[(size_t)c * m];
            if (tj != 0.0f) {
                float w = col[j];
                for (int i = j + 1; i < m; ++i) w += v[i] * col[i];
                w *= tj;
                col[j] -= w;
                for (int i = j + 1; i < m; ++i) col[i] -= w * v[i];
            }
            if (vn1[c] != 0.0f) {
                float r = fabsf(col[j]) / vn1[c];
                float t = 1.0f - r * r;
                if (t < 0.0f) t = 0.0f;
                float q = vn1[c] / vn2[c];
                if (t * q * q <= tol3z) {
                    vn1[c] = (j + 1 < m) ? nrm2_f32(m - j - 1, &col[j + 1]) : 0.0f;
                    vn2[c] = vn1[c];
                } else {
                    vn1[c] *= sqrtf(t);
                }
            }
        }
    }
    free(L); free(vn1); free(vn2); free(v);
    return 0;
}

/* Alg. 5: pivots from binary32, then the QR of A P in working precision. */
int orc_geqp3_mixed(int m, int n, orc_real* A, int lda, int* jpvt, orc_real* tau)
{
    int rc = orc_qrcp_pivots_f32(m, n, A, lda, jpvt);
    if (rc) return rc;
    orc_real* T = (orc_real*)malloc(sizeof(orc_real) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
    if (!T) return -9;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) T[(size_t)j * m + i] = AT(A, i, jpvt[j], lda);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) AT(A, i, j, lda) = T[(size_t)j * m + i];
    free(T);
    return orc_geqrf(m, n, A, lda, tau);
}

void orc_apply_q(int trans, int m, int ncols, int k, const orc_real* V, int ldv,
                 const orc_real* tau, orc_real* C, int ldc)
{
    /* Q = H_0 H_1 ... H_{k-1}: Q C applies H_{k-1} first, Q^T C applies H_0 first. */
    for (int s = 0; s < k; ++s) {
        int j = trans ? s : (k - 1 - s);
        const orc_real* v = &AT(V, j, j, ldv);
        for (int c = 0; c < ncols; ++c) house_apply(m - j, v, tau[j], &AT(C, j, c, ldc));
    }
}

/* ---------------------------------------------------------------------------------
 * Jacobi rotation (Section 2.1). [x_p, x_q] J with J = [c s; -s c] gives
 *   x_p' = c x_p - s x_q,  x_q' = s x_p + c x_q,
 * and x_p'^T x_q' = c^2 (gamma (1 - t^2) - t (beta - alpha)) with t = s / c. Setting it
 * to zero gives t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 gamma). Of its two
 * roots the one of modulus <= 1 gives the J closest to the identity (the footnote of
 * Section 2.1): t = sign(zeta) / (|zeta| + RSQRT(1 + zeta^2)).
 * ------------------------------------------------------------------------------- */
orc_real orc_rot_tangent(orc_real alpha, orc_real beta, orc_real gamma)
{
    orc_real zeta = (beta - alpha) / (2.0 * gamma);
    orc_real az = RFABS(zeta);
    orc_real t;
    if (az > 1e150) t = 1.0 / (2.0 * az); /* zeta^2 would overflow; t -> 1/(2|zeta|) */
    else t = 1.0 / (az + RSQRT(1.0 + az * az));
    return (zeta >= 0.0) ? t : -t;
}

/* Stopping rule of the paper's experiments (Section 7.1 runs Alg. 1 as LAPACK's xGESVJ):
 * besides a sweep without rotations, a sweep other than the first ends the iteration when
 * every rotation in it was negligible: the largest cosine |x_p^T x_q| / (|x_p| |x_q|) among
 * the rotated pairs is below sqrt(n) tol, and n times it times the largest |tan| of those
 * rotations is below tol. */
static int negligible_sweep(int n, double tol, double cos_max, double tan_max)
{
    return cos_max < sqrt((double)n) * tol && (double)n * cos_max * tan_max < tol;
}

/* One pair step of Alg. 1: (p, q) is rotated when |x_q^T x_p| > tol |x_p| |x_q|, with alpha,
 * beta, gamma recomputed from the columns; the rotation is applied to x_p, x_q and (if vp)
 * to v_p, v_q (nv rows). Returns 1 if it rotated; tracks the largest cosine and |tan|. */
static int jacobi_pair(int m, orc_real* xp, orc_real* xq, orc_real* vp, orc_real* vq, int nv, orc_real tol,
                       double* cos_max, double* tan_max)
{
    orc_real alpha = 0.0, beta = 0.0, gamma = 0.0;
    for (int i = 0; i < m; ++i) {
        alpha += xp[i] * xp[i];
        beta += xq[i] * xq[i];
        gamma += xp[i] * xq[i];
    }
    if (!(RFABS(gamma) > tol * RSQRT(alpha) * RSQRT(beta))) return 0;
    orc_real t = orc_rot_tangent(alpha, beta, gamma);
    const double cs = (double)(RFABS(gamma) / (RSQRT(alpha) * RSQRT(beta)));
    if (cs > *cos_max) *cos_max = cs;
    if (fabs((double)t) > *tan_max) *tan_max = fabs((double)t);
    orc_real c = 1.0 / RSQRT(1.0 + t * t);
    orc_real s = c * t;
    for (int i = 0; i < m; ++i) {
        orc_real a = xp[i], b = xq[i];
        xp[i] = c * a - s * b;
        xq[i] = s * a + c * b;
    }
    if (vp) {
        for (int i = 0; i < nv; ++i) {
            orc_real a = vp[i], b = vq[i];
            vp[i] = c * a - s * b;
            vq[i] = s * a + c * b;
        }
    }
    return 1;
}

/* Alg. 1 in binary64. Cyclic order (1,2),(1,3),...,(n-1,n) of eq. (cyclic). The pair
 * (p, q) is rotated when |x_q^T x_p| > tol |x_p| |x_q|; a sweep without rotations
 * means convergence (stop = 1), or also a negligible sweep (stop = 0, negligible_sweep).
 * alpha, beta, gamma are recomputed from the columns for each pair. */
int orc_jacobi(int m, int n, orc_real* X, int ldx, orc_real* V, int ldv, int nv, orc_real tol,
               int maxsweep, int stop, int* sweeps, long long* rotations)
{
    long long rot = 0;
    int sweep = 0, converged = 0;
    while (sweep < maxsweep && !converged) {
        converged = 1;
        double cos_max = 0.0, tan_max = 0.0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                if (jacobi_pair(m, &AT(X, 0, p, ldx), &AT(X, 0, q, ldx), V ? &AT(V, 0, p, ldv) : NULL,
                                V ? &AT(V, 0, q, ldv) : NULL, nv, tol, &cos_max, &tan_max)) {
                    ++rot;
                    converged = 0;
                }
            }
        }
        if (!converged && stop == 0 && sweep > 0 && negligible_sweep(n, (double)tol, cos_max, tan_max))
            converged = 1;
        ++sweep;
    }
    if (sweeps) *sweeps = sweep;
    if (rotations) *rotations = rot;
    return converged ? 0 : 1;
}

/* Alg. 1 in binary64 with de Rijk's pivoting (Section 2.1): a sweep is n - 1 subsweeps; subsweep
 * p first moves the column of largest Euclidean norm among columns p .. n - 1 to position p
 * (interchanging it with column p, and the same columns of V; the first such column on ties),
 * then orthogonalizes the pairs (p, q), q = p + 1 .. n - 1, with the same test, rotation and
 * stopping rules as orc_jacobi. The column order of the result is therefore the one the last
 * sweep left: descending norms. perm (optional, n entries): perm[j] = the input column now in
 * position j. */
int orc_jacobi_derijk(int m, int n, orc_real* X, int ldx, orc_real* V, int ldv, int nv, orc_real tol,
                      int maxsweep, int stop, int* perm, int* sweeps, long long* rotations)
{
    long long rot = 0;
    int sweep = 0, converged = 0;
    if (perm)
        for (int j = 0; j < n; ++j) perm[j] = j;
    while (sweep < maxsweep && !converged) {
        converged = 1;
        double cos_max = 0.0, tan_max = 0.0;
        for (int p = 0; p < n - 1; ++p) {
            /* the dominant column of X(:, p:n) */
            int jmax = p;
            orc_real nmax = -1.0;
            for (int j = p; j < n; ++j) {
                orc_real s2 = 0.0;
                for (int i = 0; i < m; ++i) s2 += AT(X, i, j, ldx) * AT(X, i, j, ldx);
                if (s2 > nmax) {
                    nmax = s2;
                    jmax = j;
                }
            }
            if (jmax != p) {
                for (int i = 0; i < m; ++i) {
                    orc_real t = AT(X, i, p, ldx);
                    AT(X, i, p, ldx) = AT(X, i, jmax, ldx);
                    AT(X, i, jmax, ldx) = t;
                }
                if (V)
                    for (int i = 0; i < nv; ++i) {
                        orc_real t = AT(V, i, p, ldv);
                        AT(V, i, p, ldv) = AT(V, i, jmax, ldv);
                        AT(V, i, jmax, ldv) = t;
                    }
                if (perm) {
                    int t = perm[p];
                    perm[p] = perm[jmax];
                    perm[jmax] = t;
                }
            }
            for (int q = p + 1; q < n; ++q) {
                if (jacobi_pair(m, &AT(X, 0, p, ldx), &AT(X, 0, q, ldx), V ? &AT(V, 0, p, ldv) : NULL,
                                V ? &AT(V, 0, q, ldv) : NULL, nv, tol, &cos_max, &tan_max)) {
                    ++rot;
                    converged = 0;
                }
            }
        }
        if (!converged && stop == 0 && sweep > 0 && negligible_sweep(n, (double)tol, cos_max, tan_max))
            converged = 1;
        ++sweep;
    }
    if (sweeps) *sweeps = sweep;
    if (rotations) *rotations = rot;
    return converged ? 0 : 1;
}

/* Alg. 1 in binary32 without V (the lower-precision stage of Alg. 4). Same steps and
 * stopping rules as orc_jacobi; every operation rounds to binary32. */
int orc_jacobi_f32(int m, int n, float* X, int ldx, float* V, int ldv, int nv, float tol, int maxsweep,
                   int stop, int* sweeps, long long* rotations)
{
    long long rot = 0;
    int sweep = 0, converged = 0;
    while (sweep < maxsweep && !converged) {
        converged = 1;
        double cos_max = 0.0, tan_max = 0.0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                float* xp = &AT(X, 0, p, ldx);
                float* xq = &AT(X, 0, q, ldx);
                float alpha = 0.0f, beta = 0.0f, gamma = 0.0f;
                for (int i = 0; i < m; ++i) {
                    alpha += xp[i] * xp[i];
                    beta += xq[i] * xq[i];
                    gamma += xp[i] * xq[i];
                }
                if (!(fabsf(gamma) > tol * sqrtf(alpha) * sqrtf(beta))) continue;
                float zeta = (beta - alpha) / (2.0f * gamma);
                float az = fabsf(zeta);
                float t = (az > 1e18f) ? 1.0f / (2.0f * az) : 1.0f / (az + sqrtf(1.0f + az * az));
                if (zeta < 0.0f) t = -t;
                const double cs = (double)(fabsf(gamma) / (sqrtf(alpha) * sqrtf(beta)));
                if (cs > cos_max) cos_max = cs;
                if (fabsf(t) > tan_max) tan_max = fabsf(t);
                float c = 1.0f / sqrtf(1.0f + t * t);
                float s = c * t;
                for (int i = 0; i < m; ++i) {
                    float a = xp[i], b = xq[i];
                    xp[i] = c * a - s * b;
                    xq[i] = s * a + c * b;
                }
                if (V) {
                    float* vp = &AT(V, 0, p, ldv);
                    float* vq = &AT(V, 0, q, ldv);
                    for (int i = 0; i < nv; ++i) {
                        float a = vp[i], b = vq[i];
                        vp[i] = c * a - s * b;
                        vq[i] = s * a + c * b;
                    }
                }
                ++rot;
                converged = 0;
            }
        }
        if (!converged && stop == 0 && sweep > 0 && negligible_sweep(n, (double)tol, cos_max, tan_max))
            converged = 1;
        ++sweep;
    }
    if (sweeps) *sweeps = sweep;
    if (rotations) *rotations = rot;
    return converged ? 0 : 1;
}

/* ---------------------------------------------------------------------------------
 * Algorithm 4.
 * ------------------------------------------------------------------------------- */
static int all_finite(int m, int n, const orc_real* A, int lda)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i)
            if (!isfinite(AT(A, i, j, lda))) return 0;
    return 1;
}

/* max_{i != j} |y_i^T y_j| / (|y_i| |y_j|): orthogonality of Y after the switch. */
static orc_real scaled_offdiag(int m, int n, const orc_real* Y)
{
    orc_real worst = 0.0;
    for (int p = 0; p < n; ++p) {
        orc_real np = nrm2(m, &AT(Y, 0, p, m));
        for (int q = p + 1; q < n; ++q) {
            orc_real nq = nrm2(m, &AT(Y, 0, q, m));
            orc_real g = 0.0;
            for (int i = 0; i < m; ++i) g += AT(Y, i, p, m) * AT(Y, i, q, m);
            orc_real r = (np > 0.0 && nq > 0.0) ? RFABS(g) / (np * nq) : 0.0;
            if (r > worst) worst = r;
        }
    }
    return worst;
}

int orc_svd(int m, int n, const orc_real* A, int lda, orc_real* U, orc_real* S, orc_real* V,
            const orc_params* pin, orc_stats* st)
{
    orc_params p;
    if (pin) p = *pin; else orc_default_params(&p);
    orc_stats s;
    memset(&s, 0, sizeof(s));
    if (n < 1) { s.status = -3; if (st) *st = s; return -3; }
    if (m < n) { s.status = -2; if (st) *st = s; return -2; }
    if (lda < m) { s.status = -5; if (st) *st = s; return -5; }
    if (!all_finite(m, n, A, lda)) { s.status = 2; if (st) *st = s; return 2; }

    const size_t nn = (size_t)n * (size_t)n;
    orc_real* W0 = (orc_real*)malloc(sizeof(orc_real) * (size_t)m * (size_t)n); /* A, then Q0 \ R1 */
    orc_real* tau0 = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
    orc_real* R = (orc_real*)calloc(nn, sizeof(orc_real));                      /* R1, then Q1 \ R */
    orc_real* tau1 = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
    int* jpvt = (int*)malloc(sizeof(int) * (size_t)n);
    orc_real* X = (orc_real*)calloc(nn, sizeof(orc_real));
    orc_real* Y = (orc_real*)malloc(sizeof(orc_real) * nn);
    orc_real* Vacc = (orc_real*)calloc(nn, sizeof(orc_real));
    orc_real* Ux = (orc_real*)calloc((size_t)m * (size_t)n, sizeof(orc_real));
    int* order = (int*)malloc(sizeof(int) * (size_t)n);
    orc_real* sig = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
    orc_real* Lq = NULL;   /* R^T = Q' R' (geqrf layout) when X = L: L = R'^T, Q2 = Q'^T */
    orc_real* tauq = NULL;
    if (!W0 || !tau0 || !R || !tau1 || !jpvt || !X || !Y || !Vacc || !Ux || !order || !sig) {
        s.status = -9;
        goto done;
    }

    /* Alg. 4 preprocessing: A = Q0 R1 when m > n, else A1 = A (Q0 = I). */
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) AT(W0, i, j, m) = AT(A, i, j, lda);
    if (m > n) {
        orc_geqrf(m, n, W0, m, tau0);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i <= j; ++i) AT(R, i, j, n) = AT(W0, i, j, m);
    } else {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) AT(R, i, j, n) = AT(W0, i, j, m);
    }
    /* QR preconditioning: A1 P = Q1 R; X = R^T (default), X = R (Q2 = I), or X = L from
     * R = L Q2 (Alg. 2). */
    if (p.qrcp == 1) orc_geqp3_mixed(n, n, R, n, jpvt, tau1);
    else orc_geqp3(n, n, R, n, jpvt, tau1);
    int pc = p.precond;
    if (pc == 3) {
        /* Alg. 2's test "R is almost diagonal", read as: every column of R is diagonally
         * dominant, |r_jj| >= sum_{i<j} |r_ij| (the paper's "close to diagonally dominant") */
        int dominant = 1;
        for (int j = 0; j < n && dominant; ++j) {
            orc_real off = 0.0;
            for (int i = 0; i < j; ++i) off += RFABS(AT(R, i, j, n));
            if (off > RFABS(AT(R, j, j, n))) dominant = 0;
        }
        pc = dominant ? 1 : 2;
    }
    s.precond = (pc == 1) ? 1 : (pc == 2 ? 2 : 0);
    if (pc == 2) {
        /* LQ of R as the QR of R^T: R^T = Q' R', so R = R'^T Q'^T, L = R'^T, Q2 = Q'^T */
        Lq = (orc_real*)calloc(nn, sizeof(orc_real));
        tauq = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
        if (!Lq || !tauq) { s.status = -9; goto done; }
        for (int j = 0; j < n; ++j)
            for (int i = 0; i <= j; ++i) AT(Lq, j, i, n) = AT(R, i, j, n);
        orc_geqrf(n, n, Lq, n, tauq);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i <= j; ++i) AT(X, j, i, n) = AT(Lq, i, j, n);
    } else {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i <= j; ++i) {
                if (pc == 1) AT(X, i, j, n) = AT(R, i, j, n);
                else AT(X, j, i, n) = AT(R, i, j, n);
            }
    }

    /* Special cases of Section 3.5. */
    {
        orc_real rnn = RFABS(AT(X, n - 1, n - 1, n));
        s.cond_r = (rnn > 0.0) ? RFABS(AT(X, 0, 0, n)) / rnn : INFINITY;
        orc_real tol_cond = p.tol_cond_coef * pow((orc_real)n, 0.25);
        orc_real maxnorm = 0.0;
        for (int j = 0; j < n; ++j) {
            orc_real c = nrm2(n, &AT(X, 0, j, n));
            if (c > maxnorm) maxnorm = c;
        }
        int ntrail = (int)ceil(p.trailing_frac * (orc_real)n);
        int trailing_small = ntrail > 0;
        for (int j = n - ntrail; j < n; ++j)
            if (nrm2(n, &AT(X, 0, j, n)) > RSQRT(U_LOW) * maxnorm) trailing_small = 0;
        /* orth = |Xt^T Xt - I|_max, Xt = low(X) D^-1, in binary32. */
        float* Xt = (float*)malloc(sizeof(float) * nn);
        if (!Xt) { s.status = -9; goto done; }
        for (size_t i = 0; i < nn; ++i) Xt[i] = (float)X[i];
        for (int j = 0; j < n; ++j) {
            float d = 0.0f;
            for (int i = 0; i < n; ++i) d += AT(Xt, i, j, n) * AT(Xt, i, j, n);
            d = sqrtf(d);
            if (d > 0.0f)
                for (int i = 0; i < n; ++i) AT(Xt, i, j, n) /= d;
        }
        float orth = 0.0f;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                float g = 0.0f;
                for (int i = 0; i < n; ++i) g += AT(Xt, i, a, n) * AT(Xt, i, b, n);
                float e = fabsf(g - (a == b ? 1.0f : 0.0f));
                if (e > orth) orth = e;
            }
        free(Xt);
        s.orth = orth;
        if (p.mode == 2) s.branch = 4;
        else if (p.mode == 1) s.branch = 0;
        else if (s.cond_r <= tol_cond) s.branch = 1;
        else if (trailing_small) s.branch = 2;
        else if (s.orth <= p.tol_orth) s.branch = 3;
        else s.branch = 0;
    }

    if (s.branch == 0) {
        /* Lower-precision SVD of low(X), U only (Section 3.2). The paper would use QR-SVD
         * when orth > tol_alg; this oracle always uses Alg. 1 (Jacobi). */
        float* Xl = (float*)malloc(sizeof(float) * nn);
        orc_real* B = (orc_real*)malloc(sizeof(orc_real) * nn);
        orc_real* tau2 = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
        if (!Xl || !B || !tau2) { free(Xl); free(B); free(tau2); s.status = -9; goto done; }
        for (size_t i = 0; i < nn; ++i) Xl[i] = (float)X[i];
        float* Vl = NULL;  /* binary32 V of the low stage, only for the alternative switch */
        if (p.switch_method == 1) {
            Vl = (float*)calloc(nn, sizeof(float));
            if (!Vl) { free(Xl); free(B); free(tau2); s.status = -9; goto done; }
            for (int j = 0; j < n; ++j) AT(Vl, j, j, n) = 1.0f;
        }
        orc_jacobi_f32(n, n, Xl, n, Vl, n, Vl ? n : 0, (float)(RSQRT((orc_real)n) * U_LOW), p.maxsweep,
                       p.stop, &s.sweeps_low, &s.rot_low);
        if (Vl) {
            /* Alternative switch: V_low = Q2 R2 in binary64, Y = X Q2, V_acc = Q2. */
            for (size_t i = 0; i < nn; ++i) B[i] = (orc_real)Vl[i];
            free(Vl);
            orc_geqrf(n, n, B, n, tau2);
            for (int j = 0; j < n; ++j) AT(Vacc, j, j, n) = 1.0;
            orc_apply_q(0, n, n, n, B, n, tau2, Vacc, n);
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    orc_real acc = 0.0;
                    for (int i = 0; i < n; ++i) acc += AT(X, a, i, n) * AT(Vacc, i, b, n);
                    AT(Y, a, b, n) = acc;
                }
            s.switch_off = scaled_offdiag(n, n, Y);
            free(Xl);
            free(B);
            free(tau2);
            goto refine;
        }
        /* U_low = normalized columns sorted by descending norm (Alg. 1 final loop and
         * sort), promoted to binary64. The sort matters for the switch: the QR of
         * B = X^T U_low removes from each column its error along the directions of the
         * columns before it, which must be those of larger singular values. */
        float* sl = (float*)malloc(sizeof(float) * (size_t)n);
        int* ord = (int*)malloc(sizeof(int) * (size_t)n);
        if (!sl || !ord) { free(sl); free(ord); free(Xl); free(B); free(tau2); s.status = -9; goto done; }
        for (int j = 0; j < n; ++j) {
            float d = 0.0f;
            for (int i = 0; i < n; ++i) d += AT(Xl, i, j, n) * AT(Xl, i, j, n);
            sl[j] = sqrtf(d);
            for (int i = 0; i < n; ++i) AT(Xl, i, j, n) = (sl[j] > 0.0f) ? AT(Xl, i, j, n) / sl[j] : 0.0f;
            ord[j] = j;
        }
        for (int a = 1; a < n; ++a) { /* stable insertion sort, descending */
            int oj = ord[a];
            int b = a - 1;
            while (b >= 0 && sl[ord[b]] < sl[oj]) { ord[b + 1] = ord[b]; --b; }
            ord[b + 1] = oj;
        }
        /* Switch (Section 3.3, method preferred there): B = X^T orc_real(U_low),
         * B = Q R2, Y = X Q; the refinement's V accumulator starts at Q. */
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                orc_real acc = 0.0;
                for (int i = 0; i < n; ++i) acc += AT(X, i, a, n) * (orc_real)AT(Xl, i, ord[b], n);
                AT(B, a, b, n) = acc;
            }
        free(sl);
        free(ord);
        orc_geqrf(n, n, B, n, tau2);
        for (int j = 0; j < n; ++j) AT(Vacc, j, j, n) = 1.0;
        orc_apply_q(0, n, n, n, B, n, tau2, Vacc, n); /* Vacc = Q */
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                orc_real acc = 0.0;
                for (int i = 0; i < n; ++i) acc += AT(X, a, i, n) * AT(Vacc, i, b, n);
                AT(Y, a, b, n) = acc;
            }
        s.switch_off = scaled_offdiag(n, n, Y);
        free(Xl);
        free(B);
        free(tau2);
    } else {
        memcpy(Y, X, sizeof(orc_real) * nn);
        for (int j = 0; j < n; ++j) AT(Vacc, j, j, n) = 1.0;
        s.switch_off = scaled_offdiag(n, n, Y);
    }

refine:
    /* Refinement in working precision (Section 3.4): Alg. 1 on Y with V accumulated, or
     * (v_by_qr) without V, then V_X from the QR of X^T U_X (U_X sorted by descending norm, as
     * for the switch) and Alg. 1 with V accumulated from that start on Y = X Q3. */
    {
        orc_real tol = (p.tol > 0.0) ? p.tol : RSQRT((orc_real)n) * U_WORK;
        long long rot_pre = 0;  /* rotations of the safeguard, added to rot_work at the end */
        if (p.y_tol > 0.0) {
            /* Y1/Y2 safeguard: Y1 = the leading columns whose cosines with each other stay
             * below y_tol, Y2 = the rest; Alg. 1 on Y2 with its columns of V, then one sweep
             * of the pairs (p in Y1, q in Y2). */
            int j0 = n;
            for (int j = 1; j < n && j0 == n; ++j) {
                const orc_real nj = nrm2(n, &AT(Y, 0, j, n));
                for (int i = 0; i < j; ++i) {
                    orc_real g = 0.0;
                    for (int r = 0; r < n; ++r) g += AT(Y, r, i, n) * AT(Y, r, j, n);
                    const orc_real ni = nrm2(n, &AT(Y, 0, i, n));
                    if (RFABS(g) > p.y_tol * ni * nj) { j0 = j; break; }
                }
            }
            s.y2_cols = n - j0;
            if (j0 < n) {
                int sw2 = 0;
                long long rot2 = 0;
                orc_jacobi(n, n - j0, &AT(Y, 0, j0, n), n, &AT(Vacc, 0, j0, n), n, n, tol, p.maxsweep,
                           p.stop, &sw2, &rot2);
                double cmax = 0.0, tmax = 0.0;
                for (int pp = 0; pp < j0; ++pp)
                    for (int q = j0; q < n; ++q)
                        rot2 += jacobi_pair(n, &AT(Y, 0, pp, n), &AT(Y, 0, q, n), &AT(Vacc, 0, pp, n),
                                            &AT(Vacc, 0, q, n), n, tol, &cmax, &tmax);
                rot_pre = rot2;
            }
        }
        if (!p.v_by_qr) {
            int rc = orc_jacobi(n, n, Y, n, Vacc, n, n, tol, p.maxsweep, p.stop, &s.sweeps_work, &s.rot_work);
            if (rc != 0) s.status = 1;
        } else {
            int rc = orc_jacobi(n, n, Y, n, NULL, 1, 0, tol, p.maxsweep, p.stop, &s.sweeps_work, &s.rot_work);
            if (rc != 0) s.status = 1;
            orc_real* B3 = (orc_real*)malloc(sizeof(orc_real) * nn);
            orc_real* tau3 = (orc_real*)malloc(sizeof(orc_real) * (size_t)n);
            if (!B3 || !tau3) { free(B3); free(tau3); s.status = -9; goto done; }
            for (int j = 0; j < n; ++j) {
                sig[j] = nrm2(n, &AT(Y, 0, j, n));
                order[j] = j;
            }
            for (int a = 1; a < n; ++a) { /* stable insertion sort, descending */
                int oj = order[a];
                int b = a - 1;
                while (b >= 0 && sig[order[b]] < sig[oj]) { order[b + 1] = order[b]; --b; }
                order[b + 1] = oj;
            }
            for (int b = 0; b < n; ++b) { /* B3 = X^T U_X */
                const int j = order[b];
                const orc_real inv = (sig[j] > 0.0) ? 1.0 / sig[j] : 0.0;
                for (int a = 0; a < n; ++a) {
                    orc_real acc = 0.0;
                    for (int i = 0; i < n; ++i) acc += AT(X, i, a, n) * AT(Y, i, j, n);
                    AT(B3, a, b, n) = acc * inv;
                }
            }
            orc_geqrf(n, n, B3, n, tau3);
            memset(Vacc, 0, sizeof(orc_real) * nn);
            for (int j = 0; j < n; ++j) AT(Vacc, j, j, n) = 1.0;
            orc_apply_q(0, n, n, n, B3, n, tau3, Vacc, n); /* Vacc = Q3 */
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    orc_real acc = 0.0;
                    for (int i = 0; i < n; ++i) acc += AT(X, a, i, n) * AT(Vacc, i, b, n);
                    AT(Y, a, b, n) = acc;
                }
            free(B3);
            free(tau3);
            long long rot_v = 0;
            rc = orc_jacobi(n, n, Y, n, Vacc, n, n, tol, p.maxsweep, p.stop, &s.sweeps_v, &rot_v);
            if (rc != 0) s.status = 1;
            s.rot_work += rot_v;
        }
        s.rot_work += rot_pre;
    }

    /* Sigma = column norms, U_X = normalized columns, sorted descending (Alg. 1). */
    for (int j = 0; j < n; ++j) {
        sig[j] = nrm2(n, &AT(Y, 0, j, n));
        order[j] = j;
    }
    for (int a = 1; a < n; ++a) { /* stable insertion sort, descending */
        int oj = order[a];
        int b = a - 1;
        while (b >= 0 && sig[order[b]] < sig[oj]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = oj;
    }
    /* X = U_X Sigma V_acc^T. For X = R: U_R = U_X, V_R = V_acc. For X = R^T the roles
     * exchange: R = V_acc Sigma U_X^T, so U_R = V_acc and V_R = U_X. For X = L = R Q':
     * R = U_X Sigma (Q' V_acc)^T, so U_R = U_X and V_R = Q' V_acc. */
    if (pc == 2) orc_apply_q(0, n, n, n, Lq, n, tauq, Vacc, n);
    for (int k = 0; k < n; ++k) {
        int j = order[k];
        S[k] = sig[j];
        for (int i = 0; i < n; ++i) {
            orc_real ux = (sig[j] > 0.0) ? AT(Y, i, j, n) / sig[j] : 0.0;
            orc_real uR = (pc == 0) ? AT(Vacc, i, j, n) : ux;
            orc_real vR = (pc == 0) ? ux : AT(Vacc, i, j, n);
            AT(Ux, i, k, m) = uR;
            /* V = P V_R: row jpvt[i] of V is row i of V_R (Alg. 2, V <- P V_X). */
            AT(V, jpvt[i], k, n) = vR;
        }
    }
    /* U = Q0 Q1 [U_X; 0] (Alg. 4, last line). */
    orc_apply_q(0, n, n, n, R, n, tau1, Ux, m);
    if (m > n) orc_apply_q(0, m, n, n, W0, m, tau0, Ux, m);
    /* Sign convention: the largest-magnitude entry of each v_k is positive. */
    for (int k = 0; k < n; ++k) {
        int r = 0;
        for (int i = 1; i < n; ++i)
            if (RFABS(AT(V, i, k, n)) > RFABS(AT(V, r, k, n))) r = i;
        orc_real sgn = (AT(V, r, k, n) < 0.0) ? -1.0 : 1.0;
        for (int i = 0; i < n; ++i) AT(V, i, k, n) *= sgn;
        for (int i = 0; i < m; ++i) AT(U, i, k, m) = sgn * AT(Ux, i, k, m);
    }

done:
    free(W0); free(tau0); free(R); free(tau1); free(jpvt); free(X); free(Y);
    free(Vacc); free(Ux); free(order); free(sig); free(Lq); free(tauq);
    if (st) *st = s;
    return s.status;
}

/* ---------------------------------------------------------------------------------
 * Adjoint of the thin SVD A = U S V^T (m >= n, U^T U = I, V^T V = I). With
 * dP = U^T dA V one has dS = diag(dP), U^T dU = F o (dP S + S dP^T),
 * V^T dV = F o (S dP + dP^T S), (I - U U^T) dU = (I - U U^T) dA V S^-1, where
 * F_ij = 1 / (s_j^2 - s_i^2) (i != j), F_ii = 0. Collecting <gS, dS> + <gU, dU> +
 * <gV, dV> = <gA, dA> gives
 *   gA = U [ (F o (U^T gU - gU^T U)) S + diag(gS) + S (F o (V^T gV - gV^T V)) ] V^T
 *        + (I - U U^T) gU S^-1 V^T.
 * ------------------------------------------------------------------------------- */
int orc_svd_backward(int m, int n, const orc_real* U, const orc_real* S, const orc_real* V,
                     const orc_real* gU, const orc_real* gS, const orc_real* gV, orc_real* gA,
                     orc_real gap_tol, int* n_flagged)
{
    if (n < 1 || m < n) return -1;
    const size_t nn = (size_t)n * (size_t)n;
    orc_real* M1 = (orc_real*)calloc(nn, sizeof(orc_real)); /* U^T gU */
    orc_real* M2 = (orc_real*)calloc(nn, sizeof(orc_real)); /* V^T gV */
    orc_real* K = (orc_real*)calloc(nn, sizeof(orc_real));
    orc_real* T = (orc_real*)calloc((size_t)m * (size_t)n, sizeof(orc_real));
    if (!M1 || !M2 || !K || !T) { free(M1); free(M2); free(K); free(T); return -9; }
    int flagged = 0;
    for (int i = 0; i < n; ++i) {
        if (S[i] <= U_WORK * S[0]) ++flagged;
        for (int j = i + 1; j < n; ++j) {
            orc_real big = S[i] > S[j] ? S[i] : S[j];
            if (RFABS(S[i] - S[j]) <= gap_tol * big) ++flagged;
        }
    }
    if (gU)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                orc_real acc = 0.0;
                for (int r = 0; r < m; ++r) acc += AT(U, r, i, m) * AT(gU, r, j, m);
                AT(M1, i, j, n) = acc;
            }
    if (gV)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                orc_real acc = 0.0;
                for (int r = 0; r < n; ++r) acc += AT(V, r, i, n) * AT(gV, r, j, n);
                AT(M2, i, j, n) = acc;
            }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            if (i == j) { AT(K, i, i, n) = gS ? gS[i] : 0.0; continue; }
            orc_real f = 1.0 / (S[j] * S[j] - S[i] * S[i]);
            AT(K, i, j, n) = f * (AT(M1, i, j, n) - AT(M1, j, i, n)) * S[j] +
                             S[i] * f * (AT(M2, i, j, n) - AT(M2, j, i, n));
        }
    /* T = U K + (gU - U M1) S^-1 */
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < m; ++r) {
            orc_real acc = 0.0;
            for (int i = 0; i < n; ++i) acc += AT(U, r, i, m) * AT(K, i, j, n);
            if (gU) {
                orc_real proj = 0.0;
                for (int i = 0; i < n; ++i) proj += AT(U, r, i, m) * AT(M1, i, j, n);
                acc += (AT(gU, r, j, m) - proj) / S[j];
            }
            AT(T, r, j, m) = acc;
        }
    /* gA = T V^T */
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) {
            orc_real acc = 0.0;
            for (int j = 0; j < n; ++j) acc += AT(T, r, j, m) * AT(V, c, j, n);
            AT(gA, r, c, m) = acc;
        }
    free(M1); free(M2); free(K); free(T);
    if (n_flagged) *n_flagged = flagged;
    return 0;
}
