// qr_outer.cu -- two-level blocked Householder QR (Section 3.1: QR preconditioning; Section 3.3:
// QR of B and forming Q; Alg. 4 last line: U = Q [U_R; 0]) whose outer trailing updates run on
// the tensor cores.
//
// Outer panels of kQrOuter = 256 columns are factored by the one-level blocked QR of
// qr_blocked.cu (32-column cluster panels, binary64 compact-WY updates of the panel's own
// columns). The block of 256 reflectors H_j .. H_{j+255} is then applied to the trailing
// columns at once in the "UT" compact form (Joffrain, Low, Quintana-Orti, van de Geijn 2006):
//     Q_blk = I - V T V^T,   T^{-1} = S = striu(V^T V) + diag(1 / tau),
// so that
//     Q_blk^T C = C - V X,   S^T X = V^T C     (the QR's trailing update),
//     Q_blk   C = C - V X,   S   X = V^T C     (applying Q: forming Q, U = Q [U_R; 0]),
// with V the explicit unit lower-trapezoidal reflector block (zeros above the diagonal, ones on
// it) and G = V^T V in binary64. X comes from a triangular substitution in binary64 (x_i is
// multiplied by tau_i, so a zero reflector, tau = 0, contributes nothing); the two products
// V^T C (K = rows) and C - V X (K = 256) are binary64 products on the bf16 tensor cores by
// error-free operand splitting (ozaki.cu). Their scaling is per row of op(A) and per column
// of B: per reflector and per column of C for V^T C, per row of V and per column of X for
// V X, so the error of every product entry is a few units of 2^-56 of the largest entries of
// its own reflector (row of V) and its own column of C (X), the columnwise normwise error of
// the binary64 update (a column-scaled matrix stays accurate column by column).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"
#include "internal.h"

namespace mpj {

constexpr int kQrOuter = 256;

static inline size_t hcm(int i, int j, int ld) { return (size_t)j * (size_t)ld + (size_t)i; }
constexpr int kUtThreads = 64;  // columns per CTA of the triangular substitution

// Vx (mp x nb, ld mp) <- the explicit reflectors of the panel at A (geqrf layout, ld lda):
// Vx(i, k) = 0 for i < k, 1 for i = k, A(i, k) below.
__global__ void k_explicit_v(int mp, int nb, const double* __restrict__ A, int lda, double* __restrict__ Vx,
                             DevState* st, int gate_want)
{
    if (call_failed(st) || !gate_open(st, gate_want)) return;
    const size_t total = (size_t)mp * nb;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % mp), k = (int)(e / mp);
        Vx[e] = (i < k) ? 0.0 : ((i == k) ? 1.0 : A[cm(i, k, lda)]);
    }
}

// In place on X (nb x ncols, ld ldx; holds V^T C on entry): trans: S^T X = V^T C (forward,
// x_i = tau_i (w_i - sum_{l < i} G(l, i) x_l)), else S X = V^T C (backward, x_i = tau_i (w_i -
// sum_{l > i} G(i, l) x_l)); G = V^T V (nb x nb, ld nb). Thread per column; the column in
// shared memory (column stride kUtThreads + 1), G read by all threads alike (L1 broadcast).
__global__ void __launch_bounds__(kUtThreads)
    k_ut_solve(int nb, int ncols, const double* __restrict__ G, const double* __restrict__ tau, double* X,
               int ldx, bool trans, DevState* st, int gate_want)
{
    extern __shared__ double xs[];  // nb x (kUtThreads + 1)
    if (call_failed(st) || !gate_open(st, gate_want)) return;
    const int c = blockIdx.x * kUtThreads + threadIdx.x;
    const bool ok = c < ncols;
    double* col = X + (size_t)(ok ? c : 0) * ldx;
    for (int i = 0; i < nb; ++i) xs[i * (kUtThreads + 1) + threadIdx.x] = ok ? col[i] : 0.0;
    if (trans) {
        for (int i = 0; i < nb; ++i) {
            double s0 = xs[i * (kUtThreads + 1) + threadIdx.x], s1 = 0.0, s2 = 0.0, s3 = 0.0;
            const double* gi = G + (size_t)i * nb;  // G(l, i), l = 0 .. i - 1 (column i)
            int l = 0;
            for (; l + 3 < i; l += 4) {
                s0 = fma(-gi[l], xs[l * (kUtThreads + 1) + threadIdx.x], s0);
                s1 = fma(-gi[l + 1], xs[(l + 1) * (kUtThreads + 1) + threadIdx.x], s1);
                s2 = fma(-gi[l + 2], xs[(l + 2) * (kUtThreads + 1) + threadIdx.x], s2);
                s3 = fma(-gi[l + 3], xs[(l + 3) * (kUtThreads + 1) + threadIdx.x], s3);
            }
            for (; l < i; ++l) s0 = fma(-gi[l], xs[l * (kUtThreads + 1) + threadIdx.x], s0);
            xs[i * (kUtThreads + 1) + threadIdx.x] = ((s0 + s1) + (s2 + s3)) * tau[i];
        }
    } else {
        for (int i = nb - 1; i >= 0; --i) {
            double s0 = xs[i * (kUtThreads + 1) + threadIdx.x], s1 = 0.0, s2 = 0.0, s3 = 0.0;
            // G(i, l) = G(l, i), l = i + 1 .. nb - 1: column i of the symmetric G
            const double* gi = G + (size_t)i * nb;
            int l = i + 1;
            for (; l + 3 < nb; l += 4) {
                s0 = fma(-gi[l], xs[l * (kUtThreads + 1) + threadIdx.x], s0);
                s1 = fma(-gi[l + 1], xs[(l + 1) * (kUtThreads + 1) + threadIdx.x], s1);
                s2 = fma(-gi[l + 2], xs[(l + 2) * (kUtThreads + 1) + threadIdx.x], s2);
                s3 = fma(-gi[l + 3], xs[(l + 3) * (kUtThreads + 1) + threadIdx.x], s3);
            }
            for (; l < nb; ++l) s0 = fma(-gi[l], xs[l * (kUtThreads + 1) + threadIdx.x], s0);
            xs[i * (kUtThreads + 1) + threadIdx.x] = ((s0 + s1) + (s2 + s3)) * tau[i];
        }
    }
    if (ok)
        for (int i = 0; i < nb; ++i) col[i] = xs[i * (kUtThreads + 1) + threadIdx.x];
}

// The gate of a QR stage as a (pointer, value) pair for the product kernels (null: always).
static const int* gate_ptr(DevState* st, int gate_want, int* want)
{
    if (gate_want < 0) {
        *want = 0;
        return nullptr;
    }
    if (gate_want >= kGateY2) {
        *want = gate_want - kGateY2;
        return &st->gate_y2;
    }
    if (gate_want >= kGateLq) {
        *want = gate_want - kGateLq;
        return &st->gate_lq;
    }
    *want = gate_want;
    return &st->gate_low;
}

// Scratch of the outer updates for up to m rows and n columns (bytes; the one-level QR's own
// scratch for the 256-column panels comes after it).
static size_t outer_own_bytes(int m, int n)
{
    const size_t vx = sizeof(double) * (size_t)m * kQrOuter;
    const size_t g = sizeof(double) * (size_t)kQrOuter * kQrOuter;
    const size_t x = sizeof(double) * (size_t)kQrOuter * std::max(1, n);
    const size_t oz = std::max(ozaki_ws_bytes(kQrOuter, n, m), ozaki_ws_bytes(m, n, kQrOuter));
    auto r = [](size_t b) { return (b + 1023) & ~size_t(1023); };
    return r(vx) + r(g) + r(x) + r(oz);
}

size_t bqr_outer_ws_bytes(int m, int n)
{
    return outer_own_bytes(m, n) + sizeof(double) * bqr_wbuf_doubles(kQrOuter, m);
}

// Whether the two-level form with tensor-core updates runs for an m x n factorization (or an
// application of n reflectors) at this site of the pipeline under the handle's params.
// Measured on the large recipe (A = B D, D over 10 decades): 8192 x 8192 preconditioner QR
// 1254 -> 1108 ms, U assembly 984 -> 544 ms; the switch's QR and Q 2214 -> 1841 ms, but the
// refinement after it then rotates 12% more (its B is graded by rows, which the per-column
// scaling of the split products does not follow); at n = 2048 and 4096 the QRs are slower
// (51 -> 71 ms, 212 -> 244 ms), the U assembly at 4096 faster (133 -> 118 ms).
bool bqr_outer_used(const mpjsvd_ctx* h, int m, int n, int site)
{
    const int mode = h->params.qr_update;
    if (mode == MPJSVD_QRU_F64) return false;
    if (n <= kQrOuter || m < n) return false;
    if (mode == MPJSVD_QRU_TC) return true;
    if (site == kQrSitePrecond) return n >= kQrOuterMinNFactor;
    if (site == kQrSiteFinal || site == kQrSiteCall) return n >= kQrOuterMinNApply;
    return false;
}

struct OuterWs {
    double* Vx;
    double* G;
    double* X;
    void* oz;
    double* inner;
};
static OuterWs outer_ws(void* base, int m, int n)
{
    auto r = [](size_t b) { return (b + 1023) & ~size_t(1023); };
    unsigned char* p = (unsigned char*)base;
    OuterWs w;
    w.Vx = (double*)p;
    p += r(sizeof(double) * (size_t)m * kQrOuter);
    w.G = (double*)p;
    p += r(sizeof(double) * (size_t)kQrOuter * kQrOuter);
    w.X = (double*)p;
    p += r(sizeof(double) * (size_t)kQrOuter * std::max(1, n));
    w.oz = p;
    p += r(std::max(ozaki_ws_bytes(kQrOuter, n, m), ozaki_ws_bytes(m, n, kQrOuter)));
    w.inner = (double*)p;
    return w;
}

// C (mp x nc at C, ld ldc) <- (I - V op(T) V^T) C for the nb reflectors whose explicit block is
// in w.Vx (mp x nb) and whose Gram matrix is in w.G: trans (Q^T C) or not (Q C).
static int outer_update(mpjsvd_ctx* h, int mp, int nb, int nc, const double* tau, double* C, int ldc, bool trans,
                        const OuterWs& w, DevState* st, int gate_want)
{
    int want = 0;
    const int* gate = gate_ptr(st, gate_want, &want);
    GemmArgs g1;  // X = V^T C
    g1.M = nb; g1.N = nc; g1.K = mp;
    g1.A = w.Vx; g1.lda = mp; g1.transA = true;
    g1.B = C; g1.ldb = ldc; g1.transB = false;
    g1.C = w.X; g1.ldc = nb;
    g1.klo_from_row = false;  // op(A)(i, k) = V(k, i) = 0 for k < i: the tiles of 128 rows clip little
    g1.khi_from_row = false;
    int rc = ozaki_dgemm(h, g1, w.oz, gate, want, st);
    if (rc) return rc;
    const size_t smem = sizeof(double) * (size_t)nb * (kUtThreads + 1);
    cudaError_t e = cudaFuncSetAttribute(k_ut_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail("outer QR: solve smem attribute", e);
    k_ut_solve<<<(nc + kUtThreads - 1) / kUtThreads, kUtThreads, smem, h->stream>>>(nb, nc, w.G, tau, w.X, nb, trans,
                                                                                   st, gate_want);
    ++h->launch_count;
    GemmArgs g2;  // C <- C - V X
    g2.M = mp; g2.N = nc; g2.K = nb;
    g2.A = w.Vx; g2.lda = mp; g2.transA = false;
    g2.B = w.X; g2.ldb = nb; g2.transB = false;
    g2.C = C; g2.ldc = ldc;
    g2.klo_from_row = false;
    g2.khi_from_row = false;
    g2.sub = true;
    rc = ozaki_dgemm(h, g2, w.oz, gate, want, st);
    if (rc) return rc;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("outer QR update", e);
    return 0;
}

// Explicit reflector block and its Gram matrix for the nb reflectors of the panel at P.
static int outer_block(mpjsvd_ctx* h, int mp, int nb, const double* P, int ldp, const OuterWs& w, DevState* st,
                       int gate_want)
{
    const int grid = std::min(h->num_sms * 8, (int)(((size_t)mp * nb + 255) / 256));
    k_explicit_v<<<std::max(1, grid), 256, 0, h->stream>>>(mp, nb, P, ldp, w.Vx, st, gate_want);
    ++h->launch_count;
    int want = 0;
    const int* gate = gate_ptr(st, gate_want, &want);
    GemmArgs gg;  // G = V^T V in binary64 (the FP64 pipe: nb^2 mp flops)
    gg.M = nb; gg.N = nb; gg.K = mp;
    gg.A = w.Vx; gg.lda = mp; gg.transA = true;
    gg.B = w.Vx; gg.ldb = mp; gg.transB = false;
    gg.C = w.G; gg.ldc = nb;
    gg.klo_from_row = gg.khi_from_row = false;
    return launch_gemm_d(h, gg, gate, want);
}

int bqr_factor_outer(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau, void* W, DevState* st,
                     int gate_want)
{
    const OuterWs w = outer_ws(W, m, n);
    for (int jo = 0; jo < n; jo += kQrOuter) {
        const int nb = std::min(kQrOuter, n - jo), mp = m - jo;
        double* P = A + hcm(jo, jo, lda);
        int rc = bqr_factor(h, mp, nb, P, lda, tau + jo, w.inner, st, gate_want, kQrSiteCall);
        if (rc) return rc;
        const int nt = n - jo - nb;
        if (nt <= 0) break;
        if ((rc = outer_block(h, mp, nb, P, lda, w, st, gate_want))) return rc;
        if ((rc = outer_update(h, mp, nb, nt, tau + jo, A + hcm(jo, jo + nb, lda), lda, true, w, st, gate_want)))
            return rc;
    }
    return 0;
}

int bqr_apply_outer(mpjsvd_ctx* h, int m, int ncols, int k, const double* V, int ldv, const double* tau, double* C,
                    int ldc, bool ident, void* W, DevState* st, int gate_want)
{
    const OuterWs w = outer_ws(W, m, ncols);
    for (int jo = ((k - 1) / kQrOuter) * kQrOuter; jo >= 0; jo -= kQrOuter) {
        const int nb = std::min(kQrOuter, k - jo), mp = m - jo;
        const int cstart = ident ? jo : 0;
        const int nc = ncols - cstart;
        if (nc <= 0) continue;
        int rc = outer_block(h, mp, nb, V + hcm(jo, jo, ldv), ldv, w, st, gate_want);
        if (rc) return rc;
        if ((rc = outer_update(h, mp, nb, nc, tau + jo, C + hcm(jo, cstart, ldc), ldc, false, w, st, gate_want)))
            return rc;
    }
    return 0;
}

}  // namespace mpj
