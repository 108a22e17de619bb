// svd_single.cu -- Algorithm 4 of the paper for one matrix, every stage spread over all
// SMs. Stages (paper sections in brackets):
//   [3.1] QRCP of A (optionally after a plain QR when m > n)      hh_qr<true>, persistent
//   [3.5] special-case tests (cond_R, trailing norms, orth)        small kernels + FP32 GEMM
//   [3.2] FP32 one-sided Jacobi on low(X), U only                   jacobi_sweeps<float>
//   [3.3] switch: B = X^T U_low, B = Q R2, Y = X Q, V_acc = Q       GEMM, hh_qr<false>, GEMM
//   [3.4] FP64 one-sided Jacobi on Y accumulating V_acc             jacobi_sweeps<double>
//   [Alg. 1 end, Alg. 4 last line] Sigma, U_X, sort, U = Q [U_R; 0], V = P V_R
// The branch decision stays on the device (gate_low); the kernels of the skipped stage
// return immediately, so the whole call is asynchronous.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "gemm.cuh"
#include "internal.h"
#include "qr.cuh"
#include "sweep.cuh"

namespace mpj {

constexpr int kWmaxLow = 16;   // widest binary32 block (register-resident visits)
constexpr int kLowTcMinN = 5120;  // MPJSVD_LOWK_AUTO: tensor-core binary32 stage from this n on
// MPJSVD_GEMMK_AUTO: tensor-core binary64 products for n in [kGemmTcMinN, kGemmTcMaxN]. The
// split product keeps 56 bits of each row relative to the row's largest entry; on graded inputs
// the refinement then needs a few % more rotations (2048 x 1024 workload: +2.3%, a net gain of
// 1.4% of the SVD; 8192 x 8192: +10%, a net loss), so large n stays on the FP64 pipe.
constexpr int kGemmTcMinN = 1024;
constexpr int kGemmTcMaxN = 4096;
constexpr int kWmaxWork = 8;   // widest binary64 block
constexpr int kQrThreads = 256;
constexpr int kMaxGroupCtas = kQrSlotStride;  // CTAs of a cooperative QR launch

// True once the call cannot produce meaningful output: a non-finite input, or a
// cooperative stage that gave up on a bounded wait. Later stages then return at once.
__device__ __forceinline__ bool input_nonfinite(const DevState* st)
{
    return (*(volatile const int*)&st->status &
            (MPJSVD_STATUS_NONFINITE | MPJSVD_STATUS_TIMEOUT)) != 0;
}


// ------------------------------------------------------------------------------------
// elementwise / small kernels
// ------------------------------------------------------------------------------------

__global__ void k_copy_check(int m, int n, const double* __restrict__ A, int lda, double* W,
                             int ldw, DevState* st)
{
    size_t total = (size_t)m * n;
    int bad = 0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % m), j = (int)(e / m);
        double v = A[cm(i, j, lda)];
        if (!isfinite(v)) bad = 1;
        W[cm(i, j, ldw)] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->status, MPJSVD_STATUS_NONFINITE);
}

// Wq(0:n-1, 0:n-1) = triu(W0(0:n-1, :)), zeros below (R1 of the plain QR).
__global__ void k_extract_upper(int n, const double* __restrict__ W0, int ld0, double* Wq, int ldq)
{
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        Wq[cm(i, j, ldq)] = (i <= j) ? W0[cm(i, j, ld0)] : 0.0;
    }
}

// Logical order of the pivoted factorization: L(:, j) = W(:, perm[j]).
__global__ void k_gather_cols(int m, int n, const double* __restrict__ W, int ldw, const int* perm,
                              double* L, int ldl, const DevState* st)
{
    if (input_nonfinite(st)) return;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        int pj = perm[j];
        if (pj < 0 || pj >= n) continue;  // only after a failed stage (status already set)
        const double* src = W + cm(0, pj, ldw);
        double* dst = L + cm(0, j, ldl);
        for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = src[i];
    }
}

// The Jacobi input X from the upper triangle R of L (n x n part): X = R^T (precond RT), X = R
// (precond R), or, for precond L / AUTO, X = R'^T when st->gate_lq (Lq holds R' of the QR
// R^T = Q' R', so that R = R'^T Q'^T and L = R'^T) and X = R otherwise.
__global__ void k_form_x(int n, const double* __restrict__ L, int ldl, const double* __restrict__ Lq,
                         double* X, int precond, const DevState* st)
{
    const bool use_l = (precond >= MPJSVD_PRECOND_L) && *(volatile const int*)&st->gate_lq;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        double v;
        if (use_l) v = (i >= j) ? Lq[cm(j, i, n)] : 0.0;
        else if (precond != MPJSVD_PRECOND_RT) v = (i <= j) ? L[cm(i, j, ldl)] : 0.0;
        else v = (i >= j) ? L[cm(j, i, ldl)] : 0.0;
        X[cm(i, j, n)] = v;
    }
}

// Alg. 2's choice between X = R and X = L: gate_lq = 1 when force, or when some column of R
// is not diagonally dominant (|r_jj| < sum_{i<j} |r_ij|: R is not "almost diagonal").
// One warp per column.
__global__ void k_lq_decide(int n, const double* __restrict__ L, int ldl, int force, DevState* st)
{
    if (call_failed(st)) return;
    if (force) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->gate_lq = 1;
        return;
    }
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nw) {
        double off = 0.0;
        for (int i = lane; i < j; i += 32) off += fabs(L[cm(i, j, ldl)]);
        off = warp_sum(off);
        if (lane == 0 && off > fabs(L[cm(j, j, ldl)])) atomicOr(&st->gate_lq, 1);
    }
}

// Lq = R^T (n x n, zero above the diagonal) when gate_lq: the matrix whose QR gives L.
__global__ void k_rt_copy(int n, const double* __restrict__ L, int ldl, double* Lq, const DevState* st)
{
    if (call_failed(st) || !*(volatile const int*)&st->gate_lq) return;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        Lq[cm(i, j, n)] = (i >= j) ? L[cm(j, i, ldl)] : 0.0;
    }
}

// One warp per column: norms of an FP64 n-row matrix.
__global__ void k_colnorms(int rows, int cols, const double* __restrict__ X, int ldx, double* out)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < cols; c += nw) {
        const double* col = X + cm(0, c, ldx);
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s = fma(col[i], col[i], s);
        s = warp_sum(s);
        if (lane == 0) out[c] = sqrt(s);
    }
}

// Section 3.5 tests that need no GEMM: cond_R and the trailing-norm test. Decides the branch
// unless the orth test is still needed (branch = -1 then). One CTA.
__global__ void k_branch_first(int n, const double* __restrict__ X, const double* cn,
                               int mode, double tol_cond_coef, double trailing_frac, DevState* st)
{
    __shared__ double red[32];
    double mx = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, cn[j]);
    // block max
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, red[w]);
        st->maxnorm = m2;
        // cond_R from the diagonal of the Jacobi input X (that of R for X = R or R^T)
        double r00 = fabs(X[cm(0, 0, n)]), rnn = fabs(X[cm(n - 1, n - 1, n)]);
        double cond = (rnn > 0.0) ? r00 / rnn : INFINITY;
        st->cond_r = cond;
        int ntrail = (int)ceil(trailing_frac * (double)n);
        int trailing_small = ntrail > 0;
        const double sq_ulow = 2.44140625e-04;  // sqrt(2^-24)
        for (int j = n - ntrail; j < n; ++j)
            if (cn[j] > sq_ulow * m2) { trailing_small = 0; break; }
        double tol_cond = tol_cond_coef * pow((double)n, 0.25);
        int branch;
        if (mode == MPJSVD_MODE_PLAIN) branch = 4;
        else if (mode == MPJSVD_MODE_MIXED) branch = 0;
        else if (cond <= tol_cond) branch = 1;
        else if (trailing_small) branch = 2;
        else branch = -1;  // orth test decides
        st->branch = branch;
        st->gate_low = (branch == 0) ? 1 : 0;
        st->orth = -1.0;
    }
}

// Xt = low(X) D^-1 with D the binary32 column norms of low(X). One warp per column.
__global__ void k_scaled_low(int n, const double* __restrict__ X, float* Xt, const DevState* st)
{
    if (st->branch != -1) return;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < n; c += nw) {
        const double* col = X + cm(0, c, n);
        float s = 0.0f;
        for (int i = lane; i < n; i += 32) {
            float v = (float)col[i];
            s = fmaf(v, v, s);
        }
        s = warp_sum(s);
        float d = sqrtf(s);
        for (int i = lane; i < n; i += 32) {
            float v = (float)col[i];
            Xt[cm(i, c, n)] = (d > 0.0f) ? v / d : 0.0f;
        }
    }
}

template <typename T>
__global__ void k_gemm(GemmArgs g, const int* gate, int gate_want)
{
    if (gate && *(volatile const int*)gate != gate_want) return;
    int tiles_m = (g.M + kGemmBM - 1) / kGemmBM;
    int tiles_n = (g.N + kGemmBN - 1) / kGemmBN;
    for (int t = blockIdx.x; t < tiles_m * tiles_n; t += gridDim.x) {
        int tm = t % tiles_m, tn = t / tiles_m;
        gemm_tile<T>(g, tm * kGemmBM, tn * kGemmBN);
    }
}

// Binary64 switch GEMMs (dgemm_tile); gate as k_gemm.
__global__ void __launch_bounds__(kDgThreads) k_dgemm(GemmArgs g, const int* gate, int gate_want)
{
    if (gate && *(volatile const int*)gate != gate_want) return;
    dgemm_tile(g, blockIdx.x);
}

// orth = max |G - I| over the n x n FP32 Gram; atomicMax on the float bit pattern (>= 0).
__global__ void k_orth_max(int n, const float* __restrict__ G, DevState* st, unsigned int* bits)
{
    if (st->branch != -1) return;
    float mx = 0.0f;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        float v = fabsf(G[e] - (i == j ? 1.0f : 0.0f));
        mx = fmaxf(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits, __float_as_uint(mx));
}

__global__ void k_branch_final(DevState* st, const unsigned int* bits, double tol_orth)
{
    if (st->branch != -1) return;
    float orth = __uint_as_float(*bits);
    st->orth = orth;
    st->branch = (orth <= tol_orth) ? 3 : 0;
    st->gate_low = (st->branch == 0) ? 1 : 0;
}

__global__ void k_to_float(size_t count, const double* __restrict__ X, float* Xl, const DevState* st)
{
    if (!st->gate_low) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        Xl[e] = (float)X[e];
}

// Descending stable rank sort of n keys: order[rank] = index. Grid-stride, O(n^2).
template <typename T>
__global__ void k_rank_desc(int n, const T* __restrict__ key, int* order, const DevState* st,
                            int gate_want)
{
    if (gate_want >= 0 && st->gate_low != gate_want) return;
    // keys are norms (>= 0); a NaN key is ordered below every number, so the ranks always
    // form a permutation of 0..n-1
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        T kj = key[j];
        kj = (kj == kj) ? kj : T(-1);
        int r = 0;
        for (int i = 0; i < n; ++i) {
            T ki = key[i];
            ki = (ki == ki) ? ki : T(-1);
            r += (ki > kj) || (ki == kj && i < j);
        }
        order[r] = j;
    }
}

template <typename T>
__global__ void k_colnorms_gated(int rows, int cols, const T* __restrict__ X, int ldx, T* out,
                                 const DevState* st)
{
    if (!st->gate_low) return;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < cols; c += nw) {
        const T* col = X + cm(0, c, ldx);
        T s = T(0);
        for (int i = lane; i < rows; i += 32) s = fma(col[i], col[i], s);
        s = warp_sum(s);
        if (lane == 0) out[c] = sqrt(s);
    }
}

// Ul(:, r) = double(Xl(:, order[r]) / sig[order[r]]) (normalized in binary32, Alg. 1 end).
__global__ void k_make_ul(int n, const float* __restrict__ Xl, const float* sig, const int* order,
                          double* Ul, const DevState* st)
{
    if (!st->gate_low) return;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        int j = order[r];
        float s = sig[j];
        const float* src = Xl + cm(0, j, n);
        double* dst = Ul + cm(0, r, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            dst[i] = (s > 0.0f) ? (double)(src[i] / s) : 0.0;
    }
}

__global__ void k_identity(int n, double* Q, const DevState* st, int gate_want)
{
    if (gate_want >= 0 && st->gate_low != gate_want) return;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        Q[e] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void k_copy_gated(size_t count, const double* __restrict__ src, double* dst,
                             const DevState* st, int gate_want)
{
    if (st->gate_low != gate_want) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// C <- Q C on columns split across CTAs (no grid synchronization needed).
__global__ void k_apply_q(bool trans, int mrows, int ncols, int k, const double* Vr, int ldv,
                          const double* tau, double* C, int ldc, int per_cta, int ident,
                          const DevState* st, int gate_want)
{
    if (gate_want >= 0 && st->gate_low != gate_want) return;
    int c0 = blockIdx.x * per_cta;
    int c1 = min(ncols, c0 + per_cta);
    if (c0 >= c1) return;
    apply_q_cols(trans, mrows, k, Vr, ldv, tau, C, ldc, c0, c1, ident ? c0 : -1);
}

// Y1/Y2 partition of the safeguard: y_j0 = the first column j with |y_i^T y_j| > y_tol |y_i| |y_j|
// for some i < j (G = Y^T Y, cn = column norms); n if there is none.
__global__ void k_y_partition_init(int n, DevState* st)
{
    st->y_j0 = n;
    st->y2_cols_n = n;
}

__global__ void k_y_partition(int n, const double* __restrict__ G, const double* __restrict__ cn,
                              double y_tol, DevState* st)
{
    if (call_failed(st)) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nw) {
        int hit = 0;
        for (int i = lane; i < j; i += 32)
            if (fabs(G[cm(i, j, n)]) > y_tol * cn[i] * cn[j]) hit = 1;
        if (__any_sync(0xffffffffu, hit) && lane == 0) atomicMin(&st->y_j0, j);
    }
}

__global__ void k_y_partition_done(int n, DevState* st)
{
    st->gate_y2 = (st->y_j0 < n) ? 1 : 0;
}

// Ux(:, r) = Y(:, order[r]) / sig[order[r]] (binary64; the U_X of the refinement, sorted).
__global__ void k_make_ux(int n, const double* __restrict__ Y, const double* sig, const int* order,
                          double* Ux, const DevState* st)
{
    if (call_failed(st)) return;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const int j = order[r];
        const double sj = sig[j];
        const double inv = (sj > 0.0) ? 1.0 / sj : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) Ux[cm(i, r, n)] = Y[cm(i, j, n)] * inv;
    }
}

// ---- persistent cooperative kernels

__global__ void k_hhqr_piv(int m, int n, double* W, int ldw, double* tau, int* perm, DevState* st)
{
    extern __shared__ double qr_dyn[];
    if (input_nonfinite(st)) return;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    hh_qr<true>(g, m, n, W, ldw, tau, perm, qr_dyn);
}

__global__ void k_hhqr_res_piv(int m, int n, double* W, int ldw, double* tau, int* perm,
                               DevState* st, double* bcast)
{
    extern __shared__ double qr_dyn[];
    if (input_nonfinite(st)) return;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    hh_qr_res<true>(g, m, n, W, ldw, tau, perm, qr_dyn, bcast, nullptr);
}

__global__ void k_hhqr_res_plain(int m, int n, double* W, int ldw, double* tau, int* perm,
                                 DevState* st, double* bcast, int* flags, int gate_want)
{
    extern __shared__ double qr_dyn[];
    if (input_nonfinite(st)) return;
    if (gate_want >= 0 && *(volatile int*)&st->gate_low != gate_want) return;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    hh_qr_res<false>(g, m, n, W, ldw, tau, perm, qr_dyn, bcast, flags);
}

__global__ void k_hhqr_plain(int m, int n, double* W, int ldw, double* tau, int* perm, DevState* st,
                             int gate_want)
{
    extern __shared__ double qr_dyn[];
    if (input_nonfinite(st)) return;
    if (gate_want >= 0 && *(volatile int*)&st->gate_low != gate_want) return;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    hh_qr<false>(g, m, n, W, ldw, tau, perm, qr_dyn);
}

// Final assembly (Alg. 1 end; Alg. 4 last line). One CTA per output column k:
//   j = order[k]; S[k] = sig[j]; U_X(:, j) = Y(:, j) / sig[j];
//   precond R^T: U_R = V_acc(:, j), V_R = U_X(:, j);  precond R: U_R = U_X(:, j), V_R = V_acc(:, j)
//   V(jpvt[i], k) = s V_R(i, j); U(0:n-1, k) = s U_R(:, j); U(n:m-1, k) = 0,
// with s = +-1 making the largest-magnitude entry of V(:, k) positive (lowest row on ties).
__global__ void k_finalize(int m, int n, const double* __restrict__ Y, const double* __restrict__ Vacc,
                           const double* sig, const int* order, const int* jpvt, int precond,
                           double* U, double* S, double* V, DevState* st)
{
    __shared__ double s_val[32];
    __shared__ int s_row[32];
    __shared__ double s_sign;
    if (input_nonfinite(st)) {  // outputs are not meaningful: make that visible
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        for (int k = blockIdx.x; k < n; k += gridDim.x) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) U[cm(i, k, m)] = qnan;
            for (int i = threadIdx.x; i < n; i += blockDim.x) V[cm(i, k, n)] = qnan;
            if (threadIdx.x == 0) S[k] = qnan;
        }
        return;
    }
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        int j = order[k];
        double sj = sig[j];
        const double* y = Y + cm(0, j, n);
        const double* va = Vacc + cm(0, j, n);
        bool rt = (precond != MPJSVD_PRECOND_R);
        // sign from V_R
        double bv = -1.0;
        int br = 0x7fffffff;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double vr = rt ? ((sj > 0.0) ? y[i] / sj : 0.0) : va[i];
            double a = fabs(vr);
            int row = jpvt[i];
            if (a > bv || (a == bv && row < br)) { bv = a; br = row; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int orow = __shfl_xor_sync(0xffffffffu, br, o);
            if (ov > bv || (ov == bv && orow < br)) { bv = ov; br = orow; }
        }
        if ((threadIdx.x & 31) == 0) { s_val[threadIdx.x >> 5] = bv; s_row[threadIdx.x >> 5] = br; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b2 = -1.0;
            int r2 = 0x7fffffff;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (s_val[w] > b2 || (s_val[w] == b2 && s_row[w] < r2)) { b2 = s_val[w]; r2 = s_row[w]; }
            // find the signed value at row r2
            s_sign = 1.0;
            s_row[0] = r2;
        }
        __syncthreads();
        int rbest = s_row[0];
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (jpvt[i] == rbest) {
                double vr = rt ? ((sj > 0.0) ? y[i] / sj : 0.0) : va[i];
                s_sign = (vr < 0.0) ? -1.0 : 1.0;
            }
        }
        __syncthreads();
        double sg = s_sign;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double ux = (sj > 0.0) ? y[i] / sj : 0.0;
            double uR = rt ? va[i] : ux;
            double vR = rt ? ux : va[i];
            U[cm(i, k, m)] = sg * uR;
            V[cm(jpvt[i], k, n)] = sg * vR;
        }
        for (int i = n + threadIdx.x; i < m; i += blockDim.x) U[cm(i, k, m)] = 0.0;
        if (threadIdx.x == 0) {
            S[k] = sj;
            if (sj == 0.0) atomicOr(&st->status, MPJSVD_STATUS_ZERO_SIGMA);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------

static inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct SingleLayout {
    size_t off[40];  // >= L_COUNT (static_assert below)
    size_t total;
};

enum {
    L_WQ, L_WQL, L_W0, L_TAU0, L_TAU, L_PERM, L_IPOS, L_VN1, L_VN2, L_X, L_XL, L_CN, L_G,
    L_SIGL, L_ORD, L_UL, L_BQ, L_TAU2, L_Y, L_VACC, L_SIG, L_ORD2, L_BITS, L_PERM2, L_DSC,
    L_ALPH, L_BCAST, L_FLAGS, L_VER, L_WY, L_LQ, L_TAUQ, L_OZ, L_COUNT
};
static_assert(L_COUNT <= 40, "SingleLayout::off is too small");

// wy: scratch bytes of the blocked QRs and their applications (bqr_ws_bytes for m rows, n columns)
static SingleLayout single_layout(int m, int n, bool qr_first, bool lq, bool oz, size_t wy)
{
    size_t nn = (size_t)n * n;
    int mq = qr_first ? n : m;
    size_t sz[L_COUNT] = {};
    sz[L_WQ] = sizeof(double) * (size_t)mq * n;
    sz[L_WQL] = sizeof(double) * (size_t)mq * n;
    sz[L_W0] = qr_first ? sizeof(double) * (size_t)m * n : 0;
    sz[L_TAU0] = sizeof(double) * n;
    sz[L_TAU] = sizeof(double) * n;
    sz[L_PERM] = sizeof(int) * n;
    sz[L_IPOS] = sizeof(int) * n;
    sz[L_VN1] = sizeof(double) * n;
    sz[L_VN2] = sizeof(double) * n;
    sz[L_X] = sizeof(double) * nn;
    sz[L_XL] = sizeof(float) * nn;
    sz[L_CN] = sizeof(double) * n;
    sz[L_G] = sizeof(float) * nn;
    sz[L_SIGL] = sizeof(float) * n;
    sz[L_ORD] = sizeof(int) * n;
    sz[L_UL] = sizeof(double) * nn;
    sz[L_BQ] = sizeof(double) * nn;
    sz[L_TAU2] = sizeof(double) * n;
    sz[L_Y] = sizeof(double) * nn;
    sz[L_VACC] = sizeof(double) * nn;
    sz[L_SIG] = sizeof(double) * n;
    sz[L_ORD2] = sizeof(int) * n;
    sz[L_BITS] = 256;
    sz[L_PERM2] = sizeof(int) * n;
    sz[L_DSC] = sizeof(double) * n;
    sz[L_ALPH] = sizeof(double) * n;
    sz[L_BCAST] = std::max(sizeof(double) * (size_t)std::max(m, n) * (size_t)std::max(n, 2 * kMaxGroupCtas),
                           qrcp_low_bcast_bytes(qr_first ? n : m, n, kMaxGroupCtas));
    sz[L_FLAGS] = sizeof(int) * n;
    sz[L_VER] = sizeof(unsigned) * 2 * ((size_t)n + 2);  // 2 * sweep_blocks(n, w) for any w
    sz[L_WY] = wy;
    sz[L_LQ] = lq ? sizeof(double) * nn : 0;   // the QR of R^T (second preconditioning)
    sz[L_TAUQ] = lq ? sizeof(double) * n : 0;
    sz[L_OZ] = oz ? ozaki_ws_bytes(n, n, n) : 0;  // split operands of the tensor-core GEMMs
    // The QRCP's broadcast slots are live only during the QR preconditioning; the buffers
    // from X up to V_acc are first written after it, so the slots share their memory when
    // they fit (L_BITS, zeroed at the start of a call, is not in that span).
    size_t span = 0;
    for (int i = L_X; i < L_SIG; ++i) span += align256(sz[i] ? sz[i] : 16);
    const bool alias_bcast = sz[L_BCAST] <= span;
    if (alias_bcast) sz[L_BCAST] = 0;
    SingleLayout L;
    size_t o = 0;
    for (int i = 0; i < L_COUNT; ++i) {
        L.off[i] = o;
        o += align256(sz[i] ? sz[i] : 16);
    }
    if (alias_bcast) L.off[L_BCAST] = L.off[L_X];
    L.total = o;
    return L;
}

static int sweep_blocks(int n, int w)
{
    int nb = (n + w - 1) / w;
    return std::max(2, nb + (nb & 1));
}

// Block width of the sweeps. FP64 (work): narrow blocks, so that enough visits run at once
// for several CTAs per SM (the stage is FP64-throughput bound once latency is hidden).
// FP32 (low): wide blocks (the stage is latency bound: fewer rounds). A visit keeps 2w
// columns x (mX / threads) rows in registers, which caps w for tall X (<= 1024 threads,
// <= 32 doubles / 64 floats each).
static int pick_w(int n, int mX, bool low, int sms, int forced)
{
    int wmax = low ? kWmaxLow : kWmaxWork;
    int rpt_min = std::max(2, (mX + 1023) / 1024);
    int smem_cap = std::max(1, (low ? 64 : 32) / rpt_min);
    int w;
    if (forced > 0) {
        w = forced;
    } else if (low) {
        w = 8;
    } else {
        // narrowest power of two that leaves fewer than 0.75 visits per SM in a round: a
        // sweep is a chain of n / w - 1 rounds, so wider blocks shorten it, while the visits
        // of a round (and of the next rounds, released as their blocks arrive) still cover
        // the SMs (1024 columns: w = 4, 128 visits per round)
        w = 1;
        while ((double)n / (4.0 * w) >= 0.75 * sms) w *= 2;
        if (n <= 512) w = std::max(w, 8);  // small n: latency bound, fewer rounds win
    }
    w = std::min(w, std::min(wmax, smem_cap));
    w = std::min(w, std::max(1, n / 2));
    int p2 = 1;  // the kernels exist for power-of-two widths
    while (p2 * 2 <= w) p2 *= 2;
    return std::max(p2, 1);
}

// Resident variant (owned columns in shared memory) when they fit, else the global one.
// bcast: >= max(n, 2 * grid) * m doubles; flags: n ints (zeroed here for the plain QR).
static int launch_hhqr(mpjsvd_ctx* h, bool pivot, int m, int n, double* W, int ldw, double* tau,
                       int* perm, DevState* st, int gate_want, double* bcast, int* flags)
{
    int grid = std::max(1, std::min(n, std::min(h->num_sms, kMaxGroupCtas)));
    size_t rsmem = hh_qr_res_smem_bytes(m, n, grid);
    if (bcast && rsmem <= 200 * 1024) {
        void* kern = pivot ? (void*)k_hhqr_res_piv : (void*)k_hhqr_res_plain;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
        if (e != cudaSuccess) return cuda_fail("hhqr_res smem attribute", e);
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kQrThreads, rsmem);
        if (e != cudaSuccess) return cuda_fail("hhqr_res occupancy", e);
        if (occ >= 1) {
            if (pivot) {
                void* args[] = {&m, &n, &W, &ldw, &tau, &perm, &st, &bcast};
                e = cudaLaunchCooperativeKernel(kern, grid, kQrThreads, args, rsmem, h->stream);
            } else {
                e = cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n, h->stream);
                if (e != cudaSuccess) return cuda_fail("hhqr_res flags", e);
                void* args[] = {&m, &n, &W, &ldw, &tau, &perm, &st, &bcast, &flags, &gate_want};
                e = cudaLaunchCooperativeKernel(kern, grid, kQrThreads, args, rsmem, h->stream);
            }
            if (e != cudaSuccess) return cuda_fail("hhqr_res launch", e);
            ++h->launch_count;
            return 0;
        }
    }
    size_t smem = hh_qr_smem_bytes(m, n, grid);
    if (smem > 200 * 1024) return cuda_fail("hh_qr: too many rows", cudaErrorInvalidValue);
    void* kern = pivot ? (void*)k_hhqr_piv : (void*)k_hhqr_plain;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail("hhqr smem attribute", e);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kQrThreads, smem);
    if (e != cudaSuccess) return cuda_fail("hhqr occupancy", e);
    if (occ < 1) return cuda_fail("hhqr occupancy (0 blocks fit)", cudaErrorInvalidConfiguration);
    if (pivot) {
        void* args[] = {&m, &n, &W, &ldw, &tau, &perm, &st};
        e = cudaLaunchCooperativeKernel(kern, grid, kQrThreads, args, smem, h->stream);
    } else {
        void* args[] = {&m, &n, &W, &ldw, &tau, &perm, &st, &gate_want};
        e = cudaLaunchCooperativeKernel(kern, grid, kQrThreads, args, smem, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail("hhqr launch", e);
    ++h->launch_count;
    return 0;
}

static int launch_apply_q(mpjsvd_ctx* h, int mrows, int ncols, int k, const double* Vr, int ldv,
                          const double* tau, double* C, int ldc, bool ident, DevState* st,
                          int gate_want)
{
    int per = std::max(1, (ncols + h->num_sms - 1) / h->num_sms);
    int grid = (ncols + per - 1) / per;
    k_apply_q<<<grid, 256, 0, h->stream>>>(false, mrows, ncols, k, Vr, ldv, tau, C, ldc, per,
                                           ident ? 1 : 0, st, gate_want);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("apply_q launch", e);
    ++h->launch_count;
    return 0;
}

int launch_gemm_d(mpjsvd_ctx* h, const GemmArgs& g, const int* gate, int want)
{
    const int tiles = ((g.M + kDgBM - 1) / kDgBM) * ((g.N + kDgBN - 1) / kDgBN);
    k_dgemm<<<tiles, kDgThreads, 0, h->stream>>>(g, gate, want);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("gemm launch", e);
    ++h->launch_count;
    return 0;
}

static void record(mpjsvd_ctx* h, int i)
{
    if (h->params.timing && h->have_events) cudaEventRecord(h->ev[i], h->stream);
}

int svd_single(mpjsvd_ctx* h, int m, int n, const double* A, int lda, double* U, double* S,
               double* V, double tol)
{
    const mpjsvd_params& P = h->params;
    const bool qr_first = P.qr_first && m > n;
    const bool lq = P.precond >= MPJSVD_PRECOND_L;
    // the n x n x n binary64 GEMMs (switch, safeguard, V from QR): on the tensor cores by
    // operand splitting, or on the FP64 pipe
    const bool oz = P.gemm_kernel == MPJSVD_GEMMK_TC ||
                    (P.gemm_kernel == MPJSVD_GEMMK_AUTO && n >= kGemmTcMinN && n <= kGemmTcMaxN);
    SingleLayout L = single_layout(m, n, qr_first, lq, oz, bqr_ws_bytes(h, m, n));
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, L.total);
    if (rc) return rc;
    char* base = (char*)h->ws;
    auto ptr = [&](int i) { return (void*)(base + L.off[i]); };
    double* Wq = (double*)ptr(L_WQ);
    double* WqL = (double*)ptr(L_WQL);
    double* W0 = (double*)ptr(L_W0);
    double* tau0 = (double*)ptr(L_TAU0);
    double* tau = (double*)ptr(L_TAU);
    int* perm = (int*)ptr(L_PERM);
    double* X = (double*)ptr(L_X);
    float* Xl = (float*)ptr(L_XL);
    double* cn = (double*)ptr(L_CN);
    float* G = (float*)ptr(L_G);
    float* sigl = (float*)ptr(L_SIGL);
    int* ord = (int*)ptr(L_ORD);
    double* Ul = (double*)ptr(L_UL);
    double* Bq = (double*)ptr(L_BQ);
    double* tau2 = (double*)ptr(L_TAU2);
    double* Y = (double*)ptr(L_Y);
    double* Vacc = (double*)ptr(L_VACC);
    double* sig = (double*)ptr(L_SIG);
    int* ord2 = (int*)ptr(L_ORD2);
    unsigned int* bits = (unsigned int*)ptr(L_BITS);
    int* perm2 = (int*)ptr(L_PERM2);
    void* dsc = ptr(L_DSC);
    void* alph = ptr(L_ALPH);
    double* bcast = (double*)ptr(L_BCAST);
    int* qflags = (int*)ptr(L_FLAGS);
    unsigned* ver = (unsigned*)ptr(L_VER);
    double* wy = (double*)ptr(L_WY);
    double* Lq = (double*)ptr(L_LQ);
    void* ozws = ptr(L_OZ);
    // The split product scales each row of op(A) by its largest entry. That suits X Q (the rows
    // of X = R^T carry the grading of A's columns) and the Gram Y^T Y (each row of Y^T is one
    // column of Y, compared with its own norm), but not X^T U (a column of X mixes the column
    // scales of R, so its small entries would lose relative accuracy): that product stays on the
    // FP64 pipe (measured on the 8192 x 8192 workload: with it split, the refinement needs 10%
    // more rotations).
    auto gemm64 = [&](const GemmArgs& ga, const int* gate, int want) {
        const bool split_ok = !ga.transA || ga.A == ga.B;
        return (oz && split_ok) ? ozaki_dgemm(h, ga, ozws, gate, want, (DevState*)h->dstate)
                                : launch_gemm_d(h, ga, gate, want);
    };
    double* tauq = (double*)ptr(L_TAUQ);
    // n x n factorizations are always blocked (every n <= 12288 has a panel width); the QRCP's
    // broadcast slots may alias the stage buffers, so no unblocked kernel runs after it
    if (bqr_nb(n) == 0) return cuda_fail("blocked QR: no panel width for n", cudaErrorInvalidValue);
    const bool blocked_m = bqr_nb(m) > 0 && m <= 12480;
    DevState* st = (DevState*)h->dstate;
    cudaStream_t s = h->stream;
    const int T256 = 256;
    const int egrid = h->num_sms * 4;
    const int mq = qr_first ? n : m;
    cudaError_t e;
    h->launch_count = 0;

    if ((rc = state_reset(h, st))) return rc;
    e = cudaMemsetAsync(bits, 0, 256, s);
    if (e != cudaSuccess) return cuda_fail("memset bits", e);
    record(h, 0);

    // ---- [3.1] QR preconditioning
    if (qr_first) {
        k_copy_check<<<egrid, T256, 0, s>>>(m, n, A, lda, W0, m, st); ++h->launch_count;
        if (blocked_m) {
            if ((rc = bqr_factor(h, m, n, W0, m, tau0, wy, st, -1, kQrSitePrecond))) return rc;
        } else {
            if ((rc = launch_hhqr(h, false, m, n, W0, m, tau0, perm2, st, -1, bcast, qflags))) return rc;
        }
        k_extract_upper<<<egrid, T256, 0, s>>>(n, W0, m, Wq, n); ++h->launch_count;
    } else {
        k_copy_check<<<egrid, T256, 0, s>>>(m, n, A, lda, Wq, m, st); ++h->launch_count;
    }
    // RRQR: Alg. 5 (binary32 pivots, then the blocked binary64 QR of A P in pivot order) or
    // the binary64 Businger-Golub kernel (reflectors gathered into pivot order afterwards)
    bool mixed_done = false;
    if (P.qrcp == MPJSVD_QRCP_MIXED && bqr_nb(mq) > 0 && mq <= 12480) {
        // the broadcast region: its own buffer, or the stage buffers it aliases (X .. V_acc)
        const size_t bc_bytes = (L.off[L_BCAST] == L.off[L_X]) ? (L.off[L_SIG] - L.off[L_X])
                                                                : (L.off[L_BCAST + 1] - L.off[L_BCAST]);
        rc = launch_qrcp_low(h, mq, n, Wq, mq, perm, (float*)bcast, bc_bytes, st);
        if (rc < 0) return rc;
        if (rc == 0) {
            k_gather_cols<<<std::min(n, egrid), T256, 0, s>>>(mq, n, Wq, mq, perm, WqL, mq, st); ++h->launch_count;
            if ((rc = bqr_factor(h, mq, n, WqL, mq, tau, wy, st, -1, kQrSitePrecond))) return rc;
            mixed_done = true;
        }
    }
    h->last_qrcp = mixed_done ? MPJSVD_QRCP_MIXED : MPJSVD_QRCP_F64;
    if (!mixed_done) {
        if ((rc = launch_hhqr(h, true, mq, n, Wq, mq, tau, perm, st, -1, bcast, qflags))) return rc;
        k_gather_cols<<<std::min(n, egrid), T256, 0, s>>>(mq, n, Wq, mq, perm, WqL, mq, st); ++h->launch_count;
    }
    if (lq) {
        // second preconditioning (Alg. 2): R = L Q2^T from the QR of R^T, when forced or when
        // R is not almost diagonal (decided on the device)
        k_lq_decide<<<std::max(1, std::min(egrid, (n * 32 + T256 - 1) / T256)), T256, 0, s>>>(
            n, WqL, mq, P.precond == MPJSVD_PRECOND_L ? 1 : 0, st); ++h->launch_count;
        k_rt_copy<<<egrid, T256, 0, s>>>(n, WqL, mq, Lq, st); ++h->launch_count;
        if ((rc = bqr_factor(h, n, n, Lq, n, tauq, wy, st, kGateLq + 1, kQrSiteSwitch))) return rc;
    }
    k_form_x<<<egrid, T256, 0, s>>>(n, WqL, mq, Lq, X, P.precond, st); ++h->launch_count;
    h->last_precond = P.precond;
    record(h, 1);

    // triangular structure of X for the GEMMs (unknown on the host for AUTO: full products)
    const bool x_lower = P.precond == MPJSVD_PRECOND_RT || P.precond == MPJSVD_PRECOND_L;
    const bool x_upper = P.precond == MPJSVD_PRECOND_R;

    // ---- [3.5] special cases
    k_colnorms<<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, n, X, n, cn); ++h->launch_count;
    k_branch_first<<<1, 1024, 0, s>>>(n, X, cn, P.mode, P.tol_cond_coef, P.trailing_frac, st); ++h->launch_count;
    if (P.mode == MPJSVD_MODE_AUTO) {
        k_scaled_low<<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, X, Xl, st); ++h->launch_count;
        GemmArgs g;
        g.M = n; g.N = n; g.K = n;
        g.A = Xl; g.lda = n; g.transA = true;
        g.B = Xl; g.ldb = n; g.C = G; g.ldc = n;
        // Xt^T Xt: X = R^T (lower) -> Xt(i, a) = 0 for i < a; X = R (upper) -> 0 for i > a
        g.klo_from_row = x_lower;
        g.khi_from_row = x_upper;
        int tiles = ((n + kGemmBM - 1) / kGemmBM) * ((n + kGemmBN - 1) / kGemmBN);
        // gate on branch == -1 is checked inside k_orth_max/k_branch_final; the Gram runs
        // unconditionally in auto mode (one FP32 GEMM, cheap)
        k_gemm<float><<<tiles, kGemmThreads, 0, s>>>(g, nullptr, 0); ++h->launch_count;
        k_orth_max<<<egrid, T256, 0, s>>>(n, G, st, bits); ++h->launch_count;
        k_branch_final<<<1, 1, 0, s>>>(st, bits, P.tol_orth); ++h->launch_count;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("branch kernels", e);
    record(h, 2);

    // ---- [3.2] binary32 Jacobi on low(X), U only (gated)
    const size_t nn = (size_t)n * n;
    // the register file bounds the width for tall X: fall back to narrower blocks
    // binary32 stage: the blocked tensor-core form (64-column blocks) or register-resident
    // level-1 visits
    // (the alternative switch needs the stage's V: register-resident visits replay it)
    const bool alt_switch = P.switch_method == MPJSVD_SWITCH_V;
    const bool low_tc = !alt_switch && (P.low_kernel == MPJSVD_LOWK_TC ||
                                        (P.low_kernel == MPJSVD_LOWK_AUTO && n >= kLowTcMinN));
    int w_low = low_tc ? 64 : sweep_fit_w_f32(n, pick_w(n, n, true, h->num_sms, P.block_w));
    // binary64 sweeps: one CTA per visit (width limited by its registers for tall Y), or every
    // visit split by rows over a cluster (block width 4)
    const int w_cta = sweep_fit_w_f64(n, pick_w(n, n, false, h->num_sms, P.block_w));
    const int w_cl = sweep_cl_width(P.block_w);
    const int work_cs = sweep_cl_size(n, P.work_kernel, P.work_cluster, w_cl);
    int w_work = work_cs ? w_cl : w_cta;
    if (w_low == 0 || (w_cta == 0 && work_cs == 0))
        return cuda_fail("sweeps: no register-resident variant holds n rows", cudaErrorInvalidValue);
    h->last_block_w_low = (P.mode == MPJSVD_MODE_PLAIN) ? 0 : w_low;
    h->last_block_w_work = w_work;
    h->last_work_cs = work_cs ? work_cs : 1;
    // a binary64 sweep stage on Y (and V): the cluster form, else (or where the cluster launch is
    // unavailable) the single-CTA form at its own width
    auto work_sweeps = [&](const SweepDims& D, double* Yp, double* Vp, int phase, int gate) -> int {
        if (work_cs) {
            const int r = launch_sweeps_f64_cl(h, D, Yp, Vp, st, phase, gate, work_cs);
            if (r != 1) return r;
            if (w_cta == 0) return cuda_fail("sweeps: cluster launch unavailable", cudaErrorNotSupported);
            h->last_block_w_work = w_cta;
            h->last_work_cs = 1;
        }
        SweepDims Dc = D;
        Dc.w = w_cta;
        Dc.k = sweep_blocks(D.n, w_cta);
        return launch_sweeps_f64(h, Dc, Yp, Vp, st, phase, gate, nullptr);
    };
    if (P.mode != MPJSVD_MODE_PLAIN) {
        k_to_float<<<egrid, T256, 0, s>>>(nn, X, Xl, st); ++h->launch_count;
        const double tol_low = std::sqrt((double)n) * 5.9604644775390625e-08;
        SweepDims Dl;
        Dl.n = n; Dl.mX = n; Dl.ldX = n; Dl.nV = 0; Dl.ldV = n; Dl.w = w_low;
        Dl.k = sweep_blocks(n, w_low); Dl.maxsweep = std::min(P.maxsweep, 64); Dl.tol = tol_low;
        Dl.stop = P.stop;
        Dl.dsc = dsc; Dl.alph = alph; Dl.ver = ver;
        if (alt_switch) {
            // the stage also accumulates its rotations into V_low (binary64 copy of the binary32
            // rotations), kept in B's buffer
            Dl.nV = n;
            k_identity<<<egrid, T256, 0, s>>>(n, Bq, st, 1); ++h->launch_count;
            if ((rc = launch_sweeps_f32v(h, Dl, Xl, Bq, st, 0, 1))) return rc;
            record(h, 3);
            // ---- [3.3] the alternative switch: V_low = Q R2, V_acc = Q, Y = X Q
            if ((rc = bqr_factor(h, n, n, Bq, n, tau2, wy, st, 1, kQrSiteSwitch))) return rc;
            k_identity<<<egrid, T256, 0, s>>>(n, Vacc, st, 1); ++h->launch_count;
            if ((rc = bqr_apply(h, n, n, n, Bq, n, tau2, Vacc, n, true, wy, st, 1, kQrSiteSwitch))) return rc;
            GemmArgs g2;
            g2.M = n; g2.N = n; g2.K = n;
            g2.A = X; g2.lda = n; g2.transA = false;
            g2.B = Vacc; g2.ldb = n; g2.C = Y; g2.ldc = n;
            g2.klo_from_row = x_upper;
            g2.khi_from_row = x_lower;
            if ((rc = gemm64(g2, &st->gate_low, 1))) return rc;
        } else {
            if (low_tc) {
                if ((rc = launch_bsweeps_tf32(h, Dl, Xl, st, 0, 1))) return rc;
            } else {
                if ((rc = launch_sweeps_f32(h, Dl, Xl, st, 0, 1, nullptr))) return rc;
            }
            k_colnorms_gated<float><<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, n, Xl, n, sigl, st); ++h->launch_count;
            k_rank_desc<float><<<(n + T256 - 1) / T256, T256, 0, s>>>(n, sigl, ord, st, 1); ++h->launch_count;
            k_make_ul<<<std::min(n, egrid), T256, 0, s>>>(n, Xl, sigl, ord, Ul, st); ++h->launch_count;
            record(h, 3);
            // ---- [3.3] switch: B = X^T U_low; B = Q R2; V_acc = Q; Y = X Q
            GemmArgs g;
            g.M = n; g.N = n; g.K = n;
            g.A = X; g.lda = n; g.transA = true;
            g.B = Ul; g.ldb = n; g.C = Bq; g.ldc = n;
            g.klo_from_row = x_lower;  // X^T upper when X lower
            g.khi_from_row = x_upper;
            if ((rc = gemm64(g, &st->gate_low, 1))) return rc;
            if ((rc = bqr_factor(h, n, n, Bq, n, tau2, wy, st, 1, kQrSiteSwitch))) return rc;
            k_identity<<<egrid, T256, 0, s>>>(n, Vacc, st, 1); ++h->launch_count;
            if ((rc = bqr_apply(h, n, n, n, Bq, n, tau2, Vacc, n, true, wy, st, 1, kQrSiteSwitch))) return rc;
            GemmArgs g2;
            g2.M = n; g2.N = n; g2.K = n;
            g2.A = X; g2.lda = n; g2.transA = false;
            g2.B = Vacc; g2.ldb = n; g2.C = Y; g2.ldc = n;
            g2.klo_from_row = x_upper;  // X upper: X(i, k) = 0 for k < i
            g2.khi_from_row = x_lower;  // X lower: X(i, k) = 0 for k > i
            if ((rc = gemm64(g2, &st->gate_low, 1))) return rc;
        }
    } else {
        record(h, 3);
    }
    // skipped low stage: Y = X, V_acc = I
    k_copy_gated<<<egrid, T256, 0, s>>>(nn, X, Y, st, 0); ++h->launch_count;
    k_identity<<<egrid, T256, 0, s>>>(n, Vacc, st, 0); ++h->launch_count;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("switch kernels", e);
    record(h, 4);

    // ---- [3.4] binary64 refinement with V accumulation
    const double tol_work = (tol > 0.0) ? tol : std::sqrt((double)n) * 1.1102230246251565e-16;
    SweepDims Dw;
    Dw.n = n; Dw.mX = n; Dw.ldX = n; Dw.nV = n; Dw.ldV = n; Dw.w = w_work;
    Dw.k = sweep_blocks(n, w_work); Dw.maxsweep = std::min(P.maxsweep, 64); Dw.tol = tol_work;
    Dw.stop = P.stop;
    Dw.dsc = dsc; Dw.alph = alph; Dw.ver = ver;
    if (P.y_tol > 0.0) {
        // Y1/Y2 safeguard (Section 3.4): Y2 = the columns of Y from the first one whose largest
        // cosine with an earlier column exceeds y_tol; Alg. 1 on Y2 (with its columns of V),
        // then one pass over the pairs between Y1 and Y2, then the refinement as usual. The
        // Gram Y^T Y goes to B's buffer (dead after the switch); j0 stays on the device.
        k_colnorms<<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, n, Y, n, cn); ++h->launch_count;
        GemmArgs gy;
        gy.M = n; gy.N = n; gy.K = n;
        gy.A = Y; gy.lda = n; gy.transA = true;
        gy.B = Y; gy.ldb = n; gy.C = Bq; gy.ldc = n;
        gy.klo_from_row = gy.khi_from_row = false;
        if ((rc = gemm64(gy, nullptr, 0))) return rc;
        k_y_partition_init<<<1, 1, 0, s>>>(n, st); ++h->launch_count;  // also records n
        k_y_partition<<<std::max(1, std::min(egrid, (n * 32 + T256 - 1) / T256)), T256, 0, s>>>(
            n, Bq, cn, P.y_tol, st); ++h->launch_count;
        k_y_partition_done<<<1, 1, 0, s>>>(n, st); ++h->launch_count;
        SweepDims Dy = Dw;
        Dy.filter = 1;
        Dy.j0 = &st->y_j0;
        if ((rc = work_sweeps(Dy, Y, Vacc, 2, kGateY2 + 1))) return rc;
        Dy.filter = 2;
        Dy.maxsweep = 1;
        if ((rc = work_sweeps(Dy, Y, Vacc, 2, kGateY2 + 1))) return rc;
    }
    if (!P.v_by_qr) {
        if ((rc = work_sweeps(Dw, Y, Vacc, 1, -1))) return rc;
    } else {
        // V from the QR of X^T U_X (Section 3.4): Alg. 1 on Y without V; U_X = the normalized
        // columns of Y sorted by descending norm; B3 = X^T U_X = Q3 R3; Y = X Q3 and Alg. 1
        // with V accumulated from V_acc = Q3
        SweepDims Dn = Dw;
        Dn.nV = 0;
        if ((rc = work_sweeps(Dn, Y, nullptr, 1, -1))) return rc;
        k_colnorms<<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, n, Y, n, sig); ++h->launch_count;
        k_rank_desc<double><<<(n + T256 - 1) / T256, T256, 0, s>>>(n, sig, ord2, st, -1); ++h->launch_count;
        k_make_ux<<<std::min(n, egrid), T256, 0, s>>>(n, Y, sig, ord2, Ul, st); ++h->launch_count;
        GemmArgs g3;
        g3.M = n; g3.N = n; g3.K = n;
        g3.A = X; g3.lda = n; g3.transA = true;
        g3.B = Ul; g3.ldb = n; g3.C = Bq; g3.ldc = n;
        g3.klo_from_row = x_lower;
        g3.khi_from_row = x_upper;
        if ((rc = gemm64(g3, nullptr, 0))) return rc;
        if ((rc = bqr_factor(h, n, n, Bq, n, tau2, wy, st, -1, kQrSiteSwitch))) return rc;
        k_identity<<<egrid, T256, 0, s>>>(n, Vacc, st, -1); ++h->launch_count;
        if ((rc = bqr_apply(h, n, n, n, Bq, n, tau2, Vacc, n, true, wy, st, -1, kQrSiteSwitch))) return rc;
        GemmArgs g4;
        g4.M = n; g4.N = n; g4.K = n;
        g4.A = X; g4.lda = n; g4.transA = false;
        g4.B = Vacc; g4.ldb = n; g4.C = Y; g4.ldc = n;
        g4.klo_from_row = x_upper;
        g4.khi_from_row = x_lower;
        if ((rc = gemm64(g4, nullptr, 0))) return rc;
        if ((rc = work_sweeps(Dw, Y, Vacc, 2, -1))) return rc;
    }
    record(h, 5);

    // ---- Sigma, U_X, sort, U = Q [U_R; 0], V = P V_R
    k_colnorms<<<std::max(1, (n * 32 + T256 - 1) / T256), T256, 0, s>>>(n, n, Y, n, sig); ++h->launch_count;
    k_rank_desc<double><<<(n + T256 - 1) / T256, T256, 0, s>>>(n, sig, ord2, st, -1); ++h->launch_count;
    if (lq) {
        // X = L = R Q': R = U_X Sigma (Q' V_acc)^T, so V_R = Q' V_acc
        if ((rc = bqr_apply(h, n, n, n, Lq, n, tauq, Vacc, n, false, wy, st, kGateLq + 1, kQrSiteSwitch))) return rc;
    }
    k_finalize<<<std::min(n, egrid), T256, 0, s>>>(m, n, Y, Vacc, sig, ord2, perm,
                                                    lq ? MPJSVD_PRECOND_R : P.precond, U, S, V, st); ++h->launch_count;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("finalize kernels", e);
    if (qr_first) {
        if ((rc = bqr_apply(h, n, n, n, WqL, n, tau, U, m, false, wy, st, -1, kQrSiteFinal))) return rc;
        if (blocked_m) {
            if ((rc = bqr_apply(h, m, n, n, W0, m, tau0, U, m, false, wy, st, -1, kQrSiteFinal))) return rc;
        } else {
            if ((rc = launch_apply_q(h, m, n, n, W0, m, tau0, U, m, false, st, -1))) return rc;
        }
    } else if (blocked_m) {
        if ((rc = bqr_apply(h, m, n, n, WqL, m, tau, U, m, false, wy, st, -1, kQrSiteFinal))) return rc;
    } else {
        if ((rc = launch_apply_q(h, m, n, n, WqL, m, tau, U, m, false, st, -1))) return rc;
    }
    record(h, 6);
    return 0;
}

// The preconditioner's RRQR as a standalone call (mpjsvd_geqp3): A P = Q R with the QR of A P
// in pivot order (geqrf layout) written over A and jpvt[j] = the column of A in position j.
int geqp3_call(mpjsvd_ctx* h, int m, int n, double* A, int lda, int* jpvt, double* tau)
{
    const size_t sz_tmp = align256(sizeof(double) * (size_t)m * n);
    const size_t sz_bc = align256(std::max(sizeof(double) * (size_t)std::max(m, n) * (size_t)std::max(n, 2 * kMaxGroupCtas),
                                           qrcp_low_bcast_bytes(m, n, kMaxGroupCtas)));
    const size_t sz_wy = align256(bqr_ws_bytes(h, m, n));
    const size_t sz_fl = align256(sizeof(int) * (size_t)n);
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, sz_tmp + sz_bc + sz_wy + sz_fl);
    if (rc) return rc;
    char* base = (char*)h->ws;
    double* tmp = (double*)base;
    double* bcast = (double*)(base + sz_tmp);
    double* wy = (double*)(base + sz_tmp + sz_bc);
    int* flags = (int*)(base + sz_tmp + sz_bc + sz_wy);
    DevState* st = (DevState*)h->dstate;
    cudaStream_t s = h->stream;
    const int egrid = h->num_sms * 4;
    h->launch_count = 0;
    if ((rc = state_reset(h, st))) return rc;
    cudaError_t e;
    bool mixed_done = false;
    if (h->params.qrcp == MPJSVD_QRCP_MIXED && bqr_nb(m) > 0 && m <= 12480) {
        rc = launch_qrcp_low(h, m, n, A, lda, jpvt, (float*)bcast, sz_bc, st);
        if (rc < 0) return rc;
        if (rc == 0) {
            k_gather_cols<<<std::min(n, egrid), 256, 0, s>>>(m, n, A, lda, jpvt, tmp, m, st); ++h->launch_count;
            if ((rc = bqr_factor(h, m, n, tmp, m, tau, wy, st, -1, kQrSitePrecond))) return rc;
            mixed_done = true;
        }
    }
    h->last_qrcp = mixed_done ? MPJSVD_QRCP_MIXED : MPJSVD_QRCP_F64;
    if (!mixed_done) {
        if ((rc = launch_hhqr(h, true, m, n, A, lda, tau, jpvt, st, -1, bcast, flags))) return rc;
        k_gather_cols<<<std::min(n, egrid), 256, 0, s>>>(m, n, A, lda, jpvt, tmp, m, st); ++h->launch_count;
    }
    e = cudaMemcpy2DAsync(A, sizeof(double) * lda, tmp, sizeof(double) * m, sizeof(double) * m, n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail("geqp3 copy back", e);
    e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_fail("geqp3 kernels", e);
}

static int n_minus_j0(const DevState& st) { return st.gate_y2 ? st.y2_cols_n - st.y_j0 : 0; }

int read_stats(mpjsvd_ctx* h, mpjsvd_stats* out)
{
    DevState st;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail("stream sync", e);
    e = cudaMemcpy(&st, h->dstate, sizeof(DevState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("stats copy", e);
    mpjsvd_stats r;
    memset(&r, 0, sizeof(r));
    r.status = st.status;
    r.branch = st.branch;
    r.sweeps_low = st.sweeps_low;
    r.sweeps_work = st.sweeps_work;
    r.rot_low = (long long)st.rot_low;
    r.rot_work = (long long)st.rot_work;
    r.cond_r = st.cond_r;
    r.orth = st.orth;
    r.block_w_low = st.branch == 0 ? h->last_block_w_low : 0;
    r.block_w_work = h->last_block_w_work;
    r.work_cluster = h->last_work_cs;
    for (int s = 0; s < 16; ++s) {
        r.rot_sweep_low[s] = s < st.sweeps_low ? (long long)st.rot_sweep[0][s] : 0;
        r.rot_sweep_work[s] = s < st.sweeps_work ? (long long)st.rot_sweep[1][s] : 0;
        unsigned cl = s < st.sweeps_low ? st.mx_cos[0][s] : 0u, cw = s < st.sweeps_work ? st.mx_cos[1][s] : 0u;
        memcpy(&r.cos_sweep_low[s], &cl, sizeof(float));
        memcpy(&r.cos_sweep_work[s], &cw, sizeof(float));
    }
    r.launches = h->launch_count;
    r.qrcp = h->last_qrcp;
    r.precond = h->last_precond >= MPJSVD_PRECOND_L ? (st.gate_lq ? MPJSVD_PRECOND_L : MPJSVD_PRECOND_R)
                                                    : h->last_precond;
    r.sweeps_v = st.sweeps_v;
    r.rot_v = (long long)st.rot_v;
    r.y2_cols = h->params.y_tol > 0.0 ? n_minus_j0(st) : 0;
    r.n_flagged = -1;
    if (h->last_flag_dev) {
        e = cudaMemcpy(&r.n_flagged, h->last_flag_dev, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail("stats: flag count", e);
    }
    if (h->params.timing && h->have_events) {
        float* t[6] = {&r.ms_qr, &r.ms_branch, &r.ms_low, &r.ms_switch, &r.ms_work, &r.ms_final};
        for (int i = 0; i < 6; ++i) cudaEventElapsedTime(t[i], h->ev[i], h->ev[i + 1]);
    }
    *out = r;
    return 0;
}

// ------------------------------------------------------------------------------------
// Allocation-free variant of mpjsvd_svd for callers that must not allocate device memory.
// Its scratch (the per-call state block plus the same workspace layout mpjsvd_svd uses) is
// one file-scope device array of kNoAllocBytes, present on every GPU that loads this
// library until the process exits. Every call shares it, so calls that overlap on the GPU
// (different streams, or different host threads without ordering) race on it. The state
// block is cleared by each call itself (svd_single's first memset), and the workspace holds
// nothing that must start at zero.
// ------------------------------------------------------------------------------------

constexpr size_t kNoAllocBytes = size_t(6) << 20;  // 6 MiB
constexpr int kNoAllocMaxM = 512;
constexpr int kNoAllocMaxN = 256;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device. In host code the symbol
// g_noalloc_scratch is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
static int noalloc_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return cuda_fail("mpjsvd_svd_noalloc: device index", cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail("mpjsvd_svd_noalloc: cudaGetSymbolAddress", e);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return 0;
}

// status[0] = the call's MPJSVD_STATUS_* bits, enqueued after the last stage.
__global__ void k_copy_status(const DevState* st, int* status)
{
    *status = *(volatile const int*)&st->status;
}

static int svd_noalloc(int m, int n, const double* A, int lda, double* U, double* S, double* V,
                       double tol, int* status, cudaStream_t stream)
{
    if (m > kNoAllocMaxM || n > kNoAllocMaxN)
        return cuda_fail("mpjsvd_svd_noalloc: m > 512 or n > 256 exceeds the static scratch",
                         cudaErrorInvalidValue);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("mpjsvd_svd_noalloc: cudaGetDevice", e);
    mpjsvd_ctx ctx;
    memset(&ctx, 0, sizeof(ctx));
    ctx.device = dev;
    mpjsvd_default_params(&ctx.params);
    // the workspace svd_single will ask for, from the same parameters it reads
    const size_t state_bytes = align256(sizeof(DevState));
    const size_t need = single_layout(m, n, ctx.params.qr_first && m > n,
                                      ctx.params.precond >= MPJSVD_PRECOND_L,
                                      ctx.params.gemm_kernel == MPJSVD_GEMMK_TC ||
                                          (ctx.params.gemm_kernel == MPJSVD_GEMMK_AUTO && n >= kGemmTcMinN &&
                                           n <= kGemmTcMaxN),
                                      bqr_ws_bytes(&ctx, m, n)).total;
    if (state_bytes + need > kNoAllocBytes)
        return cuda_fail("mpjsvd_svd_noalloc: workspace exceeds the static scratch",
                         cudaErrorInvalidValue);
    void* base = nullptr;
    int rc = noalloc_scratch(dev, &base);
    if (rc) return rc;
    e = cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("mpjsvd_svd_noalloc: SM count", e);
    ctx.stream = stream;
    ctx.dstate = base;
    void* const ws = (char*)base + state_bytes;
    ctx.ws = ws;
    ctx.ws_bytes = kNoAllocBytes - state_bytes;  // ensure_buffer never allocates below this
    ctx.have_events = false;
    rc = svd_single(&ctx, m, n, A, lda, U, S, V, tol);
    // a workspace request above ws_bytes would have replaced the static array by a cudaMalloc:
    // the size check above rules that out; if it ever did not, fail instead of continuing
    if (ctx.ws != ws || ctx.ws_bytes != kNoAllocBytes - state_bytes)
        return cuda_fail("mpjsvd_svd_noalloc: the workspace left the static scratch",
                         cudaErrorInvalidValue);
    if (rc) return rc;
    if (status) {
        k_copy_status<<<1, 1, 0, stream>>>((const DevState*)base, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail("mpjsvd_svd_noalloc: status copy", e);
    }
    return 0;
}

}  // namespace mpj

extern "C" int mpjsvd_svd_noalloc(int m, int n, const double* A, int lda, double* U, double* S,
                                  double* V, double tol, int* status, void* cuda_stream)
{
    if (m < 1 || m < n) return -1;
    if (n < 1) return -2;
    if (m > mpj::kNoAllocMaxM) {
        mpj::set_last_error("mpjsvd_svd_noalloc: m exceeds 512, the static scratch limit",
                            cudaErrorInvalidValue);
        return -1;
    }
    if (n > mpj::kNoAllocMaxN) {
        mpj::set_last_error("mpjsvd_svd_noalloc: n exceeds 256, the static scratch limit",
                            cudaErrorInvalidValue);
        return -2;
    }
    if (!A) return -3;
    if (lda < m) return -4;
    if (!U) return -5;
    if (!S) return -6;
    if (!V) return -7;
    if (!(tol <= 0.0 || (tol > 0.0 && tol < 1.0))) return -8;
    return mpj::svd_noalloc(m, n, A, lda, U, S, V, tol, status, (cudaStream_t)cuda_stream);
}
