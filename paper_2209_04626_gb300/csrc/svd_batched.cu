// svd_batched.cu -- Algorithm 4 for thousands of independent matrices of uneven sizes in one
// persistent launch.
//
// Each CTA repeatedly takes the next matrix from a work queue ordered largest first (by
// n^2 m, sorted on the host) and runs the whole pipeline of Algorithm 4 on it alone: the
// stage routines are the same device functions the single-matrix path spreads over all SMs,
// called with a one-CTA group whose barrier is __syncthreads. Every CTA owns a workspace
// slot (its QRCP matrix, X, U_low, B, Y, V_acc, vectors and a state block) reused for each
// matrix it takes. Per-matrix convergence: every matrix runs its own sweep loops; its status
// bits go to info[i].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "internal.h"
#include "qr.cuh"
#include "sweep.cuh"

namespace mpj {

constexpr int kBatchThreads = 256;
// Kernel variants (block widths of the two Jacobi stages), chosen per size class of n by the
// autotuner: variant v runs binary32 blocks of kVarWLow[v] and binary64 blocks of kVarWWork[v].
constexpr int kBatchVariants = 4;
__host__ __device__ constexpr int var_wlow(int v) { return (v & 1) ? 16 : 8; }
__host__ __device__ constexpr int var_wwork(int v) { return (v & 2) ? 8 : 4; }
constexpr int kBatchDefaultVariant = 2;  // (8, 8)
// size classes of n: <= 32, <= 64, <= 128, <= 256, <= 512
__host__ __device__ inline int size_class(int n)
{
    return n <= 32 ? 0 : (n <= 64 ? 1 : (n <= 128 ? 2 : (n <= 256 ? 3 : 4)));
}

constexpr int kBatchClasses = 5;

struct BatchArgs {
    int batch;
    const int* order;        // matrix indices, largest first
    const int* m;
    const int* n;
    const int* lda;
    const double* const* A;
    double* const* U;
    double* const* S;
    double* const* V;
    int* info;
    unsigned int* queue;     // work counter (zeroed before the launch)
    char* slots;             // per-CTA workspace
    size_t slot_bytes;
    int max_m, max_n;
    mpjsvd_params P;
    double tol;
    int variant[kBatchClasses];  // per size class of n
};

// Offsets inside a slot for (max_m, max_n).
struct SlotLayout {
    size_t st, wq, wql, tau, perm, x, xl, g, cn, sigl, ord, ul, bq, tau2, perm2, y, vacc, sig,
        ord2, dsc, alph, wl, vn, total;
};

__host__ __device__ inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ inline SlotLayout slot_layout(int M, int N)
{
    SlotLayout L;
    size_t o = 0;
    size_t nn = (size_t)N * N, mn = (size_t)M * N;
    auto put = [&](size_t bytes) {
        size_t at = o;
        o += al256(bytes ? bytes : 16);
        return at;
    };
    L.st = put(sizeof(DevState));
    L.wq = put(8 * mn);
    L.wql = put(8 * mn);
    L.tau = put(8 * (size_t)N);
    L.perm = put(4 * (size_t)N);
    L.x = put(8 * nn);
    L.xl = put(4 * nn);
    L.g = put(4 * nn);
    L.cn = put(8 * (size_t)N);
    L.sigl = put(4 * (size_t)N);
    L.ord = put(4 * (size_t)N);
    L.ul = put(8 * nn);
    L.bq = put(8 * nn);
    L.tau2 = put(8 * (size_t)N);
    L.perm2 = put(4 * (size_t)N);
    L.y = put(8 * nn);
    L.vacc = put(8 * nn);
    L.sig = put(8 * (size_t)N);
    L.ord2 = put(4 * (size_t)N);
    L.dsc = put(8 * (size_t)N);
    L.alph = put(8 * (size_t)N);
    L.wl = put(4 * mn);            // lower(A) of Alg. 5's pivot search
    L.vn = put(8 * (size_t)N);     // its two norm arrays
    L.total = o;
    return L;
}

// ---- CTA-level building blocks (the single-matrix path has grid-wide versions)

template <typename T>
__device__ void cta_colnorms(int rows, int cols, const T* X, int ld, T* out)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < cols; c += nw) {
        const T* col = X + cm(0, c, ld);
        T s = T(0);
        for (int i = lane; i < rows; i += 32) s = fma(col[i], col[i], s);
        s = warp_sum(s);
        if (lane == 0) out[c] = sqrt(s);
    }
    __syncthreads();
}

// order[rank] = index, descending stable; NaN keys rank last.
template <typename T>
__device__ void cta_rank_desc(int n, const T* key, int* order)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
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
    __syncthreads();
}

template <typename T>
__device__ void cta_gemm(const GemmArgs& g)
{
    int tiles_m = (g.M + kGemmBM - 1) / kGemmBM;
    int tiles_n = (g.N + kGemmBN - 1) / kGemmBN;
    for (int t = 0; t < tiles_m * tiles_n; ++t)
        gemm_tile<T>(g, (t % tiles_m) * kGemmBM, (t / tiles_m) * kGemmBN);
    __syncthreads();
}

// Final assembly of one matrix (as k_finalize of the single-matrix path).
__device__ void cta_finalize(int m, int n, const double* Y, const double* Vacc, const double* sig,
                             const int* order, const int* jpvt, int precond, double* U, double* S,
                             double* V, int* status)
{
    __shared__ double s_val[32];
    __shared__ int s_row[32];
    __shared__ double s_sign;
    const bool rt = (precond != MPJSVD_PRECOND_R);
    for (int k = 0; k < n; ++k) {
        int j = order[k];
        double sj = sig[j];
        const double* y = Y + cm(0, j, n);
        const double* va = Vacc + cm(0, j, n);
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
            if (sj == 0.0) *status |= MPJSVD_STATUS_ZERO_SIGMA;
        }
        __syncthreads();
    }
}

// |x(lo:len)| of a binary32 column by one warp, on entries scaled by the power of two of their
// maximum (no square underflows or overflows: single-precision LAPACK's convention).
__device__ __forceinline__ float warp_norm_scaled(const float* x, int lo, int len)
{
    const int lane = threadIdx.x & 31;
    float a = 0.0f;
    for (int i = lo + lane; i < len; i += 32) a = fmaxf(a, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (a == 0.0f) return 0.0f;
    const float sc = __int_as_float((254 - ((__float_as_int(a) >> 23) & 0xff)) << 23);  // a sc in [1, 2)
    float s = 0.0f;
    for (int i = lo + lane; i < len; i += 32) {
        const float y = x[i] * sc;
        s = fmaf(y, y, s);
    }
    s = warp_sum(s);
    return sqrtf(s) / sc;
}

// Alg. 5, step 2, for one matrix by one CTA: the Businger-Golub pivot order of lower(A) in
// binary32 (A scaled by the power of two that brings max |a_ij| into [1, 2)), columns in the
// CTA's workspace (global memory, L2-resident). The rules of the binary64 kernels: the first
// maximum of the norms (in current column order) is the pivot; norms are downdated by the new
// row entry and recomputed when the downdate keeps less than half of the binary32 digits; the
// reflector's convention is that of the binary64 QR. Only perm (the pivot order) is kept.
__device__ void cta_qrcp_pivots_f32(int m, int n, const double* A, int lda, float* Lw, float* vn1,
                                    float* vn2, int* perm)
{
    __shared__ double s_dmax[32];
    __shared__ float s_bv[32];
    __shared__ int s_bi[32];
    __shared__ int s_p;
    __shared__ float s_tj, s_den;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const float tol3z = 2.44140625e-04f;  // sqrt(2^-24)
    double am = 0.0;
    for (size_t e = tid; e < (size_t)m * n; e += nthr) am = fmax(am, fabs(A[cm((int)(e % m), (int)(e / m), lda)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    if (lane == 0) s_dmax[wid] = am;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a = fmax(a, s_dmax[w]);
        s_dmax[0] = a;
    }
    __syncthreads();
    const double amax = s_dmax[0];
    const int eb = (__double2hiint(amax) >> 20) & 0x7ff;
    const double scale = (amax > 0.0) ? __hiloint2double((2046 - min(max(eb, 1), 2045)) << 20, 0) : 1.0;
    for (size_t e = tid; e < (size_t)m * n; e += nthr)
        Lw[e] = (float)(A[cm((int)(e % m), (int)(e / m), lda)] * scale);
    for (int c = tid; c < n; c += nthr) perm[c] = c;
    __syncthreads();
    for (int c = wid; c < n; c += nw) {
        const float v = warp_norm_scaled(Lw + (size_t)c * m, 0, m);
        if (lane == 0) { vn1[c] = v; vn2[c] = v; }
    }
    __syncthreads();
    const int k = min(m, n);
    for (int j = 0; j < k; ++j) {
        // pivot: the first maximum of vn1[j..n)
        float bv = -1.0f;
        int bi = n;
        for (int c = j + tid; c < n; c += nthr) {
            const float v = vn1[c];
            if (v > bv) { bv = v; bi = c; }  // increasing c per thread: first maximum kept
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            float b = -1.0f;
            int p = n;
            for (int w = 0; w < nw; ++w)
                if (s_bv[w] > b || (s_bv[w] == b && s_bi[w] < p)) { b = s_bv[w]; p = s_bi[w]; }
            s_p = (p < n) ? p : j;
        }
        __syncthreads();
        const int p = s_p;
        if (p != j) {
            float* cj = Lw + (size_t)j * m;
            float* cp = Lw + (size_t)p * m;
            for (int i = tid; i < m; i += nthr) {
                const float t = cj[i];
                cj[i] = cp[i];
                cp[i] = t;
            }
            __syncthreads();
            if (tid == 0) {
                const int ti = perm[j]; perm[j] = perm[p]; perm[p] = ti;
                vn1[p] = vn1[j];
                vn2[p] = vn2[j];
            }
        }
        __syncthreads();
        // reflector of Lw(j:m, j), stored in place (v(j) = 1 implied)
        float* colj = Lw + (size_t)j * m;
        if (wid == 0) {
            const float tailn = warp_norm_scaled(colj, j + 1, m);
            float tj = 0.0f, den = 1.0f;
            if (tailn != 0.0f) {
                const float alpha = colj[j];
                const float nrm = warp_norm_scaled(colj, j, m);
                const float beta = (alpha >= 0.0f) ? -nrm : nrm;
                tj = (beta - alpha) / beta;
                den = alpha - beta;
                __syncwarp();
                if (lane == 0) colj[j] = beta;
            }
            if (lane == 0) { s_tj = tj; s_den = den; }
        }
        __syncthreads();
        const float tj = s_tj, den = s_den;
        if (tj != 0.0f)
            for (int i = j + 1 + tid; i < m; i += nthr) colj[i] = colj[i] / den;
        __syncthreads();
        // apply H_j to the later columns (one warp per column), downdate their norms
        for (int c = j + 1 + wid; c < n; c += nw) {
            float* col = Lw + (size_t)c * m;
            if (tj != 0.0f) {
                float w = 0.0f;
                for (int i = j + 1 + lane; i < m; i += 32) w = fmaf(colj[i], col[i], w);
                w = warp_sum(w);
                w = tj * (col[j] + w);
                __syncwarp();
                if (lane == 0) col[j] -= w;
                for (int i = j + 1 + lane; i < m; i += 32) col[i] = fmaf(-w, colj[i], col[i]);
                __syncwarp();
            }
            const float v1 = vn1[c];
            if (v1 != 0.0f) {
                const float r = fabsf(col[j]) / v1;
                float q = 1.0f - r * r;
                q = q < 0.0f ? 0.0f : q;
                const float ratio = v1 / vn2[c];
                if (q * ratio * ratio <= tol3z) {
                    const float v = warp_norm_scaled(col, j + 1, m);
                    if (lane == 0) { vn1[c] = v; vn2[c] = v; }
                } else if (lane == 0) {
                    vn1[c] = v1 * sqrtf(q);
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

// The binary32 stage of one matrix with blocks of WL columns (one CTA, visits in order).
template <int WL>
__device__ bool low_sweeps(const SweepDims& D0, float* Xl, DevState* st, VisitShared<float, WL>& sm)
{
    SweepDims D = D0;
    D.w = WL;
    const int nb = (D.n + WL - 1) / WL;
    D.k = max(2, nb + (nb & 1));
    const Group g1{0, 1, st};
    bool conv = false;
    if (D.n <= (int)blockDim.x)
        jacobi_sweeps<float, false, WL, 1>(g1, D, Xl, nullptr, st->rot_sweep[0], st->mx_cos[0], st->mx_tan[0], sm, &conv);
    else
        jacobi_sweeps<float, false, WL, 2>(g1, D, Xl, nullptr, st->rot_sweep[0], st->mx_cos[0], st->mx_tan[0], sm, &conv);
    return conv;
}

// The binary64 refinement with V of one matrix with blocks of WW columns.
template <int WW>
__device__ bool work_sweeps(const SweepDims& D0, double* Y, double* Vacc, DevState* st, VisitShared<double, WW>& sm)
{
    SweepDims D = D0;
    D.w = WW;
    const int nb = (D.n + WW - 1) / WW;
    D.k = max(2, nb + (nb & 1));
    const Group g1{0, 1, st};
    bool conv = false;
    if (D.n <= (int)blockDim.x)
        jacobi_sweeps<double, true, WW, 1>(g1, D, Y, Vacc, st->rot_sweep[1], st->mx_cos[1], st->mx_tan[1], sm, &conv);
    else
        jacobi_sweeps<double, true, WW, 2>(g1, D, Y, Vacc, st->rot_sweep[1], st->mx_cos[1], st->mx_tan[1], sm, &conv);
    return conv;
}

// The whole of Algorithm 4 for one matrix by one CTA. Returns the status bits.
__device__ int svd_one(const BatchArgs& B, int mat, char* slot, unsigned char* smem)
{
    const int m = B.m[mat], n = B.n[mat], lda = B.lda[mat];
    const double* A = B.A[mat];
    double* U = B.U[mat];
    double* S = B.S[mat];
    double* V = B.V[mat];
    const mpjsvd_params& P = B.P;
    SlotLayout L = slot_layout(B.max_m, B.max_n);
    DevState* st = (DevState*)(slot + L.st);
    double* Wq = (double*)(slot + L.wq);
    double* WqL = (double*)(slot + L.wql);
    double* tau = (double*)(slot + L.tau);
    int* perm = (int*)(slot + L.perm);
    double* X = (double*)(slot + L.x);
    float* Xl = (float*)(slot + L.xl);
    float* G = (float*)(slot + L.g);
    double* cn = (double*)(slot + L.cn);
    float* sigl = (float*)(slot + L.sigl);
    int* ord = (int*)(slot + L.ord);
    double* Ul = (double*)(slot + L.ul);
    double* Bq = (double*)(slot + L.bq);
    double* tau2 = (double*)(slot + L.tau2);
    int* perm2 = (int*)(slot + L.perm2);
    double* Y = (double*)(slot + L.y);
    double* Vacc = (double*)(slot + L.vacc);
    double* sig = (double*)(slot + L.sig);
    int* ord2 = (int*)(slot + L.ord2);
    const size_t nn = (size_t)n * n;
    const int tid = threadIdx.x, nthr = blockDim.x;
    __shared__ int s_flag;
    __shared__ int s_status;
    __shared__ VisitShared<float, 8> sm_low8;
    __shared__ VisitShared<float, 16> sm_low16;
    __shared__ VisitShared<double, 4> sm_work4;
    __shared__ VisitShared<double, 8> sm_work8;
    const int var = B.variant[size_class(n)];

    // state block: barrier words unused (group of one CTA), counters zeroed
    for (size_t i = tid; i < sizeof(DevState) / 4; i += nthr) ((int*)st)[i] = 0;
    if (tid == 0) { s_flag = 0; s_status = 0; }
    __syncthreads();

    // ---- copy A, check finiteness
    int bad = 0;
    for (size_t e = tid; e < (size_t)m * n; e += nthr) {
        int i = (int)(e % m), j = (int)(e / m);
        double v = A[cm(i, j, lda)];
        if (!isfinite(v)) bad = 1;
        Wq[cm(i, j, m)] = v;
    }
    if (__syncthreads_or(bad)) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        for (size_t e = tid; e < (size_t)m * n; e += nthr) U[e] = qnan;
        for (size_t e = tid; e < nn; e += nthr) V[e] = qnan;
        for (int e = tid; e < n; e += nthr) S[e] = qnan;
        return MPJSVD_STATUS_NONFINITE;
    }

    // ---- [3.1] RRQR of A (one CTA): Alg. 5 (binary32 pivot order, then the binary64 QR of
    // A P) or Businger-Golub in binary64
    Group g1{0, 1, st};
    if (P.qrcp == MPJSVD_QRCP_MIXED) {
        cta_qrcp_pivots_f32(m, n, A, lda, (float*)(slot + L.wl), (float*)(slot + L.vn),
                            (float*)(slot + L.vn) + B.max_n, perm);
        for (int j = 0; j < n; ++j) {
            const double* src = Wq + cm(0, perm[j], m);
            double* dst = WqL + cm(0, j, m);
            for (int i = tid; i < m; i += nthr) dst[i] = src[i];
        }
        __syncthreads();
        hh_qr<false>(g1, m, n, WqL, m, tau, perm2, (double*)smem);
        __syncthreads();
    } else {
        hh_qr<true>(g1, m, n, Wq, m, tau, perm, (double*)smem);
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const double* src = Wq + cm(0, perm[j], m);
            double* dst = WqL + cm(0, j, m);
            for (int i = tid; i < m; i += nthr) dst[i] = src[i];
        }
    }
    __syncthreads();  // X below reads entries other threads gathered
    for (size_t e = tid; e < nn; e += nthr) {
        int i = (int)(e % n), j = (int)(e / n);
        double v;
        if (P.precond == MPJSVD_PRECOND_R) v = (i <= j) ? WqL[cm(i, j, m)] : 0.0;
        else v = (i >= j) ? WqL[cm(j, i, m)] : 0.0;
        X[e] = v;
    }
    __syncthreads();

    // ---- [3.5] special cases
    int gate = 0;
    {
        cta_colnorms<double>(n, n, X, n, cn);
        if (tid == 0) {
            double mx = 0.0;
            for (int j = 0; j < n; ++j) mx = fmax(mx, cn[j]);
            double r00 = fabs(WqL[0]), rnn = fabs(WqL[cm(n - 1, n - 1, m)]);
            double cond = (rnn > 0.0) ? r00 / rnn : INFINITY;
            int ntrail = (int)ceil(P.trailing_frac * (double)n);
            int small = ntrail > 0;
            for (int j = n - ntrail; j < n; ++j)
                if (cn[j] > 2.44140625e-04 * mx) { small = 0; break; }
            int branch;
            if (P.mode == MPJSVD_MODE_PLAIN) branch = 4;
            else if (P.mode == MPJSVD_MODE_MIXED) branch = 0;
            else if (cond <= P.tol_cond_coef * pow((double)n, 0.25)) branch = 1;
            else if (small) branch = 2;
            else branch = -1;
            s_flag = branch;
        }
        __syncthreads();
        if (s_flag == -1) {  // orth test: Xt = low(X) D^-1, max |Xt^T Xt - I|
            const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
            for (int c = wid; c < n; c += nw) {
                const double* col = X + cm(0, c, n);
                float s = 0.0f;
                for (int i = lane; i < n; i += 32) { float v = (float)col[i]; s = fmaf(v, v, s); }
                s = warp_sum(s);
                float d = sqrtf(s);
                for (int i = lane; i < n; i += 32) {
                    float v = (float)col[i];
                    Xl[cm(i, c, n)] = (d > 0.0f) ? v / d : 0.0f;
                }
            }
            __syncthreads();
            GemmArgs ga;
            ga.M = n; ga.N = n; ga.K = n; ga.A = Xl; ga.lda = n; ga.transA = true;
            ga.B = Xl; ga.ldb = n; ga.transB = false; ga.C = G; ga.ldc = n;
            ga.klo_from_row = (P.precond != MPJSVD_PRECOND_R);
            ga.khi_from_row = (P.precond == MPJSVD_PRECOND_R);
            cta_gemm<float>(ga);
            float mx = 0.0f;
            for (size_t e = tid; e < nn; e += nthr) {
                int i = (int)(e % n), j = (int)(e / n);
                mx = fmaxf(mx, fabsf(G[e] - (i == j ? 1.0f : 0.0f)));
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            __shared__ float s_mx[32];
            if (lane == 0) s_mx[wid] = mx;
            __syncthreads();
            if (tid == 0) {
                float m2 = 0.0f;
                for (int w = 0; w < nw; ++w) m2 = fmaxf(m2, s_mx[w]);
                s_flag = (m2 <= P.tol_orth) ? 3 : 0;
            }
            __syncthreads();
        }
        gate = (s_flag == 0);
    }

    // ---- [3.2]-[3.3] low-precision stage and switch, or Y = X, V_acc = I
    if (gate) {
        for (size_t e = tid; e < nn; e += nthr) Xl[e] = (float)X[e];
        __syncthreads();
        SweepDims D;
        D.n = n; D.mX = n; D.ldX = n; D.nV = 0; D.ldV = n;
        D.maxsweep = min(P.maxsweep, 64);
        D.stop = P.stop;
        D.tol = sqrt((double)n) * 5.9604644775390625e-08;
        float* dscf = (float*)(slot + L.dsc);
        D.dsc = dscf;
        D.alph = slot + L.alph;
        D.ver = nullptr;  // one CTA per matrix: visits run in order, no hand-off
        for (int j = tid; j < n; j += nthr) dscf[j] = 1.0f;
        __syncthreads();
        const bool conv = (var_wlow(var) == 16) ? low_sweeps<16>(D, Xl, st, sm_low16)
                                                : low_sweeps<8>(D, Xl, st, sm_low8);
        fold_scales_cols<float>(g1, n, n, Xl, n, 0, nullptr, n, dscf);
        if (!conv) s_status |= MPJSVD_STATUS_NOT_CONVERGED;
        __syncthreads();
        cta_colnorms<float>(n, n, Xl, n, sigl);
        cta_rank_desc<float>(n, sigl, ord);
        for (size_t e = tid; e < nn; e += nthr) {
            int i = (int)(e % n), r = (int)(e / n);
            int j = ord[r];
            float s = sigl[j];
            Ul[e] = (s > 0.0f) ? (double)(Xl[cm(i, j, n)] / s) : 0.0;
        }
        __syncthreads();
        GemmArgs gb;
        gb.M = n; gb.N = n; gb.K = n; gb.A = X; gb.lda = n; gb.transA = true;
        gb.B = Ul; gb.ldb = n; gb.transB = false; gb.C = Bq; gb.ldc = n;
        gb.klo_from_row = (P.precond != MPJSVD_PRECOND_R);
        gb.khi_from_row = (P.precond == MPJSVD_PRECOND_R);
        cta_gemm<double>(gb);
        hh_qr<false>(g1, n, n, Bq, n, tau2, perm2, (double*)smem);
        for (size_t e = tid; e < nn; e += nthr) Vacc[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
        __syncthreads();
        apply_q_cols(false, n, n, Bq, n, tau2, Vacc, n, 0, n, 0);
        __syncthreads();
        GemmArgs gy;
        gy.M = n; gy.N = n; gy.K = n; gy.A = X; gy.lda = n; gy.transA = false;
        gy.B = Vacc; gy.ldb = n; gy.transB = false; gy.C = Y; gy.ldc = n;
        gy.klo_from_row = (P.precond == MPJSVD_PRECOND_R);
        gy.khi_from_row = (P.precond != MPJSVD_PRECOND_R);
        cta_gemm<double>(gy);
    } else {
        for (size_t e = tid; e < nn; e += nthr) {
            Y[e] = X[e];
            Vacc[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
        }
        __syncthreads();
    }

    // ---- [3.4] binary64 refinement with V
    {
        SweepDims D;
        D.n = n; D.mX = n; D.ldX = n; D.nV = n; D.ldV = n;
        D.maxsweep = min(P.maxsweep, 64);
        D.stop = P.stop;
        D.tol = (B.tol > 0.0) ? B.tol : sqrt((double)n) * 1.1102230246251565e-16;
        double* dscd = (double*)(slot + L.dsc);
        D.dsc = dscd;
        D.alph = slot + L.alph;
        D.ver = nullptr;  // one CTA per matrix: visits run in order, no hand-off
        for (int j = tid; j < n; j += nthr) dscd[j] = 1.0;
        __syncthreads();
        const bool conv = (var_wwork(var) == 8) ? work_sweeps<8>(D, Y, Vacc, st, sm_work8)
                                                : work_sweeps<4>(D, Y, Vacc, st, sm_work4);
        fold_scales_cols<double>(g1, n, n, Y, n, n, Vacc, n, dscd);
        if (!conv) s_status |= MPJSVD_STATUS_NOT_CONVERGED;
        __syncthreads();
    }

    // ---- assembly
    cta_colnorms<double>(n, n, Y, n, sig);
    cta_rank_desc<double>(n, sig, ord2);
    cta_finalize(m, n, Y, Vacc, sig, ord2, perm, P.precond, U, S, V, &s_status);
    __syncthreads();
    apply_q_cols(false, m, n, WqL, m, tau, U, m, 0, n, -1);
    __syncthreads();
    return s_status;
}

__global__ void k_batched(BatchArgs B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_idx;
    char* slot = B.slots + (size_t)blockIdx.x * B.slot_bytes;
    while (true) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(B.queue, 1u);
        __syncthreads();
        int idx = s_idx;
        __syncthreads();
        if (idx >= B.batch) break;
        int mat = B.order[idx];
        const int mi = B.m[mat], ni = B.n[mat], li = B.lda[mat];
        if (ni < 1 || ni > B.max_n || mi < ni || mi > B.max_m || li < mi) {
            // sizes outside the call's stated bounds (device-array call): reported, not run
            if (threadIdx.x == 0) B.info[mat] = -1;
            __syncthreads();
            continue;
        }
        int status = svd_one(B, mat, slot, smem_raw);
        if (threadIdx.x == 0) B.info[mat] = status;
        __syncthreads();
    }
}

// Largest first: order[rank] = i with rank by n_i^2 m_i descending (stable in i); matrices
// with sizes outside the bounds rank last (the kernel reports them with info = -1).
__global__ void k_batch_order(int batch, int max_m, int max_n, const int* m, const int* n, const int* lda,
                              int* order)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        auto key = [&](int j) {
            const int mj = m[j], nj = n[j];
            const bool ok = nj >= 1 && nj <= max_n && mj >= nj && mj <= max_m && lda[j] >= mj;
            return ok ? (double)nj * nj * mj : -1.0;
        };
        const double ki = key(i);
        int r = 0;
        for (int j = 0; j < batch; ++j) {
            const double kj = key(j);
            r += (kj > ki) || (kj == ki && j < i);
        }
        order[r] = i;
    }
}

static size_t batched_smem(int max_m, int max_n) { return hh_qr_smem_bytes(max_m, max_n, 1); }

// Workspace, launch configuration and the common arguments of a batched launch.
static int batched_setup(mpjsvd_ctx* h, int batch, int max_m, int max_n, BatchArgs& B, int& grid,
                         size_t& smem, int*& meta)
{
    smem = batched_smem(max_m, max_n);
    cudaError_t e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail("batched smem attribute", e);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched, kBatchThreads, smem);
    if (e != cudaSuccess) return cuda_fail("batched occupancy", e);
    if (occ < 1) return cuda_fail("batched occupancy (0 blocks fit)", cudaErrorInvalidConfiguration);
    grid = std::min(batch, occ * h->num_sms);
    SlotLayout L = slot_layout(max_m, max_n);
    const size_t slot_bytes = al256(L.total);
    const size_t meta_bytes = al256(sizeof(int) * (size_t)batch * 4) + 256;
    int rc = ensure_buffer(&h->bws, &h->bws_bytes, meta_bytes + slot_bytes * (size_t)grid);
    if (rc) return rc;
    char* base = (char*)h->bws;
    meta = (int*)base;
    B.queue = (unsigned int*)(base + al256(sizeof(int) * (size_t)batch * 4));
    B.slots = base + meta_bytes;
    B.slot_bytes = slot_bytes;
    B.max_m = max_m;
    B.max_n = max_n;
    B.P = h->params;
    for (int c = 0; c < kBatchClasses; ++c)
        B.variant[c] = h->params.block_w != 0 ? kBatchDefaultVariant
                                              : (h->bt_tuned[c] ? h->bt_variant[c] : kBatchDefaultVariant);
    return 0;
}

static int batched_launch(mpjsvd_ctx* h, const BatchArgs& B, int grid, size_t smem)
{
    cudaError_t e = cudaMemsetAsync(B.queue, 0, sizeof(unsigned int), h->stream);
    if (e != cudaSuccess) return cuda_fail("batched queue reset", e);
    k_batched<<<grid, kBatchThreads, smem, h->stream>>>(B);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("batched launch", e);
    ++h->launch_count;
    return 0;
}

// Autotuner: for every size class of n present in the batch and not tuned yet on this handle,
// run each kernel variant (block widths of the two stages) on a sample of that class's matrices
// (up to one per CTA slot of a wave), timed with CUDA events, and keep the fastest. The picks
// stay in the handle. Host-synchronizing; runs in the host-array call only.
static int batched_tune(mpjsvd_ctx* h, int batch, const int* m, const int* n, const int* lda,
                        const double* const* A, double* const* U, double* const* S, double* const* V,
                        double tol, int* info, int max_m, int max_n)
{
    if (h->params.block_w != 0) return 0;
    std::vector<int> cls[kBatchClasses];
    for (int i = 0; i < batch; ++i) cls[size_class(n[i])].push_back(i);
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return cuda_fail("tune event", cudaErrorUnknown);
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail("tune event", cudaErrorUnknown);
    }
    int rc = 0;
    for (int c = 0; c < kBatchClasses && rc == 0; ++c) {
        if (h->bt_tuned[c] || cls[c].empty()) continue;
        // a sample: the class's largest matrices first (the cost the launch is bound by)
        std::vector<int> smp = cls[c];
        std::stable_sort(smp.begin(), smp.end(), [&](int a, int b) {
            return (double)n[a] * n[a] * m[a] > (double)n[b] * n[b] * m[b];
        });
        BatchArgs B;
        int grid = 0;
        size_t smem = 0;
        int* meta = nullptr;
        if ((rc = batched_setup(h, batch, max_m, max_n, B, grid, smem, meta))) break;
        const int ns = std::min((int)smp.size(), grid);
        smp.resize(ns);
        std::vector<int> host(4 * (size_t)batch, 0);
        for (int i = 0; i < ns; ++i) host[i] = smp[i];
        for (int i = 0; i < batch; ++i) {
            host[batch + i] = m[i];
            host[2 * batch + i] = n[i];
            host[3 * batch + i] = lda[i];
        }
        cudaError_t e = cudaMemcpyAsync(meta, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice,
                                        h->stream);
        if (e != cudaSuccess) { rc = cuda_fail("tune metadata", e); break; }
        B.batch = ns;
        B.order = meta;
        B.m = meta + batch;
        B.n = meta + 2 * batch;
        B.lda = meta + 3 * batch;
        B.A = A; B.U = U; B.S = S; B.V = V; B.info = info; B.tol = tol;
        float best = 0.0f;
        int best_v = kBatchDefaultVariant;
        for (int v = 0; v < kBatchVariants && rc == 0; ++v) {
            for (int cc = 0; cc < kBatchClasses; ++cc) B.variant[cc] = v;
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && rc == 0; ++rep) {  // the second run is timed
                cudaEventRecord(ev[0], h->stream);
                rc = batched_launch(h, B, std::min(grid, ns), smem);
                cudaEventRecord(ev[1], h->stream);
                if (rc == 0 && cudaEventSynchronize(ev[1]) == cudaSuccess)
                    cudaEventElapsedTime(&ms, ev[0], ev[1]);
            }
            if (rc == 0 && (v == 0 || ms < best)) { best = ms; best_v = v; }
        }
        if (rc == 0) {
            h->bt_variant[c] = best_v;
            h->bt_ms[c] = best;
            h->bt_tuned[c] = true;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return rc;
}

int svd_batched(mpjsvd_ctx* h, int batch, const int* m, const int* n, const int* lda,
                const double* const* A, double* const* U, double* const* S, double* const* V,
                double tol, int* info)
{
    int max_m = 1, max_n = 1;
    for (int i = 0; i < batch; ++i) {
        max_m = std::max(max_m, m[i]);
        max_n = std::max(max_n, n[i]);
    }
    h->launch_count = 0;
    int rc = batched_tune(h, batch, m, n, lda, A, U, S, V, tol, info, max_m, max_n);
    if (rc) return rc;
    // largest first
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)n[a] * n[a] * m[a] > (double)n[b] * n[b] * m[b];
    });
    BatchArgs B;
    int grid = 0;
    size_t smem = 0;
    int* d_meta = nullptr;
    if ((rc = batched_setup(h, batch, max_m, max_n, B, grid, smem, d_meta))) return rc;
    std::vector<int> host(4 * (size_t)batch);
    for (int i = 0; i < batch; ++i) {
        host[i] = order[i];
        host[batch + i] = m[i];
        host[2 * batch + i] = n[i];
        host[3 * batch + i] = lda[i];
    }
    // from pageable memory: the copy is staged before cudaMemcpyAsync returns, so the host
    // vector may go out of scope afterwards
    cudaError_t e = cudaMemcpyAsync(d_meta, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail("batched metadata copy", e);
    B.batch = batch;
    B.order = d_meta;
    B.m = d_meta + batch;
    B.n = d_meta + 2 * batch;
    B.lda = d_meta + 3 * batch;
    B.A = A; B.U = U; B.S = S; B.V = V; B.info = info; B.tol = tol;
    h->launch_count = 0;
    return batched_launch(h, B, grid, smem);
}

// Sizes in device memory (capturable in a CUDA graph: no host copy, no allocation once the
// workspace for (batch, max_m, max_n) exists): the order is computed on the device.
int svd_batched_dev(mpjsvd_ctx* h, int batch, int max_m, int max_n, const int* m, const int* n, const int* lda,
                    const double* const* A, double* const* U, double* const* S, double* const* V, double tol,
                    int* info)
{
    BatchArgs B;
    int grid = 0;
    size_t smem = 0;
    int* d_meta = nullptr;
    h->launch_count = 0;
    int rc = batched_setup(h, batch, max_m, max_n, B, grid, smem, d_meta);
    if (rc) return rc;
    k_batch_order<<<std::max(1, std::min(h->num_sms * 4, (batch + 255) / 256)), 256, 0, h->stream>>>(
        batch, max_m, max_n, m, n, lda, d_meta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("batched order", e);
    ++h->launch_count;
    B.batch = batch;
    B.order = d_meta;
    B.m = m;
    B.n = n;
    B.lda = lda;
    B.A = A; B.U = U; B.S = S; B.V = V; B.info = info; B.tol = tol;
    return batched_launch(h, B, grid, smem);
}

void batched_tuning(const mpjsvd_ctx* h, int* wl, int* ww, float* ms)
{
    for (int c = 0; c < kBatchClasses; ++c) {
        const int v = h->bt_tuned[c] ? h->bt_variant[c] : kBatchDefaultVariant;
        if (wl) wl[c] = h->bt_tuned[c] ? var_wlow(v) : 0;
        if (ww) ww[c] = h->bt_tuned[c] ? var_wwork(v) : 0;
        if (ms) ms[c] = h->bt_tuned[c] ? h->bt_ms[c] : 0.0f;
    }
}

}  // namespace mpj
