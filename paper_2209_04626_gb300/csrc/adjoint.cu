// adjoint.cu -- reverse-mode derivative of the thin SVD (not part of the paper).
//
// With A = U S V^T (m >= n), dP = U^T dA V gives dS = diag(dP),
// U^T dU = F o (dP S + S dP^T), V^T dV = F o (S dP + dP^T S) and
// (I - U U^T) dU = (I - U U^T) dA V S^-1, F_ij = 1/(s_j^2 - s_i^2) (i != j), F_ii = 0.
// Collecting <gS, dS> + <gU, dU> + <gV, dV> = <gA, dA>:
//   gA = [U K' + gU S^-1] V^T,
//   K'_ij = F_ij (M1_ij - M1_ji) s_j + s_i F_ij (M2_ij - M2_ji) - M1_ij / s_j  (i != j),
//   K'_ii = gS_i - M1_ii / s_i,        M1 = U^T gU, M2 = V^T gV.
// Near-degenerate pairs and tiny singular values are counted, never clamped.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "gemm.cuh"
#include "internal.h"

namespace mpj {

__global__ void k_adj_gemm(GemmArgs g)
{
    int tiles_m = (g.M + kGemmBM - 1) / kGemmBM;
    int tiles_n = (g.N + kGemmBN - 1) / kGemmBN;
    for (int t = blockIdx.x; t < tiles_m * tiles_n; t += gridDim.x)
        gemm_tile<double>(g, (t % tiles_m) * kGemmBM, (t / tiles_m) * kGemmBN);
}

__global__ void k_adj_core(int n, const double* __restrict__ S, const double* M1, const double* M2,
                           const double* gS, double* K)
{
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        double si = S[i], sj = S[j];
        double m1ij = M1 ? M1[cm(i, j, n)] : 0.0;
        double v;
        if (i == j) {
            v = (gS ? gS[i] : 0.0) - m1ij / sj;
        } else {
            double f = 1.0 / (sj * sj - si * si);
            double a = M1 ? (m1ij - M1[cm(j, i, n)]) : 0.0;
            double b = M2 ? (M2[cm(i, j, n)] - M2[cm(j, i, n)]) : 0.0;
            v = f * a * sj + si * f * b - m1ij / sj;
        }
        K[e] = v;
    }
}

// T = T + gU S^-1 (T = U K' already)
__global__ void k_adj_addgu(int m, int n, const double* __restrict__ gU, const double* S, double* T)
{
    size_t total = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(e / m);
        T[e] += gU[e] / S[j];
    }
}

__global__ void k_adj_flags(int n, const double* __restrict__ S, double gap_tol, int* count)
{
    int local = 0;
    const double u = 1.1102230246251565e-16;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double si = S[i];
        if (si <= u * S[0]) ++local;
        for (int j = i + 1; j < n; ++j) {
            double sj = S[j];
            double big = fmax(si, sj);
            if (fabs(si - sj) <= gap_tol * big) ++local;
        }
    }
    if (local) atomicAdd(count, local);
}

static int launch(GemmArgs g, cudaStream_t s)
{
    int tiles = ((g.M + kGemmBM - 1) / kGemmBM) * ((g.N + kGemmBN - 1) / kGemmBN);
    k_adj_gemm<<<tiles, kGemmThreads, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_fail("adjoint gemm", e);
}

int svd_backward(mpjsvd_ctx* h, int m, int n, const double* U, const double* S, const double* V,
                 const double* gU, const double* gS, const double* gV, double* gA, double gap_tol,
                 int* n_flagged)
{
    size_t nn = (size_t)n * n;
    size_t bytes = sizeof(double) * (3 * nn + (size_t)m * n) + 256;
    int rc = ensure_buffer(&h->aws, &h->aws_bytes, bytes);
    if (rc) return rc;
    double* M1 = (double*)h->aws;
    double* M2 = M1 + nn;
    double* K = M2 + nn;
    double* T = K + nn;
    int* count = (int*)(T + (size_t)m * n);
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail("adjoint memset", e);
    GemmArgs g;
    g.klo_from_row = g.khi_from_row = false;
    if (gU) {  // M1 = U^T gU
        g.M = n; g.N = n; g.K = m; g.A = U; g.lda = m; g.transA = true; g.B = gU; g.ldb = m;
        g.transB = false; g.C = M1; g.ldc = n;
        if ((rc = launch(g, s))) return rc;
    }
    if (gV) {  // M2 = V^T gV
        g.M = n; g.N = n; g.K = n; g.A = V; g.lda = n; g.transA = true; g.B = gV; g.ldb = n;
        g.transB = false; g.C = M2; g.ldc = n;
        if ((rc = launch(g, s))) return rc;
    }
    int eg = std::max(1, std::min(h->num_sms * 4, (int)((nn + 255) / 256)));
    k_adj_core<<<eg, 256, 0, s>>>(n, S, gU ? M1 : nullptr, gV ? M2 : nullptr, gS, K);
    // T = U K'
    g.M = m; g.N = n; g.K = n; g.A = U; g.lda = m; g.transA = false; g.B = K; g.ldb = n;
    g.transB = false; g.C = T; g.ldc = m;
    if ((rc = launch(g, s))) return rc;
    if (gU) k_adj_addgu<<<h->num_sms * 4, 256, 0, s>>>(m, n, gU, S, T);
    // gA = T V^T
    g.M = m; g.N = n; g.K = n; g.A = T; g.lda = m; g.transA = false; g.B = V; g.ldb = n;
    g.transB = true; g.C = gA; g.ldc = m;
    if ((rc = launch(g, s))) return rc;
    k_adj_flags<<<std::max(1, (n + 255) / 256), 256, 0, s>>>(n, S, gap_tol, count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("adjoint kernels", e);
    h->last_flag_dev = count;
    if (n_flagged) {
        e = cudaMemcpyAsync(n_flagged, count, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail("adjoint flag copy", e);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail("adjoint sync", e);
    }
    return 0;
}

// ------------------------------------------------------------------------------------
// Batched adjoint: one CTA per matrix, the same formula as svd_backward. Small matrices (the
// differentiation workload's 64 x 32): M1 = U^T gU, M2 = V^T gV, K' and T = U K' + gU S^-1
// live in the CTA's slot of a global scratch (L2-resident at these sizes); gA = T V^T is
// written directly.
// ------------------------------------------------------------------------------------

struct BwdPtrs {
    const double* const* U;
    const double* const* S;
    const double* const* V;
    const double* const* gU;  // may be null (every cotangent zero), entries may be null
    const double* const* gS;
    const double* const* gV;
    double* const* gA;
};

__global__ void __launch_bounds__(256) k_adj_batched(BwdPtrs P, const int* dims, double* scratch,
                                                     size_t slot_doubles, double gap_tol, int* flags)
{
    const int b = blockIdx.x;
    const int m = dims[2 * b], n = dims[2 * b + 1];
    const double* U = P.U[b];
    const double* S = P.S[b];
    const double* V = P.V[b];
    const double* gU = P.gU ? P.gU[b] : nullptr;
    const double* gS = P.gS ? P.gS[b] : nullptr;
    const double* gV = P.gV ? P.gV[b] : nullptr;
    double* gA = P.gA[b];
    double* M1 = scratch + slot_doubles * (size_t)b;
    double* M2 = M1 + (size_t)n * n;
    double* K = M2 + (size_t)n * n;
    double* T = K + (size_t)n * n;  // m x n
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t nn = (size_t)n * n;
    // M1 = U^T gU (n x n, K = m), M2 = V^T gV (n x n, K = n)
    for (size_t e = tid; e < nn; e += nt) {
        const int i = (int)(e % n), j = (int)(e / n);
        double a = 0.0, c = 0.0;
        if (gU)
            for (int k = 0; k < m; ++k) a = fma(U[cm(k, i, m)], gU[cm(k, j, m)], a);
        if (gV)
            for (int k = 0; k < n; ++k) c = fma(V[cm(k, i, n)], gV[cm(k, j, n)], c);
        M1[e] = a;
        M2[e] = c;
    }
    __syncthreads();
    // K' (same entries as k_adj_core)
    for (size_t e = tid; e < nn; e += nt) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double si = S[i], sj = S[j];
        const double m1ij = M1[e];
        double v;
        if (i == j) {
            v = (gS ? gS[i] : 0.0) - m1ij / sj;
        } else {
            const double f = 1.0 / (sj * sj - si * si);
            v = f * (m1ij - M1[cm(j, i, n)]) * sj + si * f * (M2[e] - M2[cm(j, i, n)]) - m1ij / sj;
        }
        K[e] = v;
    }
    __syncthreads();
    // T = U K' + gU S^-1
    for (size_t e = tid; e < (size_t)m * n; e += nt) {
        const int i = (int)(e % m), j = (int)(e / m);
        double t = gU ? gU[e] / S[j] : 0.0;
        for (int k = 0; k < n; ++k) t = fma(U[cm(i, k, m)], K[cm(k, j, n)], t);
        T[e] = t;
    }
    __syncthreads();
    // gA = T V^T
    for (size_t e = tid; e < (size_t)m * n; e += nt) {
        const int i = (int)(e % m), j = (int)(e / m);
        double t = 0.0;
        for (int k = 0; k < n; ++k) t = fma(T[cm(i, k, m)], V[cm(j, k, n)], t);
        gA[e] = t;
    }
    // near-degenerate pairs and tiny singular values: counted, never clamped
    int local = 0;
    const double u = 1.1102230246251565e-16;
    for (int i = tid; i < n; i += nt) {
        const double si = S[i];
        if (si <= u * S[0]) ++local;
        for (int j = i + 1; j < n; ++j)
            if (fabs(si - S[j]) <= gap_tol * fmax(si, S[j])) ++local;
    }
    if (local) atomicAdd(&flags[b], local);
}

int svd_backward_batched(mpjsvd_ctx* h, int batch, const int* m, const int* n,
                         const double* const* U, const double* const* S, const double* const* V,
                         const double* const* gU, const double* const* gS, const double* const* gV,
                         double* const* gA, double gap_tol, int* n_flagged)
{
    int mmax = 0, nmax = 0;
    for (int b = 0; b < batch; ++b) {
        mmax = std::max(mmax, m[b]);
        nmax = std::max(nmax, n[b]);
    }
    const size_t slot = 3 * (size_t)nmax * nmax + (size_t)mmax * nmax;
    const size_t dims_bytes = (sizeof(int) * 2 * (size_t)batch + 255) & ~size_t(255);
    int rc = ensure_buffer(&h->aws, &h->aws_bytes, dims_bytes + sizeof(double) * slot * (size_t)batch);
    if (rc) return rc;
    int* dims = (int*)h->aws;
    double* scratch = (double*)((char*)h->aws + dims_bytes);
    // the sizes: host arrays, packed and copied once (from pageable memory the copy has taken
    // the data before cudaMemcpyAsync returns, so the packed array can be freed at once)
    int* packed = new (std::nothrow) int[2 * (size_t)batch];
    if (!packed) return MPJSVD_ERR_NOMEM;
    for (int b = 0; b < batch; ++b) {
        packed[2 * b] = m[b];
        packed[2 * b + 1] = n[b];
    }
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemcpyAsync(dims, packed, sizeof(int) * 2 * (size_t)batch,
                                    cudaMemcpyHostToDevice, s);
    delete[] packed;
    if (e != cudaSuccess) return cuda_fail("batched adjoint: sizes", e);
    e = cudaMemsetAsync(n_flagged, 0, sizeof(int) * (size_t)batch, s);
    if (e != cudaSuccess) return cuda_fail("batched adjoint: flags", e);
    BwdPtrs P{U, S, V, gU, gS, gV, gA};
    k_adj_batched<<<batch, 256, 0, s>>>(P, dims, scratch, slot, gap_tol, n_flagged);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("batched adjoint launch", e);
    h->last_flag_dev = nullptr;
    return 0;
}

}  // namespace mpj
