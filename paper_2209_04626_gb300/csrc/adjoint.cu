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
    if (n_flagged) {
        e = cudaMemcpyAsync(n_flagged, count, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail("adjoint flag copy", e);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail("adjoint sync", e);
    }
    return 0;
}

}  // namespace mpj
