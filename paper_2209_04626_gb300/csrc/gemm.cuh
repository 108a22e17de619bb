// gemm.cuh -- tiled SIMT GEMM C = op(A) op(B) for the precision switch of Section 3.3
// (B = X^T U_low, Y = X Q, in FP64) and the orthogonality test of Section 3.5
// (Xt^T Xt, in FP32). On this GPU FP64 runs on the SIMT DFMA pipe (the FP64 mma.sync path
// measured slower), so a register-blocked SIMT kernel is the FP64 contraction.
//
// The K range of each output tile can be clipped to the nonzero part of a triangular
// op(A): klo_from_row (op(A)(i, k) = 0 for k < i) and khi_from_row (zero for k > i).
#pragma once

#include "common.cuh"

namespace mpj {

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

struct GemmArgs {
    int M, N, K;
    const void* A;
    int lda;
    bool transA;       // op(A) = A^T (A stored K x M) when true
    const void* B;
    int ldb;
    bool transB = false; // op(B) = B^T (B stored N x K) when true
    void* C;
    int ldc;
    bool klo_from_row; // op(A)(i, k) = 0 for k < i
    bool khi_from_row; // op(A)(i, k) = 0 for k > i
    bool sub = false;  // C <- C - op(A) B (the tensor-core product only)
};

// One 64 x 64 tile of C, 256 threads, 4 x 4 outputs per thread.
template <typename T>
__device__ void gemm_tile(const GemmArgs& g, int m0, int n0)
{
    __shared__ T As[kGemmBK][kGemmBM + 1];
    __shared__ T Bs[kGemmBK][kGemmBN + 1];
    const T* A = (const T*)g.A;
    const T* B = (const T*)g.B;
    T* C = (T*)g.C;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;  // thread owns rows m0+ty*4.., cols n0+tx*4..
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    int klo = g.klo_from_row ? m0 : 0;
    int khi = g.khi_from_row ? min(g.K, m0 + kGemmBM) : g.K;
    klo = (klo / kGemmBK) * kGemmBK;
    for (int k0 = klo; k0 < khi; k0 += kGemmBK) {
        // op(A) tile: rows m0..m0+63, k k0..k0+15  (1024 elements, 4 per thread)
        for (int e = tid; e < kGemmBM * kGemmBK; e += kGemmThreads) {
            int i, kk;
            if (g.transA) { kk = e % kGemmBK; i = e / kGemmBK; }   // A^T: contiguous in k
            else { i = e % kGemmBM; kk = e / kGemmBM; }           // A: contiguous in i
            int gi = m0 + i, gk = k0 + kk;
            T v = T(0);
            if (gi < g.M && gk < g.K && gk < khi)
                v = g.transA ? A[cm(gk, gi, g.lda)] : A[cm(gi, gk, g.lda)];
            As[kk][i] = v;
        }
        for (int e = tid; e < kGemmBK * kGemmBN; e += kGemmThreads) {
            int kk, j;
            if (g.transB) { j = e % kGemmBN; kk = e / kGemmBN; }  // B^T: contiguous in j
            else { kk = e % kGemmBK; j = e / kGemmBK; }          // B: contiguous in k
            int gk = k0 + kk, gj = n0 + j;
            T v = T(0);
            if (gk < g.K && gj < g.N) v = g.transB ? B[cm(gj, gk, g.ldb)] : B[cm(gk, gj, g.ldb)];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmBK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gi = m0 + ty * 4 + i, gj = n0 + tx * 4 + j;
            if (gi < g.M && gj < g.N) C[cm(gi, gj, g.ldc)] = acc[i][j];
        }
}

// ------------------------------------------------------------------------------------------
// Binary64 GEMM C = op(A) B for the switch of Section 3.3 (op(A) triangular, B dense, no
// transposed B): tiles of 128 x 32 outputs, 256 threads, 4 x 4 outputs per thread (rows
// lane + 32 i, columns 4 warp + j), operands staged in shared memory in K chunks of 32. Every
// thread issues 16 DFMA per 8 shared-memory loads, so the FP64 pipe is the limit. Tiles are
// numbered heaviest first (the triangular operand clips each row block's K range).
constexpr int kDgBM = 128, kDgBN = 32, kDgBK = 32, kDgThreads = 256;

static __device__ void dgemm_tile(const GemmArgs& g, int t)
{
    __shared__ double As[kDgBK][kDgBM + 1];
    __shared__ double Bs[kDgBK][kDgBN + 1];
    const double* A = (const double*)g.A;
    const double* B = (const double*)g.B;
    double* C = (double*)g.C;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ntn = (g.N + kDgBN - 1) / kDgBN, ntm = (g.M + kDgBM - 1) / kDgBM;
    int mb = t / ntn;
    if (g.khi_from_row) mb = ntm - 1 - mb;  // the last row blocks have the longest K range
    const int m0 = mb * kDgBM, n0 = (t % ntn) * kDgBN;
    int klo = g.klo_from_row ? m0 : 0;
    const int khi = g.khi_from_row ? min(g.K, m0 + kDgBM) : g.K;
    klo = (klo / kDgBK) * kDgBK;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = klo; k0 < khi; k0 += kDgBK) {
        __syncthreads();  // the previous chunk is no longer read
        for (int e = tid; e < kDgBK * kDgBM; e += kDgThreads) {
            int i, kk;
            if (g.transA) { kk = e % kDgBK; i = e / kDgBK; }  // A^T: contiguous in k
            else { i = e % kDgBM; kk = e / kDgBM; }          // A: contiguous in i
            const int gi = m0 + i, gk = k0 + kk;
            double v = 0.0;
            if (gi < g.M && gk < khi) v = g.transA ? A[cm(gk, gi, g.lda)] : A[cm(gi, gk, g.lda)];
            As[kk][i] = v;
        }
        for (int e = tid; e < kDgBK * kDgBN; e += kDgThreads) {
            const int kk = e % kDgBK, j = e / kDgBK, gk = k0 + kk, gj = n0 + j;
            Bs[kk][j] = (gk < khi && gj < g.N) ? B[cm(gk, gj, g.ldb)] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kDgBK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][lane + 32 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][wid * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gj = n0 + wid * 4 + j;
        if (gj >= g.N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = m0 + lane + 32 * i;
            if (gi < g.M) C[cm(gi, gj, g.ldc)] = acc[i][j];
        }
    }
}

}  // namespace mpj
