// ozaki.cu -- binary64 matrix products on the bf16 tensor cores by error-free operand splitting
// (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications", 2012).
// Used for the GEMMs of the precision switch (Section 3.3) and available as a standalone call.
//
// Splitting. Row i of op(A) is scaled by 2^-e_i with e_i the binary exponent that puts its
// largest |entry| below 1 (frexp), column j of B by 2^-f_j likewise; each scaled entry x is
// cut into kOzS = 8 signed digits of 7 bits: t = 128 x_{s-1}, d_s = rint(t), x_s = t - d_s
// (|d_1| <= 128, |d_s| <= 64 for s >= 2; every step exact in binary64), stored as the bf16
// value d_s 2^-7s (exact). The product is the sum over slice pairs (s, t) with s + t <= 9 of
// the slice products (the pairs dropped weigh below 2^-56 of the row and column maxima).
//
// Exactness. A bf16 x bf16 product is exact in binary32, and a sum of such products with the
// same weight 2^-7(s+t) is exact while its integer part stays below 2^24. The weight classes
// s + t = 2 .. 7 each get their own tensor-memory accumulator and are summed over at most
// kOzKc = 512 values of k (class 2: 512 * 2^14 = 2^23; class w in 3..7: 512 * (2 * 2^13 +
// (w - 3) * 2^12) <= 2^24): exact. The classes 8 and 9 share one accumulator: its terms weigh
// at most 2^(13 - 56), so its binary32 rounding stays below 2^-53 of the row and column
// maxima. After every kOzKc values of k the eight accumulators are added into binary64
// registers (the only binary64 arithmetic: 8 additions per output per 512 k instead of 512
// fused multiply-adds); the result is scaled by 2^(e_i + f_j) at the end.
//
// Kernel. Tiles of 128 x 32 outputs per CTA. The pre-split operands are stored in the order
// the tensor core reads them: for every 128-row (32-row for B) by 16-k block, the 8 slices of
// the block one after another, each in the K-major no-swizzle core-matrix layout. One stage
// (16 k) is then one bulk copy of 32 KiB (A) and one of 8 KiB (B), cp.async.bulk completing
// on an mbarrier; five stages in flight. One thread issues the loads and the 36 tcgen05.mma
// (kind::f16, bf16 operands, M = 128, N = 32, K = 16) of each stage into the accumulator set of
// the current 512-k chunk; two accumulator sets (8 x 32 columns each) alternate, so the four
// epilogue warps fold chunk c while the tensor core works on chunk c + 1.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"
#include "internal.h"
#include "tc.cuh"

namespace mpj {

constexpr int kOzS = 8;              // slices per operand
constexpr int kOzTM = 128;           // output rows per tile (A operand rows)
constexpr int kOzTN = 32;            // output columns per tile (B operand rows)
constexpr int kOzTK = 16;            // k per stage
constexpr int kOzKc = 512;           // k per exact chunk
constexpr int kOzStagesPerChunk = kOzKc / kOzTK;
constexpr int kOzNStage = 5;         // stages in flight
constexpr int kOzNAcc = 8;           // accumulators: classes 2..7 exact, 8..9 together
constexpr int kOzShared = kOzNAcc - 1;
constexpr size_t kOzABlk = (size_t)kOzTM * kOzTK * 2;   // 4096 bytes: one slice of an A block
constexpr size_t kOzBBlk = (size_t)kOzTN * kOzTK * 2;   // 1024
constexpr size_t kOzAStage = kOzS * kOzABlk;            // 32768
constexpr size_t kOzBStage = kOzS * kOzBBlk;            // 8192
constexpr size_t kOzStage = kOzAStage + kOzBStage;      // 40960
constexpr size_t kOzSmem = kOzNStage * kOzStage;        // 204800
constexpr int kOzThreads = 256;
constexpr uint32_t kOzTmemCols = 512;                   // 2 sets x 8 accumulators x 32 columns
constexpr uint32_t kOzIdesc = tc_idesc(kOzTM, kOzTN, kTcFmtBF16);

// Bytes of the split operands (and exponents) for an M x N x K product.
size_t ozaki_ws_bytes(int M, int N, int K)
{
    const size_t MB = (M + kOzTM - 1) / kOzTM, NB = (N + kOzTN - 1) / kOzTN, KB = (K + kOzTK - 1) / kOzTK;
    const size_t a = MB * KB * kOzAStage, b = NB * KB * kOzBStage;
    const size_t ex = (sizeof(unsigned long long) + sizeof(int)) * (MB * kOzTM + NB * kOzTN);
    return ((a + 1023) & ~size_t(1023)) + ((b + 1023) & ~size_t(1023)) + ((ex + 1023) & ~size_t(1023));
}

// ---- row maxima of an operand: element (r, k) at P[r * sr + k * sk], rows R, K columns;
// mx[r] = bits of max_k |P(r, k)| (non-negative doubles order like their bit patterns)
__global__ void k_oz_rowmax(int R, int K, const double* __restrict__ P, long long sr, long long sk,
                            unsigned long long* mx, const int* gate, int want)
{
    if (gate && *(volatile const int*)gate != want) return;
    if (sr == 1) {  // rows contiguous: thread per row, a k range per blockIdx.y
        const int r = blockIdx.x * blockDim.x + threadIdx.x;
        if (r >= R) return;
        const int k0 = blockIdx.y * 256, k1 = min(K, k0 + 256);
        double m = 0.0;
        for (int k = k0; k < k1; ++k) m = fmax(m, fabs(P[r + (long long)k * sk]));
        if (m > 0.0) atomicMax(mx + r, (unsigned long long)__double_as_longlong(m));
    } else {        // k contiguous: warp per row
        const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
        if (blockIdx.y != 0 || warp >= R) return;
        double m = 0.0;
        for (int k = lane; k < K; k += 32) m = fmax(m, fabs(P[(long long)warp * sr + k * sk]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.0) atomicMax(mx + warp, (unsigned long long)__double_as_longlong(m));
    }
}

// ---- the split: thread per (row, 8 consecutive k); TR = 128 (A) or 32 (B) rows per block
template <int TR>
__global__ void k_oz_split(int R, int K, int Rpad, int Kpad, const double* __restrict__ P, long long sr,
                           long long sk, const unsigned long long* mx, int* ex, unsigned char* out,
                           const int* gate, int want)
{
    if (gate && *(volatile const int*)gate != want) return;
    const int KB = Kpad / kOzTK;
    const size_t blk = (size_t)TR * kOzTK * 2;
    const long long total = (long long)Rpad * (Kpad / 8);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e % Rpad), k8 = (int)(e / Rpad);
        int ei = 0;
        double mrow = 0.0;
        if (row < R) {
            mrow = __longlong_as_double((long long)mx[row]);
            if (mrow > 0.0) frexp(mrow, &ei);  // mrow < 2^ei
        }
        if (k8 == 0 && row < R) ex[row] = ei;
        uint32_t w[kOzS][4];  // 8 bf16 per slice, packed in pairs
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double x[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k8 * 8 + 2 * q + h;
                const double a = (row < R && k < K) ? P[(long long)row * sr + (long long)k * sk] : 0.0;
                x[h] = (mrow > 0.0) ? ldexp(a, -ei) : 0.0;
            }
#pragma unroll
            for (int s = 0; s < kOzS; ++s) {
                float f[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const double t = x[h] * 128.0;
                    const double d = rint(t);
                    x[h] = t - d;
                    f[h] = (float)ldexp(d, -7 * (s + 1));  // exact in bf16: |d| <= 128
                }
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[0], f[1]);
                w[s][q] = *reinterpret_cast<const uint32_t*>(&b2);
            }
        }
        const int rb = row / TR, r = row % TR, kb = k8 / 2;
        const size_t off = (size_t)(r / 8) * 256 + (size_t)(k8 & 1) * 128 + (size_t)(r % 8) * 16;
#pragma unroll
        for (int s = 0; s < kOzS; ++s) {
            unsigned char* dst = out + (((size_t)rb * KB + kb) * kOzS + s) * blk + off;
            *reinterpret_cast<uint4*>(dst) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        }
    }
}

// ---- mbarrier helpers for single threads (bounded waits; false = gave up)
__device__ __forceinline__ void mbar_init_n(uint64_t* mbar, unsigned n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}
struct OzArgs {
    int M, N, K, KB;             // KB = padded k / kOzTK
    const unsigned char* Asl;    // split A: [mb][kb][slice] blocks of kOzABlk
    const unsigned char* Bsl;    // split B^T: [nb][kb][slice] blocks of kOzBBlk
    const int* ea;               // row exponents of op(A)
    const int* eb;               // column exponents of B
    double* C;
    int ldc;
    int klo_from_row, khi_from_row;  // clip the k range of a tile by the triangular structure
    int sub;                         // C <- C - op(A) B instead of C <- op(A) B
};

__global__ void __launch_bounds__(kOzThreads, 1) k_oz_gemm(OzArgs g, DevState* st, const int* gate, int want)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[kOzNStage], empty[kOzNStage], accfull[2], accempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    if (gate && *(volatile const int*)gate != want) return;
    if (call_failed(st)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kOzTM, n0 = blockIdx.y * kOzTN;
    // k range in stages (triangular operands: clip by the tile's rows)
    int ks0 = 0, ks1 = g.KB;
    if (g.klo_from_row) ks0 = min(g.KB, m0 / kOzTK);
    if (g.khi_from_row) ks1 = min(g.KB, (m0 + kOzTM + kOzTK - 1) / kOzTK);
    const int nst = max(0, ks1 - ks0);
    const int nch = (nst + kOzStagesPerChunk - 1) / kOzStagesPerChunk;
    if (warp == 0) tmem_alloc(&s_tmem, kOzTmemCols);
    if (tid == 0) {
        for (int i = 0; i < kOzNStage; ++i) { mbar_init_n(&full[i], 1); mbar_init_n(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init_n(&accfull[i], 1); mbar_init_n(&accempty[i], 128); }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (tid == 0 && nst > 0) {
        // ---- loads and MMAs
        const unsigned char* Ab = g.Asl + (size_t)blockIdx.x * g.KB * kOzAStage;
        const unsigned char* Bb = g.Bsl + (size_t)blockIdx.y * g.KB * kOzBStage;
        auto load = [&](int local) {
            const int slot = local % kOzNStage;
            unsigned char* dst = sm + (size_t)slot * kOzStage;
            mbar_expect_tx(&full[slot], (uint32_t)kOzStage);
            bulk_g2s(dst, Ab + (size_t)(ks0 + local) * kOzAStage, (uint32_t)kOzAStage, &full[slot]);
            bulk_g2s(dst + kOzAStage, Bb + (size_t)(ks0 + local) * kOzBStage, (uint32_t)kOzBStage, &full[slot]);
        };
        for (int l = 0; l < min(nst, kOzNStage); ++l) load(l);
        bool ok = true;
        for (int l = 0; l < nst && ok; ++l) {
            const int slot = l % kOzNStage;
            const int c = l / kOzStagesPerChunk, buf = c & 1;
            const bool first = (l % kOzStagesPerChunk) == 0;
            const bool last = (l % kOzStagesPerChunk) == kOzStagesPerChunk - 1 || l == nst - 1;
            if (!mbar_wait1(&full[slot], (uint32_t)((l / kOzNStage) & 1), st)) { ok = false; break; }
            if (first && c >= 2 && !mbar_wait1(&accempty[buf], (uint32_t)(((c >> 1) - 1) & 1), st)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const unsigned char* As = sm + (size_t)slot * kOzStage;
            const unsigned char* Bs = As + kOzAStage;
            const uint32_t accb = tmem + (uint32_t)(buf * kOzNAcc * kOzTN);
            // slice pairs (s, t), s + t <= 7 (0-based): classes 0..5 exact, 6 and 7 together
#pragma unroll
            for (int s = 0; s < kOzS; ++s) {
                const uint64_t ad = tc_desc(As + s * kOzABlk, 128, 256);
#pragma unroll
                for (int t = 0; t < kOzS - s; ++t) {
                    const int cls = s + t < kOzShared ? s + t : kOzShared;
                    const uint64_t bd = tc_desc(Bs + t * kOzBBlk, 128, 256);
                    // the first product of a class in a chunk overwrites its accumulator
                    const bool init = first && s == 0 && t == cls;
                    tc_mma_f16(accb + (uint32_t)(cls * kOzTN), ad, bd, kOzIdesc, init ? 0u : 1u);
                }
            }
            tc_commit(&empty[slot]);
            if (last) tc_commit(&accfull[buf]);
            // refill the slot of stage l - 1 (its MMAs complete while this stage's run)
            if (l >= 1 && l - 1 + kOzNStage < nst) {
                const int ps = (l - 1) % kOzNStage;
                if (!mbar_wait1(&empty[ps], (uint32_t)(((l - 1) / kOzNStage) & 1), st)) { ok = false; break; }
                load(l - 1 + kOzNStage);
            }
        }
        if (!ok) atomicExch(&s_fail, 1);
    } else if (warp >= 4) {
        // ---- epilogue: fold each chunk's four accumulators into binary64
        const int q4 = warp & 3;
        const int r = 32 * q4 + lane;
        double acc[kOzTN];
#pragma unroll
        for (int j = 0; j < kOzTN; ++j) acc[j] = 0.0;
        bool ok = true;
        for (int c = 0; c < nch && ok; ++c) {
            const int buf = c & 1;
            if (!mbar_wait1(&accfull[buf], (uint32_t)((c >> 1) & 1), st)) { ok = false; break; }
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(buf * kOzNAcc * kOzTN);
#pragma unroll
            for (int q = 0; q < kOzTN / 16; ++q) {
#pragma unroll
                for (int cls = 0; cls < kOzNAcc; ++cls) {
                    float v[16];
                    tmem_ld16(base + (uint32_t)(cls * kOzTN + 16 * q), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[16 * q + e] += (double)v[e];
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[buf]);
        }
        if (!ok) atomicExch(&s_fail, 1);
        if (ok) {
            const int row = m0 + r;
            if (row < g.M) {
                const int er = g.ea[row];
#pragma unroll
                for (int j = 0; j < kOzTN; ++j) {
                    const int col = n0 + j;
                    if (col < g.N) {
                        double* cp = g.C + (size_t)col * g.ldc + row;
                        const double pv = ldexp(acc[j], er + g.eb[col]);
                        *cp = g.sub ? *cp - pv : pv;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (s_fail && tid == 0) {
        // a wait gave up: let the MMAs already issued finish (bounded) before the memory goes
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < 20000000ull) {}
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tmem, kOzTmemCols);
}

// C = op(A) B (GemmArgs: transA, no transB) in binary64 via the split products above. ws: at
// least ozaki_ws_bytes(M, N, K) bytes of device memory. gate / want as k_dgemm's.
int ozaki_dgemm(mpjsvd_ctx* h, const GemmArgs& ga, void* ws, const int* gate, int want, DevState* st)
{
    const int M = ga.M, N = ga.N, K = ga.K;
    if (ga.transB) return cuda_fail("ozaki_dgemm: op(B) must be B", cudaErrorInvalidValue);
    const int MB = (M + kOzTM - 1) / kOzTM, NB = (N + kOzTN - 1) / kOzTN, KB = (K + kOzTK - 1) / kOzTK;
    const int Mp = MB * kOzTM, Np = NB * kOzTN, Kp = KB * kOzTK;
    const size_t a = (size_t)MB * KB * kOzAStage, b = (size_t)NB * KB * kOzBStage;
    unsigned char* base = (unsigned char*)ws;
    unsigned char* Asl = base;
    unsigned char* Bsl = base + ((a + 1023) & ~size_t(1023));
    // row maxima of op(A) and of B^T, then their exponents
    unsigned long long* mx = (unsigned long long*)(Bsl + ((b + 1023) & ~size_t(1023)));
    unsigned long long* mxa = mx;
    unsigned long long* mxb = mx + Mp;
    int* exA = (int*)(mx + Mp + Np);
    int* exB = exA + Mp;
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (size_t)(Mp + Np), s);
    if (e != cudaSuccess) return cuda_fail("ozaki: memset", e);
    // op(A)(i, k): A[k * lda + i] (A) or A[i * lda + k] (A^T); B(k, j): B[j * ldb + k]
    const long long sra = ga.transA ? ga.lda : 1, ska = ga.transA ? 1 : ga.lda;
    const long long srb = ga.ldb, skb = 1;
    {
        dim3 gr(ga.transA ? (M * 32 + 255) / 256 : (M + 255) / 256, ga.transA ? 1 : (K + 255) / 256);
        k_oz_rowmax<<<gr, 256, 0, s>>>(M, K, (const double*)ga.A, sra, ska, mxa, gate, want);
        dim3 gb((N * 32 + 255) / 256, 1);
        k_oz_rowmax<<<gb, 256, 0, s>>>(N, K, (const double*)ga.B, srb, skb, mxb, gate, want);
    }
    const int gsa = std::min(h->num_sms * 8, (int)(((long long)Mp * (Kp / 8) + 255) / 256));
    const int gsb = std::min(h->num_sms * 8, (int)(((long long)Np * (Kp / 8) + 255) / 256));
    k_oz_split<kOzTM><<<std::max(1, gsa), 256, 0, s>>>(M, K, Mp, Kp, (const double*)ga.A, sra, ska, mxa, exA, Asl,
                                                       gate, want);
    k_oz_split<kOzTN><<<std::max(1, gsb), 256, 0, s>>>(N, K, Np, Kp, (const double*)ga.B, srb, skb, mxb, exB, Bsl,
                                                       gate, want);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("ozaki: split kernels", e);
    e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return cuda_fail("ozaki: smem attribute", e);
    OzArgs g;
    g.M = M; g.N = N; g.K = K; g.KB = KB;
    g.Asl = Asl; g.Bsl = Bsl; g.ea = exA; g.eb = exB;
    g.C = (double*)ga.C; g.ldc = ga.ldc;
    g.klo_from_row = ga.klo_from_row ? 1 : 0;
    g.sub = ga.sub ? 1 : 0;
    g.khi_from_row = ga.khi_from_row ? 1 : 0;
    k_oz_gemm<<<dim3(MB, NB), kOzThreads, kOzSmem, s>>>(g, st, gate, want);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("ozaki: gemm launch", e);
    h->launch_count += 5;
    return 0;
}

int dgemm_tc_call(mpjsvd_ctx* h, int M, int N, int K, const double* A, int lda, int transA, const double* B,
                  int ldb, double* C, int ldc)
{
    h->launch_count = 0;
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, ozaki_ws_bytes(M, N, K));
    if (rc) return rc;
    if ((rc = state_reset(h, h->dstate))) return rc;
    GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.transA = transA != 0;
    g.B = B; g.ldb = ldb; g.transB = false;
    g.C = C; g.ldc = ldc;
    g.klo_from_row = g.khi_from_row = false;
    g.sub = false;
    return ozaki_dgemm(h, g, h->ws, nullptr, 0, (DevState*)h->dstate);
}

}  // namespace mpj

extern "C" int mpjsvd_dgemm_tc(mpjsvd_handle h, int M, int N, int K, const double* A, int lda, int transA,
                               const double* B, int ldb, double* C, int ldc)
{
    if (!h) return -1;
    if (M < 1) return -2;
    if (N < 1) return -3;
    if (K < 1) return -4;
    if (!A) return -5;
    if (lda < (transA ? K : M)) return -6;
    if (!B) return -8;
    if (ldb < K) return -9;
    if (!C) return -10;
    if (ldc < M) return -11;
    return mpj::dgemm_tc_call(h, M, N, K, A, lda, transA, B, ldb, C, ldc);
}
