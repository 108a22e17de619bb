// qrcp_low.cu -- the binary32 pivot search of the mixed-precision RRQR (Alg. 5, step 2).
//
// lower(A) is A scaled by the power of two that brings max |a_ij| into [1, 2) and rounded to
// binary32; a Businger-Golub QR with column pivoting of lower(A) then yields the permutation P
// (the binary32 R is discarded; the binary64 QR of A P follows in qr_blocked.cu). Same steps
// as the binary64 kernel: the first maximum of the downdated norms wins, the norms are
// downdated by the new row entry and recomputed when the downdate keeps less than half of
// the binary32 digits. Every norm is taken on power-of-two scaled entries, so the squares of
// small columns do not underflow (the convention of single-precision LAPACK norms).
//
// Shared-memory kernel: one cooperative launch; CTA r owns the columns r, r + G, ... resident
// in shared memory. Each step publishes every CTA's candidate (norm, column) and the
// candidate's rows in one slot, then one grid barrier: every CTA then reads the winner's
// column from its slot. The register-resident kernel below replaces the barrier by per-CTA
// step records.
#include "common.cuh"
#include "internal.h"
#include "qr.cuh"

namespace mpj {

constexpr int kLowThreads = 256;
constexpr int kLowThreadsGlobal = 512;  // columns in global memory: more loads in flight
constexpr int kLowBatch = 4;
constexpr int kLowUnroll = 4;  // rows per thread whose loads are issued together

__device__ __forceinline__ float block_max_f(float v, float* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float r = (lane < nw) ? red[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

// |x(lo:m)| of a shared-memory column without underflow or overflow of the squares.
__device__ float norm_scaled(const float* x, int lo, int m, float* red)
{
    float a = 0.0f;
    for (int i = lo + threadIdx.x; i < m; i += blockDim.x) a = fmaxf(a, fabsf(x[i]));
    a = block_max_f(a, red);
    if (a == 0.0f) return 0.0f;
    const int eb = (__float_as_int(a) >> 23) & 0xff;
    const float sc = __int_as_float((254 - eb) << 23);  // a * sc in [1, 2)
    float s = 0.0f;
    for (int i = lo + threadIdx.x; i < m; i += blockDim.x) {
        const float y = x[i] * sc;
        s = fmaf(y, y, s);
    }
    s = block_sum(s, red);
    return sqrtf(s) / sc;
}

__host__ __device__ inline size_t qrcp_low_smem_bytes(int m, int n, int gsize, bool global_cols = false)
{
    const int own = (n + gsize - 1) / gsize;
    return sizeof(float) * ((global_cols ? 0 : (size_t)own * m) + m + 3 * (size_t)own) + sizeof(int) * own;
}

// GLOBAL = false: the owned columns in shared memory; GLOBAL = true (columns too long for it):
// in global memory, gcols + rank * own_max * m (L2 and HBM traffic instead of shared memory).
template <bool GLOBAL>
__global__ void __launch_bounds__(GLOBAL ? kLowThreadsGlobal : kLowThreads)
    k_qrcp_low(int m, int n, const double* __restrict__ A, int lda, int* perm, float* bcast,
               DevState* st, float* gcols)
{
    extern __shared__ float lsm[];
    __shared__ float red[kLowBatch * 33];
    __shared__ double s_amax;
    __shared__ int s_piv, s_src, s_recompute;
    if (call_failed(st)) return;
    const Group g{(int)blockIdx.x, (int)gridDim.x, st};
    const int own = (n - g.rank + g.size - 1) / g.size;
    const int own_max = (n + g.size - 1) / g.size;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    float* C = GLOBAL ? gcols + (size_t)g.rank * own_max * m : lsm;  // own x m
    float* vs = GLOBAL ? lsm : C + (size_t)own * m;                   // m: the step's column, then its reflector
    float* vn1 = vs + m;
    float* vn2 = vn1 + own;
    float* rowj = vn2 + own;
    int* act = (int*)(rowj + own);
    const float tol3z = 2.44140625e-04f;  // sqrt(2^-24)

    // ---- lower(A): global max |a_ij| (non-negative doubles order like their bit patterns)
    double am = 0.0;
    for (int t = 0; t < own; ++t) {
        const double* src = A + cm(0, g.rank + t * g.size, lda);
        for (int i = tid; i < m; i += nthr) am = fmax(am, fabs(src[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    if (lane == 0) atomicMax(&st->amax_bits, (unsigned long long)__double_as_longlong(am));
    // slot of (parity, CTA r): m row words, then alpha, |tail|, |column|
    unsigned long long* const llb = reinterpret_cast<unsigned long long*>(bcast);
    const size_t slot_words = (size_t)m + 4;
    if (tid < 2) st->cand_rec[tid * kQrSlotStride + g.rank] = 0ull;  // no step tag yet
    for (size_t i = tid; i < 2 * slot_words; i += blockDim.x)
        llb[((i / slot_words) * g.size + g.rank) * slot_words + i % slot_words] = 0ull;
    if (!g.sync()) return;
    if (tid == 0) s_amax = __longlong_as_double((long long)__ldcg(&st->amax_bits));
    __syncthreads();
    const double amax = s_amax;
    const int eb = (__double2hiint(amax) >> 20) & 0x7ff;
    const double scale = (amax > 0.0) ? __hiloint2double((2046 - min(max(eb, 1), 2045)) << 20, 0) : 1.0;
    for (int t = 0; t < own; ++t) {
        const double* src = A + cm(0, g.rank + t * g.size, lda);
        float* dst = C + (size_t)t * m;
        for (int i = tid; i < m; i += nthr) dst[i] = (float)(src[i] * scale);
    }
    for (int t = tid; t < own; t += nthr) act[t] = 1;
    __syncthreads();
    for (int t = 0; t < own; ++t) {
        const float v = norm_scaled(C + (size_t)t * m, 0, m, red);
        if (tid == 0) { vn1[t] = v; vn2[t] = v; }
    }
    __syncthreads();

    const int k = min(m, n);
    for (int j = 0; j < k; ++j) {
        // ---- candidate of this CTA (first maximum in column order), published with its rows
        if (tid < 32) {
            int best = -1;
            float bv = 0.0f;
            for (int t = lane; t < own; t += 32) {
                if (!act[t]) continue;
                if (best < 0 || vn1[t] > bv) { bv = vn1[t]; best = t; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int ob = __shfl_xor_sync(0xffffffffu, best, o);
                if (ob >= 0 && (best < 0 || ov > bv || (ov == bv && ob < best))) { bv = ov; best = ob; }
            }
            if (lane == 0) {
                put_candidate(st, j & 1, g.rank, (double)bv, best >= 0 ? g.rank + best * g.size : -1);
                s_src = best;
            }
        }
        __syncthreads();
        if (s_src >= 0) {
            const float* c = C + (size_t)s_src * m;
            float* slot = bcast + ((size_t)(j & 1) * g.size + g.rank) * m;
            for (int i = j + tid; i < m; i += nthr) slot[i] = c[i];
        }
        if (!g.sync()) return;
        if (tid < 32) {
            const int best = pivot_argmax(st, j & 1, g.size, lane);
            if (lane == 0) s_piv = best;
        }
        __syncthreads();
        const int p = s_piv;
        if (p < 0 || p >= n) {
            if (tid == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
            return;
        }
        const float* src = bcast + ((size_t)(j & 1) * g.size + (p % g.size)) * m;
        for (int i = j + tid; i < m; i += nthr) vs[i] = __ldcg(src + i);
        __syncthreads();

        // ---- reflector of the pivot column (the convention of the binary64 kernels)
        float tj = 0.0f;
        const float tailn = norm_scaled(vs, j + 1, m, red);
        if (tailn != 0.0f) {
            const float alpha = vs[j];
            const float nrm = norm_scaled(vs, j, m, red);
            const float beta = (alpha >= 0.0f) ? -nrm : nrm;
            tj = (beta - alpha) / beta;
            const float den = alpha - beta;
            __syncthreads();
            for (int i = j + 1 + tid; i < m; i += nthr) vs[i] = vs[i] / den;
        }
        __syncthreads();
        const bool mine = (p % g.size == g.rank);
        const int tp = (p - g.rank) / g.size;

        // ---- apply it to the other active columns, downdate their norms
        int t = 0;
        while (true) {
            float* cols[kLowBatch];
            int tix[kLowBatch];
            int nb = 0;
            for (; t < own && nb < kLowBatch; ++t) {
                if (act[t] && !(mine && t == tp)) {
                    tix[nb] = t;
                    cols[nb] = C + (size_t)t * m;
                    ++nb;
                }
            }
            if (nb == 0) break;
            for (int b = nb; b < kLowBatch; ++b) { cols[b] = cols[0]; tix[b] = tix[0]; }
            if (tj != 0.0f) {
                float acc[kLowBatch], w[kLowBatch];
#pragma unroll
                for (int b = 0; b < kLowBatch; ++b) acc[b] = 0.0f;
                // kLowUnroll rows at a time: their loads are in flight together; each thread
                // still sums its rows in increasing order
                int i = j + 1 + tid;
                if (GLOBAL) {
                    for (; i + (kLowUnroll - 1) * nthr < m; i += kLowUnroll * nthr) {
                        float vu[kLowUnroll], cu[kLowUnroll][kLowBatch];
#pragma unroll
                        for (int u = 0; u < kLowUnroll; ++u) {
                            vu[u] = vs[i + u * nthr];
#pragma unroll
                            for (int b = 0; b < kLowBatch; ++b) cu[u][b] = cols[b][i + u * nthr];
                        }
#pragma unroll
                        for (int u = 0; u < kLowUnroll; ++u)
#pragma unroll
                            for (int b = 0; b < kLowBatch; ++b) acc[b] = fmaf(vu[u], cu[u][b], acc[b]);
                    }
                }
                for (; i < m; i += nthr) {
                    const float vi = vs[i];
#pragma unroll
                    for (int b = 0; b < kLowBatch; ++b) acc[b] = fmaf(vi, cols[b][i], acc[b]);
                }
                block_sum_multi<kLowBatch>(acc, red, w);
#pragma unroll
                for (int b = 0; b < kLowBatch; ++b) w[b] = tj * (cols[b][j] + w[b]);
                __syncthreads();  // every thread has read c_j before it changes
                if (tid == 0)
                    for (int b = 0; b < nb; ++b) cols[b][j] -= w[b];
                i = j + 1 + tid;
                if (GLOBAL) {
                    for (; i + (kLowUnroll - 1) * nthr < m; i += kLowUnroll * nthr) {
                        float vu[kLowUnroll], cu[kLowUnroll][kLowBatch];
#pragma unroll
                        for (int u = 0; u < kLowUnroll; ++u) {
                            vu[u] = vs[i + u * nthr];
#pragma unroll
                            for (int b = 0; b < kLowBatch; ++b) cu[u][b] = cols[b][i + u * nthr];
                        }
#pragma unroll
                        for (int u = 0; u < kLowUnroll; ++u)
#pragma unroll
                            for (int b = 0; b < kLowBatch; ++b)
                                if (b < nb) cols[b][i + u * nthr] = fmaf(-w[b], vu[u], cu[u][b]);
                    }
                }
                for (; i < m; i += nthr) {
                    const float vi = vs[i];
#pragma unroll
                    for (int b = 0; b < kLowBatch; ++b)
                        if (b < nb) cols[b][i] = fmaf(-w[b], vi, cols[b][i]);
                }
                __syncthreads();
            }
            if (tid == 0) {
                s_recompute = 0;
                for (int b = 0; b < nb; ++b) rowj[tix[b]] = cols[b][j];
            }
            __syncthreads();
            if (tid < nb) {
                const int tt = tix[tid];
                const float v1 = vn1[tt];
                if (v1 != 0.0f) {
                    const float r = fabsf(rowj[tt]) / v1;
                    float q = 1.0f - r * r;
                    q = q < 0.0f ? 0.0f : q;
                    const float ratio = v1 / vn2[tt];
                    if (q * ratio * ratio <= tol3z) atomicOr(&s_recompute, 1 << tid);
                    else vn1[tt] = v1 * sqrtf(q);
                }
            }
            __syncthreads();
            const int mask = s_recompute;
            for (int b = 0; b < nb; ++b) {
                if (!(mask & (1 << b))) continue;
                const float v = norm_scaled(cols[b], j + 1, m, red);
                if (tid == 0) { vn1[tix[b]] = v; vn2[tix[b]] = v; }
            }
            __syncthreads();
        }
        if (mine && tid == 0) {
            act[tp] = 0;
            perm[j] = p;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Register-resident variant: warp w of CTA b owns column c = 8 b + w, its rows lane + 32 k
// (k < KR) in registers, so applying a reflector is warp-local (no CTA barrier).
//
// Exchange without barriers or fences. Every word a CTA publishes in step j is 64 bits wide
// and carries the tag j + 1 in its upper half, so a reader that sees the tag sees the value
// (an aligned 8-byte access is single-copy atomic), whatever order the writer's stores land
// in. In step j the CTA's candidate warp writes its rows j.. and the reflector's scalars
// (alpha, |tail|, |column|, computed exactly from its registers) to its slot, then the record
// {tag, column, norm}. Warp 0 of every CTA polls the G records of step j until all carry the
// tag, takes the argmax; then each thread reads its rows of the winner's slot, re-reading a
// word until its tag is j + 1. A CTA cannot publish step j + 2 (same slot parity as j) before
// every CTA has published step j + 1, i.e. has finished reading step j, so two slot sets
// suffice; each CTA clears its slots and records before the one grid barrier at the start,
// so words of an earlier call never carry a tag of this one. Same pivot rule, downdating and
// norms as the kernel above.
constexpr int kRegWarps = 8;

// record of CTA candidate (column c, norm v >= 0) for step j; none: c = 0xffff
__device__ __forceinline__ unsigned long long cand_record(int j, int c, float v)
{
    return ((unsigned long long)((j + 1) & 0xffff) << 48) | ((unsigned long long)(c & 0xffff) << 32) |
           (unsigned long long)__float_as_uint(v);
}
// tagged word of step j: {value, j + 1}
__device__ __forceinline__ unsigned long long tagged(float v, int j)
{
    return ((unsigned long long)(unsigned)(j + 1) << 32) | (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Phase probes of the register-resident kernel: empty here; a profiling build may define them.
#ifndef MPJ_QRCP_PROBE_BEGIN
#define MPJ_QRCP_PROBE_BEGIN
#define MPJ_QRCP_PROBE(i)
#define MPJ_QRCP_PROBE_END
#endif
#ifndef MPJ_QRCP_MARK
#define MPJ_QRCP_MARK(k, j, extra) {}
#endif

template <int KR>
__device__ __forceinline__ float reg_norm_scaled(const float (&x)[KR], int lo, int lane)
{
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (lane + 32 * k >= lo) a = fmaxf(a, fabsf(x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (a == 0.0f) return 0.0f;
    const int eb = (__float_as_int(a) >> 23) & 0xff;
    const float sc = __int_as_float((254 - eb) << 23);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (lane + 32 * k >= lo) {
            const float y = x[k] * sc;
            s = fmaf(y, y, s);
        }
    s = warp_sum(s);
    return sqrtf(s) / sc;
}

// Reflector scalars of the candidate column in one pass over the registers: |x(j+1:m)| on
// entries scaled by the power of two of its own maximum, and |x(j:m)| from it and alpha =
// x(j) (both on power-of-two scaled values, so no square underflows or overflows). Four
// independent chains per lane; the maximum is one redux (non-negative binary32 values order
// like their bit patterns).
template <int KR>
__device__ __forceinline__ void reg_cand_scalars(const float (&x)[KR], int j, int lane, float alpha, float& tailn,
                                                 float& nrm)
{
    unsigned mb[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (lane + 32 * k > j) mb[k & 3] = max(mb[k & 3], __float_as_uint(fabsf(x[k])));
    const unsigned mt = __reduce_max_sync(0xffffffffu, max(max(mb[0], mb[1]), max(mb[2], mb[3])));
    const float aa = fabsf(alpha);
    if (mt == 0u) {
        tailn = 0.0f;
        nrm = aa;
        return;
    }
    const int et = (int)(mt >> 23) & 0xff;
    const float sct = __int_as_float((254 - et) << 23);  // max |tail| * sct in [1, 2)
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (lane + 32 * k > j) {
            const float y = x[k] * sct;
            s[k & 3] = fmaf(y, y, s[k & 3]);
        }
    const float st = warp_sum((s[0] + s[1]) + (s[2] + s[3]));
    tailn = sqrtf(st) / sct;
    const int ea = (int)(__float_as_uint(aa) >> 23) & 0xff;
    if (ea <= et) {
        const float ya = alpha * sct;
        nrm = sqrtf(fmaf(ya, ya, st)) / sct;
    } else {
        // |alpha| is the larger: scale by its power of two; the tail's sum moves by an exact
        // power of two (its square, 2^(2 (et - ea)))
        const float sca = __int_as_float((254 - ea) << 23);
        const float ya = alpha * sca;
        const int d = et - ea;  // < 0
        const float r2 = (2 * d >= -149) ? ldexpf(1.0f, 2 * d) : 0.0f;
        nrm = sqrtf(fmaf(st, r2, ya * ya)) / sca;
    }
}

// the entry of row r (all lanes receive it)
template <int KR>
__device__ __forceinline__ float reg_row(const float (&x)[KR], int r, int lane)
{
    float v = 0.0f;
    const int kr = r >> 5;
#pragma unroll
    for (int k = 0; k < KR; ++k)
        if (k == kr) v = x[k];
    return __shfl_sync(0xffffffffu, v, r & 31);
}

template <int KR>
__global__ void __launch_bounds__(kRegWarps * 32)
    k_qrcp_low_reg(int m, int n, const double* __restrict__ A, int lda, int* perm, float* bcast,
                   DevState* st)
{
    __shared__ float vs[32 * KR];
    __shared__ float wvn[kRegWarps];
    __shared__ int wcol[kRegWarps];
    __shared__ double s_amax;
    __shared__ int s_piv;
    __shared__ float s_scal[3];
    if (call_failed(st)) return;
    const Group g{(int)blockIdx.x, (int)gridDim.x, st};
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int c = blockIdx.x * kRegWarps + wid;  // this warp's column
    bool act = c < n;
    const float tol3z = 2.44140625e-04f;  // sqrt(2^-24)

    // ---- lower(A): global max |a_ij|, then the scaled binary32 column in registers
    double am = 0.0;
    if (act)
        for (int i = lane; i < m; i += 32) am = fmax(am, fabs(A[cm(i, c, lda)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    if (lane == 0) atomicMax(&st->amax_bits, (unsigned long long)__double_as_longlong(am));
    // slot of (parity, CTA r): m row words, then alpha, |tail|, |column|
    unsigned long long* const llb = reinterpret_cast<unsigned long long*>(bcast);
    const size_t slot_words = (size_t)m + 4;
    if (tid < 2) st->cand_rec[tid * kQrSlotStride + g.rank] = 0ull;  // no step tag yet
    for (size_t i = tid; i < 2 * slot_words; i += blockDim.x)
        llb[((i / slot_words) * g.size + g.rank) * slot_words + i % slot_words] = 0ull;
    if (!g.sync()) return;
    if (tid == 0) s_amax = __longlong_as_double((long long)__ldcg(&st->amax_bits));
    __syncthreads();
    const double amax = s_amax;
    const int eb = (__double2hiint(amax) >> 20) & 0x7ff;
    const double scale = (amax > 0.0) ? __hiloint2double((2046 - min(max(eb, 1), 2045)) << 20, 0) : 1.0;
    float x[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int i = lane + 32 * k;
        x[k] = (act && i < m) ? (float)(A[cm(i, c, lda)] * scale) : 0.0f;
    }
    float vn1 = act ? reg_norm_scaled<KR>(x, 0, lane) : 0.0f;
    float vn2 = vn1;
    MPJ_QRCP_PROBE_BEGIN

    const int kmax = min(m, n);
    if (lane == 0) {
        wvn[wid] = act ? vn1 : -1.0f;
        wcol[wid] = act ? c : -1;
    }
    __syncthreads();
    for (int j = 0; j < kmax; ++j) {
        const int par = j & 1;
        // ---- this CTA's candidate (first maximum in column order) publishes itself
        MPJ_QRCP_PROBE(0)
        if (tid == 0) MPJ_QRCP_MARK(0, j, 0)
        int cw = -1;
        float cv = 0.0f;
#pragma unroll
        for (int w = 0; w < kRegWarps; ++w)
            if (wcol[w] >= 0 && (cw < 0 || wvn[w] > cv)) { cv = wvn[w]; cw = w; }
        if (wid == cw) {
            // rows, then scalars, then the record: a reader that sees the record rarely has
            // to wait for the rest
            unsigned long long* slot = llb + ((size_t)par * g.size + g.rank) * slot_words;
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int i = lane + 32 * k;
                if (i > j && i < m) st_relaxed_u64(slot + i, tagged(x[k], j));
            }
            const float alpha = reg_row<KR>(x, j, lane);
            float tailn, nrm;
            reg_cand_scalars<KR>(x, j, lane, alpha, tailn, nrm);
            if (lane < 3) st_relaxed_u64(slot + m + lane, tagged(lane == 0 ? alpha : (lane == 1 ? tailn : nrm), j));
            if (lane == 0) st_relaxed_u64(&st->cand_rec[par * kQrSlotStride + g.rank], cand_record(j, c, cv));
            if (lane == 0) MPJ_QRCP_MARK(1, j, 0)
        } else if (cw < 0 && tid == 0) {
            st_relaxed_u64(&st->cand_rec[par * kQrSlotStride + g.rank], cand_record(j, 0xffff, 0.0f));
        }
        MPJ_QRCP_PROBE(1)
        if (wid == 0) {
            // wait for the G records of step j (lane l holds records l, l + 32, ...)
            constexpr int K = kQrSlotStride / 32;
            const unsigned want = (unsigned)((j + 1) & 0xffff);
            unsigned long long rec[K];
#pragma unroll
            for (int q = 0; q < K; ++q) rec[q] = 0ull;
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            bool ready = false;
            while (true) {
                bool mine = true;
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    const int r = lane + 32 * q;
                    if (r < g.size && (unsigned)(rec[q] >> 48) != want)
                        rec[q] = ld_relaxed_u64(&st->cand_rec[par * kQrSlotStride + r]);
                }
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    const int r = lane + 32 * q;
                    if (r < g.size && (unsigned)(rec[q] >> 48) != want) mine = false;
                }
                if (__all_sync(0xffffffffu, mine)) {
                    ready = true;
                    break;
                }
                if ((++spins & 255u) == 0) {
                    if (*(volatile int*)&st->status & MPJSVD_STATUS_TIMEOUT) break;
                    if (globaltimer_ns() - t0 > spin_limit_ns(st)) {
                        if (lane == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                        break;
                    }
                }
            }
            if (lane == 0) MPJ_QRCP_MARK(2, j, spins)
            // argmax: largest norm, then the lowest column index (key order)
            unsigned long long best = 0ull;
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int r = lane + 32 * q;
                const unsigned cidx = (unsigned)(rec[q] >> 32) & 0xffffu;
                if (r < g.size && cidx != 0xffffu) {
                    const unsigned long long key = ((rec[q] & 0xffffffffull) << 32) | 0x80000000ull |
                                                   (unsigned long long)(0xffffu - cidx);
                    best = key > best ? key : best;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                best = ob > best ? ob : best;
            }
            if (lane == 0) s_piv = (ready && best != 0ull) ? (int)(0xffffu - (unsigned)(best & 0xffffu)) : -1;
        }
        __syncthreads();
        const int p = s_piv;
        if (p < 0 || p >= n) {
            if (tid == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
            return;
        }
        MPJ_QRCP_PROBE(2)
        MPJ_QRCP_PROBE(3)
        const int pb = p / kRegWarps;  // the winner's CTA
        const unsigned long long* src = llb + ((size_t)par * g.size + pb) * slot_words;
        constexpr int kFill = (32 * KR + kRegWarps * 32 - 1) / (kRegWarps * 32);
        const unsigned want = (unsigned)(j + 1);
        unsigned long long wv[kFill + 1];  // this thread's rows of the winner (+ one scalar for tid < 3)
#pragma unroll
        for (int q = 0; q < kFill + 1; ++q) wv[q] = 0ull;
        const bool has_sc = tid < 3;  // threads 0..2 fetch alpha, |tail|, |column| for the CTA
        bool bad = false;
        {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (true) {
                // issue every pending load, then check (no load waits on another)
#pragma unroll
                for (int q = 0; q < kFill; ++q) {
                    const int i = j + 1 + tid + q * kRegWarps * 32;
                    if (i < m && (unsigned)(wv[q] >> 32) != want) wv[q] = ld_relaxed_u64(src + i);
                }
                if (has_sc && (unsigned)(wv[kFill] >> 32) != want) wv[kFill] = ld_relaxed_u64(src + m + tid);
                bool ok = !(has_sc && (unsigned)(wv[kFill] >> 32) != want);
#pragma unroll
                for (int q = 0; q < kFill; ++q) {
                    const int i = j + 1 + tid + q * kRegWarps * 32;
                    if (i < m && (unsigned)(wv[q] >> 32) != want) ok = false;
                }
                if (ok) break;
                if ((++spins & 255u) == 0) {
                    if ((*(volatile int*)&st->status & MPJSVD_STATUS_TIMEOUT) ||
                        globaltimer_ns() - t0 > spin_limit_ns(st)) {
                        bad = true;
                        break;
                    }
                }
            }
        }
        if (has_sc) s_scal[tid] = __uint_as_float((unsigned)wv[kFill]);
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
            return;
        }
        const float alpha = s_scal[0], tailn = s_scal[1], nrm = s_scal[2];
        float tj = 0.0f, den = 1.0f;
        if (tailn != 0.0f) {
            const float beta = (alpha >= 0.0f) ? -nrm : nrm;
            tj = (beta - alpha) / beta;
            den = alpha - beta;
        }
        if (tj != 0.0f) {
#pragma unroll
            for (int q = 0; q < kFill; ++q) {
                const int i = j + 1 + tid + q * kRegWarps * 32;
                if (i < m) vs[i] = __uint_as_float((unsigned)wv[q]) / den;
            }
        }
        __syncthreads();
        MPJ_QRCP_PROBE(4)
        if (tid == 0) MPJ_QRCP_MARK(4, j, 0)

        // ---- apply H_j to this warp's column, downdate its norm
        if (act && c == p) {
            act = false;
            if (lane == 0) perm[j] = p;
        } else if (act) {
            if (tj != 0.0f) {
                float dp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    const int i = lane + 32 * k;
                    if (i > j && i < m) dp[k & 3] = fmaf(vs[i], x[k], dp[k & 3]);
                }
                const float d = warp_sum((dp[0] + dp[1]) + (dp[2] + dp[3]));
                const float w = tj * (reg_row<KR>(x, j, lane) + d);
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    const int i = lane + 32 * k;
                    if (i > j && i < m) x[k] = fmaf(-w, vs[i], x[k]);
                    else if (i == j) x[k] -= w;
                }
            }
            if (vn1 != 0.0f) {
                const float r = fabsf(reg_row<KR>(x, j, lane)) / vn1;
                float q = 1.0f - r * r;
                q = q < 0.0f ? 0.0f : q;
                const float ratio = vn1 / vn2;
                if (q * ratio * ratio <= tol3z) {
                    vn1 = reg_norm_scaled<KR>(x, j + 1, lane);
                    vn2 = vn1;
                } else {
                    vn1 = vn1 * sqrtf(q);
                }
            }
        }
        MPJ_QRCP_PROBE(5)
        if (tid == 0) MPJ_QRCP_MARK(5, j, 0)
        if (lane == 0) {
            wvn[wid] = act ? vn1 : -1.0f;
            wcol[wid] = act ? c : -1;
        }
        // the next step reads wvn / wcol; vs is rewritten only after its pivot barrier
        __syncthreads();
        MPJ_QRCP_PROBE(6)
    }
    MPJ_QRCP_PROBE_END
}

template <int KR>
static int launch_reg(mpjsvd_ctx* h, int m, int n, const double* A, int lda, int* perm, float* bcast,
                      DevState* st)
{
    const int grid = (n + kRegWarps - 1) / kRegWarps;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_qrcp_low_reg<KR>, kRegWarps * 32, 0);
    if (e != cudaSuccess) return cuda_fail("qrcp_low_reg occupancy", e);
    if (grid > kQrSlotStride || grid > occ * h->num_sms) return 1;
    void* args[] = {&m, &n, &A, &lda, &perm, &bcast, &st};
    e = cudaLaunchCooperativeKernel((void*)k_qrcp_low_reg<KR>, grid, kRegWarps * 32, args, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail("qrcp_low_reg launch", e);
    ++h->launch_count;
    return 0;
}

// Bytes of the broadcast region that the global-column variant needs (slots, then columns).
size_t qrcp_low_bcast_bytes(int m, int n, int sms)
{
    const int grid = std::max(1, std::min(n, std::min(sms, kQrSlotStride)));
    const size_t slots = ((sizeof(unsigned long long) * 2 * (size_t)grid * ((size_t)m + 4)) + 255) & ~size_t(255);
    const int own_max = (n + grid - 1) / grid;
    return slots + sizeof(float) * (size_t)grid * own_max * m;
}

// Launch the binary32 pivot search: register-resident when a column fits a warp's registers
// and there is a warp per column, else columns resident in shared memory, else (long columns)
// columns in global memory after the broadcast slots in bcast (bcast_bytes in all); returns 1
// (nothing launched) when none fits, so the caller takes the binary64 QRCP instead.
int launch_qrcp_low(mpjsvd_ctx* h, int m, int n, const double* A, int lda, int* perm, float* bcast,
                    size_t bcast_bytes, DevState* st)
{
    int rc = 1;
    if (m <= 256) rc = launch_reg<8>(h, m, n, A, lda, perm, bcast, st);
    else if (m <= 512) rc = launch_reg<16>(h, m, n, A, lda, perm, bcast, st);
    else if (m <= 1024) rc = launch_reg<32>(h, m, n, A, lda, perm, bcast, st);
    else if (m <= 2048) rc = launch_reg<64>(h, m, n, A, lda, perm, bcast, st);  // 216 registers
    if (rc <= 0) return rc;
    const int grid = std::max(1, std::min(n, std::min(h->num_sms, kQrSlotStride)));
    bool global_cols = false;
    size_t smem = qrcp_low_smem_bytes(m, n, grid);
    float* gcols = nullptr;
    if (smem > 200 * 1024) {
        // slots: 2 parities x grid CTAs x (m + 4) words of 8 bytes; then own_max x m floats per CTA
        const size_t slots = ((sizeof(unsigned long long) * 2 * (size_t)grid * ((size_t)m + 4)) + 255) & ~size_t(255);
        const int own_max = (n + grid - 1) / grid;
        const size_t cols = sizeof(float) * (size_t)grid * own_max * m;
        smem = qrcp_low_smem_bytes(m, n, grid, true);
        if (slots + cols > bcast_bytes || smem > 200 * 1024) return 1;
        gcols = (float*)((char*)bcast + slots);
        global_cols = true;
    }
    void* kern = global_cols ? (void*)k_qrcp_low<true> : (void*)k_qrcp_low<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail("qrcp_low smem attribute", e);
    const int threads = global_cols ? kLowThreadsGlobal : kLowThreads;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return cuda_fail("qrcp_low occupancy", e);
    if (occ < 1) return 1;
    void* args[] = {&m, &n, &A, &lda, &perm, &bcast, &st, &gcols};
    e = cudaLaunchCooperativeKernel(kern, grid, threads, args, smem, h->stream);
    if (e != cudaSuccess) return cuda_fail("qrcp_low launch", e);
    ++h->launch_count;
    return 0;
}

}  // namespace mpj
