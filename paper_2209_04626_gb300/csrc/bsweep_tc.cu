// bsweep_tc.cu -- the binary32 stage of the method (Section 3.2, Alg. 1 in the lower
// precision) in blocked form on the 5th-generation tensor cores.
//
// The n columns of X are cut into blocks of kBW = 64 columns and visited in the round-robin
// order of the register-resident stage (sweep.cuh): a sweep is k - 1 rounds of k / 2 disjoint
// block pairs, and a visit of (I, J) rotates every cross pair (i in I, j in J) once in kBW
// inner rounds of kBW disjoint pairs, plus, in the first round of a sweep, the pairs inside I
// and inside J. A visit works on Z = [X_I X_J] (mX x 128) in three steps:
//   1. G = Z^T Z (128 x 128) on the tensor cores, TF32 with a 3-term split (Ootomo and
//      Yokota's hi/lo split: z = hi + lo, hi = tf32(z), lo = tf32(z - hi), and
//      Z^T Z ~ hi^T hi + hi^T lo + lo^T hi), accumulated in FP32 in tensor memory;
//   2. the visit's rotations, each one the rotation of Section 2.1 for alpha = G_pp,
//      beta = G_qq, gamma = G_pq (the same test and formula as the register-resident
//      stage), applied to G (G <- J^T G J, the 2 x 2 block set to its exact result) and
//      accumulated into W (W <- W J, W = I at the start), in shared memory;
//   3. Z <- Z W on the tensor cores, TF32x3 again, in chunks of 128 rows.
// In exact arithmetic this is the register-resident visit: the dot products of an inner
// round are entries of the rotated Gram matrix. Scheduling is the same dataflow of block
// versions (a visit waits only for the two visits of the previous round that produced its
// blocks) with one grid barrier per sweep for the convergence test.
//
// Tensor-core use: one elected thread issues tcgen05.mma (kind::tf32, M = N = 128, K = 8) from
// K-major no-swizzle operand tiles that all threads write to shared memory after splitting;
// completion is tracked with tcgen05.commit on an mbarrier; the accumulator (128 lanes x 128
// FP32 columns of tensor memory) is read back with tcgen05.ld.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"
#include "tc.cuh"

// Phase probes of a visit: empty here; a profiling build may define them to record per-phase
// times (PROBE_BEGIN declares its state, PROBE(i) closes phase i).
#ifndef MPJ_TC_PROBE_BEGIN
#define MPJ_TC_PROBE_BEGIN
#define MPJ_TC_PROBE(i)
#endif

namespace mpj {

constexpr int kBW = 64;         // block width
constexpr int kB2 = 128;        // columns of a visit
constexpr int kBThreads = 256;
constexpr int kGP = 129;        // padded row stride (floats) of G and W in shared memory
constexpr uint32_t kTmemCols = 256;   // two 128-column FP32 accumulators
constexpr uint32_t kIdescTF32 = tc_idesc(128, 128, kTcFmtTF32);

// dynamic shared memory, three regions:
//   [0, 64 KiB)          Gram: two chunk buffers (hi 16 KiB + lo 16 KiB each)
//   [64 KiB, +kRegG)     G (128 x kGP floats)
//   [.., +kRegW)         W (128 x kGP floats)
// during the application of W, the B tiles of W (hi and lo, 64 KiB each) take [0, 128 KiB)
// (the Gram buffers and the dead G) and the A tiles of a 128-row chunk half (hi and lo,
// 32 KiB each) take W's region once W has been split
constexpr size_t kRegStage = 65536;
constexpr size_t kRegG = 66560;
constexpr size_t kRegW = 66560;
constexpr size_t kRegTab = 8192;                         // pairs of the intra rounds
constexpr size_t kBSmem = kRegStage + kRegG + kRegW + kRegTab;  // 206848 bytes

struct BVisitShared {
    int gidx[kB2];
    float cs[kBW], sn[kBW], nal[kBW], nbe[kBW];
    unsigned act[2];          // active pairs of the current inner round (bits 0..63)
    unsigned char pa[kBW], pb[kBW];  // the pairs of the current inner round
    int nrot;
    unsigned mxc, mxt;        // binary32 bits: largest cosine and |tan| rotated in the visit
    uint64_t mbar[2];
    int fail;                 // set by thread 0 when its bounded wait gave up
    uint32_t tmem;
    unsigned pend[2], par[2]; // per mbarrier: commits not yet waited for, parity of the next wait
};

// Pair p of an inner round of a 64-column block pair (columns 0..63 = I, 64..127 = J).
__device__ __forceinline__ void bpair(bool intra, int q, int p, int& a, int& b)
{
    if (!intra) {
        a = p;
        b = kBW + (p + q) % kBW;
        return;
    }
    const int half = kBW / 2, base = (p < half) ? 0 : kBW, ii = (p < half) ? p : p - half;
    rr_pair(kBW, q, ii, a, b);
    a += base;
    b += base;
}

// Thread 0 (the MMA issuer) waits (bounded) for every commit on mbarrier i that has not been
// waited for; then one CTA barrier. False for every thread if the wait gave up.
__device__ __forceinline__ bool drain1(BVisitShared& s, int i, DevState* st)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        while (s.pend[i]) {
            if (!mbar_wait1(&s.mbar[i], s.par[i], st)) {
                ok = 0;
                break;
            }
            s.par[i] ^= 1u;
            --s.pend[i];
        }
        s.fail = !ok;
    }
    __syncthreads();
    const bool ok = !s.fail;
    if (ok) tc_fence_after();
    return ok;
}

// Pieces of the Gram step's chunks of 32 rows (16 bytes each): the chunk is
// 128 columns x 8 pieces (rows 4 k4 .. 4 k4 + 3); warp w takes units w, w + 8, w + 16, w + 24,
// unit = (group of 8 columns cg, half kh of the chunk's rows); lane: column 8 cg + (lane & 7),
// piece k4 = 4 kh + (lane >> 3). A warp's load covers 8 columns x 64 contiguous bytes (whole
// 32-byte sectors), and the piece is one row of a K-major core matrix of the MMA operand.
__device__ __forceinline__ void gram_piece(int unit, int lane, int& cg, int& c, int& k4)
{
    cg = unit >> 1;
    c = cg * 8 + (lane & 7);
    k4 = (unit & 1) * 4 + (lane >> 3);
}

// Raw staging of the Gram step: kGramStages chunks in flight (cp.async, this thread's four
// pieces of a chunk at ((u * 8 + warp) * 32 + lane) * 16 of its stage), in the G and W regions,
// which hold nothing until the Gram is read back.
constexpr int kGramStages = 8;
constexpr size_t kGramRaw = 16384;  // one chunk: 128 columns x 32 rows of binary32
static_assert(kGramStages * kGramRaw <= kRegG + kRegW, "raw Gram stages must fit the G and W regions");

// Issue the copies of chunk ch into a raw stage. Rows at or beyond mX and phantom columns are
// zero-filled (their source address stays at the column's start). vec: X and ldX allow aligned
// 16-byte copies (else four 4-byte copies per piece).
__device__ __forceinline__ void gram_issue(const float* X, int ldX, int mX, const BVisitShared& s, int ch,
                                           bool vec, unsigned char* raw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int cg, c, k4;
        gram_piece(warp + 8 * u, lane, cg, c, k4);
        const int gc = s.gidx[c];
        const int r = ch * 32 + 4 * k4;
        const float* base = X + (size_t)(gc < 0 ? 0 : gc) * ldX;
        const int nv = (gc < 0) ? 0 : max(0, min(4, mX - r));  // rows of the piece inside X
        unsigned char* d = raw + (size_t)((u * 8 + warp) * 32 + lane) * 16;
        if (vec) {
            cp_async16(d, nv > 0 ? base + r : base, 4 * nv);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) cp_async4(d + 4 * e, e < nv ? base + r + e : base, e < nv ? 4 : 0);
        }
    }
}

// 1. G = Z^T Z into shared memory (row stride kGP); Z = columns gidx[] of X, rows 0..mX-1.
// Chunks of 32 rows stream in by cp.async, kGramStages - 1 ahead of the one being split; the
// MMAs of a chunk run while the next is split. Returns false if a wait gave up.
__device__ bool gram_tf32(const float* X, int ldX, int mX, BVisitShared& s, unsigned char* dsm,
                          float* G, DevState* st)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nch = (mX + 31) / 32;
    const bool vec = (ldX % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    unsigned char* rawb = dsm + kRegStage;
#pragma unroll 1
    for (int c = 0; c < kGramStages - 1; ++c) {
        if (c < nch) gram_issue(X, ldX, mX, s, c, vec, rawb + (size_t)c * kGramRaw);
        cp_async_commit();
    }
    for (int ch = 0; ch < nch; ++ch) {
        const int buf = ch & 1;
        // this thread's copies of chunk ch have landed (groups of chunks ch + 1 .. ch + 6 may
        // still be in flight: the copies of chunk ch + 7 are issued after this chunk's split,
        // so the proxy fence below never waits for a copy issued in this iteration)
        cp_async_wait<kGramStages - 2>();
        if (!drain1(s, buf, st)) {  // MMAs of chunk ch - 2 have read the buffer
            cp_async_wait_all();
            return false;
        }
        MPJ_TC_PROBE(4)
        const unsigned char* raw = rawb + (size_t)(ch % kGramStages) * kGramRaw;
        unsigned char* hi = dsm + buf * 32768;
        unsigned char* lo = hi + 16384;
        // one core-matrix row per piece: row group cg, k group k4, row c & 7
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int cg, c, k4;
            gram_piece(warp + 8 * u, lane, cg, c, k4);
            const float4 x4 = *(const float4*)(raw + (size_t)((u * 8 + warp) * 32 + lane) * 16);
            float4 h4, l4;
            const float* xp = &x4.x;
            float* hp = &h4.x;
            float* lp = &l4.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float hx = tf32_rna(xp[e]);
                hp[e] = hx;
                lp[e] = tf32_rna(xp[e] - hx);
            }
            const size_t off = (size_t)cg * 1024 + (size_t)k4 * 128 + (size_t)(c & 7) * 16;
            *(float4*)(hi + off) = h4;
            *(float4*)(lo + off) = l4;
        }
        fence_async_smem();
        __syncthreads();
        MPJ_TC_PROBE(5)
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ah = tc_desc(hi + ks * 256, 128, 1024);
                const uint64_t al = tc_desc(lo + ks * 256, 128, 1024);
                tc_mma_tf32(s.tmem, ah, ah, kIdescTF32, (ch > 0 || ks > 0) ? 1u : 0u);
                tc_mma_tf32(s.tmem, ah, al, kIdescTF32, 1u);
                tc_mma_tf32(s.tmem, al, ah, kIdescTF32, 1u);
            }
            tc_commit(&s.mbar[buf]);
            ++s.pend[buf];
        }
        MPJ_TC_PROBE(6)
        const int nx = ch + kGramStages - 1;  // its stage was read in iteration ch - 1
        if (nx < nch) gram_issue(X, ldX, mX, s, nx, vec, rawb + (size_t)(nx % kGramStages) * kGramRaw);
        cp_async_commit();
    }
    cp_async_wait_all();  // (only empty groups remain) before G overwrites the raw stages
    if (!drain1(s, 0, st) || !drain1(s, 1, st)) return false;
    // read back: warp w holds lanes 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63
    const int base = 32 * (warp & 3), c0 = 64 * (warp >> 2);
    const int row = base + lane;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float x[16];
        tmem_ld16(s.tmem + ((uint32_t)base << 16) + (uint32_t)(c0 + 16 * q), x);
#pragma unroll
        for (int e = 0; e < 16; ++e) G[row * kGP + c0 + 16 * q + e] = x[e];
    }
    tc_fence_before();
    __syncthreads();
    return true;
}

// Loads of one half (64 of the 128 columns) of a 128-row chunk for the application of W:
// thread: rows i = tid & 127, columns 4 k4 .. + 3 for k4 = tid >> 7, + 2, ..., + 14.
__device__ __forceinline__ void apply_load(const float* X, int ldX, int mX, const BVisitShared& s, int r0,
                                           int hlf, float (&v)[8][4])
{
    const int i = threadIdx.x & 127, k0 = threadIdx.x >> 7;
    const int r = r0 + i;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int k4 = k0 + 2 * t;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = s.gidx[64 * hlf + 4 * k4 + j];
            v[t][j] = (gc >= 0 && r < mX) ? __ldcg(X + (size_t)gc * ldX + r) : 0.0f;
        }
    }
}

__device__ __forceinline__ void apply_store_a(unsigned char* ahi, unsigned char* alo, const float (&v)[8][4])
{
    const int i = threadIdx.x & 127, k0 = threadIdx.x >> 7;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int k4 = k0 + 2 * t;
        float4 h4, l4;
        float* hp = &h4.x;
        float* lp = &l4.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float hx = tf32_rna(v[t][j]);
            hp[j] = hx;
            lp[j] = tf32_rna(v[t][j] - hx);
        }
        const size_t off = (size_t)(i >> 3) * 2048 + (size_t)k4 * 128 + (size_t)(i & 7) * 16;
        *(float4*)(ahi + off) = h4;
        *(float4*)(alo + off) = l4;
    }
}

// Epilogue of a chunk: accumulator columns (tensor memory at acc) -> rows r0.. of Z.
__device__ __forceinline__ void apply_epilogue(float* X, int ldX, int mX, const BVisitShared& s, int r0,
                                               uint32_t acc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = 32 * (warp & 3), c0 = 64 * (warp >> 2);
    const int r = r0 + base + lane;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float x[16];
        tmem_ld16(acc + ((uint32_t)base << 16) + (uint32_t)(c0 + 16 * q), x);
        if (r < mX) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int gc = s.gidx[c0 + 16 * q + e];
                if (gc >= 0) X[(size_t)gc * ldX + r] = x[e];
            }
        }
    }
}

// 3. Z <- Z W (columns gidx[] of X, rows 0..mX-1) with W (row stride kGP) in shared memory.
// Per 128-row chunk c: the two column halves of A go through one shared buffer; the chunk's
// MMAs accumulate into tensor-memory columns 128 (c & 1) .. + 127, so the epilogue of chunk
// c - 1 and the loads of the next half run while the tensor core works.
__device__ bool apply_tf32(float* X, int ldX, int mX, BVisitShared& s, unsigned char* dsm,
                           const float* W, DevState* st)
{
    const int tid = threadIdx.x;
    unsigned char* bhi = dsm;                             // over the Gram buffers and G
    unsigned char* blo = dsm + 65536;
    // B (N x K) = W^T, K-major: row n, reduction index k: B(n, k) = W(k, n)
    for (int e = tid; e < kB2 * 32; e += kBThreads) {
        const int n = e & 127, k4 = e >> 7;
        float4 h4, l4;
        float* hp = &h4.x;
        float* lp = &l4.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float x = W[(4 * k4 + j) * kGP + n];
            const float hx = tf32_rna(x);
            hp[j] = hx;
            lp[j] = tf32_rna(x - hx);
        }
        const size_t off = (size_t)(n >> 3) * 4096 + (size_t)k4 * 128 + (size_t)(n & 7) * 16;
        *(float4*)(bhi + off) = h4;
        *(float4*)(blo + off) = l4;
    }
    __syncthreads();  // W is read: its region holds the A tiles from here on
    unsigned char* ahi = dsm + kRegStage + kRegG;
    unsigned char* alo = ahi + 32768;
    const int nch = (mX + 127) / 128;
    float v[8][4];
    apply_load(X, ldX, mX, s, 0, 0, v);
    for (int ch = 0; ch < nch; ++ch) {
        const int r0 = ch * 128;
        const uint32_t acc = s.tmem + 128u * (uint32_t)(ch & 1);
        for (int hlf = 0; hlf < 2; ++hlf) {
            if (!drain1(s, 0, st)) return false;  // every MMA issued so far is complete
            apply_store_a(ahi, alo, v);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t ah = tc_desc(ahi + ks * 256, 128, 2048);
                    const uint64_t al = tc_desc(alo + ks * 256, 128, 2048);
                    const uint64_t bh = tc_desc(bhi + (8 * hlf + ks) * 256, 128, 4096);
                    const uint64_t bl = tc_desc(blo + (8 * hlf + ks) * 256, 128, 4096);
                    tc_mma_tf32(acc, ah, bh, kIdescTF32, (hlf > 0 || ks > 0) ? 1u : 0u);
                    tc_mma_tf32(acc, ah, bl, kIdescTF32, 1u);
                    tc_mma_tf32(acc, al, bh, kIdescTF32, 1u);
                }
                tc_commit(&s.mbar[0]);
                ++s.pend[0];
            }
            // the next half's (or chunk's) loads, then (after the first half) the previous
            // chunk's epilogue, while the MMAs run; its accumulator's MMAs completed before
            // this half was stored (drain above)
            if (hlf == 0) apply_load(X, ldX, mX, s, r0, 1, v);
            else if (ch + 1 < nch) apply_load(X, ldX, mX, s, r0 + 128, 0, v);
            if (hlf == 0 && ch > 0) {
                apply_epilogue(X, ldX, mX, s, r0 - 128, s.tmem + 128u * (uint32_t)((ch - 1) & 1));
                tc_fence_before();
            }
        }
    }
    if (!drain1(s, 0, st)) return false;
    apply_epilogue(X, ldX, mX, s, (nch - 1) * 128, s.tmem + 128u * (uint32_t)((nch - 1) & 1));
    tc_fence_before();
    __syncthreads();
    return true;
}

// Pair tables of the inner rounds of a 64-column block pair (columns 0..63 = I, 64..127 = J):
// cross round q pairs (p, 64 + (p + q) % 64); intra round q (first round of a sweep) pairs the
// columns inside I and inside J by the round-robin of rr_pair, 32 pairs each.
__device__ __forceinline__ void intra_table(unsigned short* tab)
{
    for (int e = threadIdx.x; e < (kBW - 1) * kBW; e += blockDim.x) {
        const int q = e / kBW, p = e % kBW;
        int a, b;
        bpair(true, q, p, a, b);
        tab[e] = (unsigned short)(a | (b << 8));
    }
}

// 2. the visit's inner rounds on G, accumulating W. Returns the number of rotations.
__device__ int rotate_gram(float* G, float* W, bool first, float tol, BVisitShared& s,
                           const unsigned short* itab)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < kB2 * kB2; e += kBThreads) {
        const int i = e >> 7, j = e & 127;
        W[i * kGP + j] = (i == j) ? 1.0f : 0.0f;
    }
    if (tid == 0) { s.nrot = 0; s.mxc = 0u; s.mxt = 0u; }
    __syncthreads();
    const int nr = first ? (kBW - 1) + kBW : kBW;
    for (int rr = 0; rr < nr; ++rr) {
        const bool intra = first && rr < kBW - 1;
        const int q = intra ? rr : rr - (first ? kBW - 1 : 0);
        // rotation parameters: thread p < 64 for pair p
        if (tid < kBW) {
            int a, b;
            if (intra) {
                const unsigned short ab = itab[q * kBW + tid];
                a = ab & 0xff;
                b = ab >> 8;
            } else {
                a = tid;
                b = kBW + ((tid + q) & (kBW - 1));
            }
            s.pa[tid] = (unsigned char)a;
            s.pb[tid] = (unsigned char)b;
            bool act = false;
            float cs = 0.0f, ta = 0.0f;
            if (s.gidx[a] >= 0 && s.gidx[b] >= 0) {
                const float al = G[a * kGP + a], be = G[b * kGP + b], ga = G[a * kGP + b];
                if (above_tol<float>(ga, al, be, tol, tol * tol)) {
                    float t, c, ic;
                    rot_params<float>(al, be, ga, t, c, ic);
                    s.cs[tid] = c;
                    s.sn[tid] = c * t;
                    s.nal[tid] = fmaf(-t, ga, al);
                    s.nbe[tid] = fmaf(t, ga, be);
                    cs = pair_cos(ga, al, be);
                    ta = fabsf(t);
                    act = true;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, act);
            const unsigned mc = __reduce_max_sync(0xffffffffu, __float_as_uint(cs));
            const unsigned mt = __reduce_max_sync(0xffffffffu, __float_as_uint(ta));
            if ((tid & 31) == 0) {
                s.act[tid >> 5] = m;
                atomicMax(&s.mxc, mc);
                atomicMax(&s.mxt, mt);
                atomicAdd(&s.nrot, __popc(m));
            }
        }
        __syncthreads();
        const unsigned m0 = s.act[0], m1 = s.act[1];
        if ((m0 | m1) == 0u) continue;  // uniform: every thread read the same masks
        const int half = tid >> 7;                       // pairs 0..31 or 32..63
        unsigned mk = half ? m1 : m0;
        // G <- J^T G (rows a, b of every active pair); thread: column j
        {
            const int j = tid & 127;
            for (unsigned m = mk; m; m &= m - 1) {
                const int p = 32 * half + __ffs(m) - 1;
                const int a = s.pa[p], b = s.pb[p];
                const float c = s.cs[p], sv = s.sn[p];
                const float ga = G[a * kGP + j], gb = G[b * kGP + j];
                G[a * kGP + j] = fmaf(c, ga, -sv * gb);
                G[b * kGP + j] = fmaf(sv, ga, c * gb);
            }
        }
        __syncthreads();
        // G <- G J and W <- W J (columns a, b); the 2 x 2 block of each pair gets its exact
        // result (alpha - t gamma, beta + t gamma, 0); thread: row i
        {
            const int i = tid & 127;
            for (unsigned m = mk; m; m &= m - 1) {
                const int p = 32 * half + __ffs(m) - 1;
                const int a = s.pa[p], b = s.pb[p];
                const float c = s.cs[p], sv = s.sn[p];
                const float ga = G[i * kGP + a], gb = G[i * kGP + b];
                float na = fmaf(c, ga, -sv * gb), nb = fmaf(sv, ga, c * gb);
                if (i == a) { na = s.nal[p]; nb = 0.0f; }
                if (i == b) { na = 0.0f; nb = s.nbe[p]; }
                G[i * kGP + a] = na;
                G[i * kGP + b] = nb;
                const float wa = W[i * kGP + a], wb = W[i * kGP + b];
                W[i * kGP + a] = fmaf(c, wa, -sv * wb);
                W[i * kGP + b] = fmaf(sv, wa, c * wb);
            }
        }
        __syncthreads();
    }
    return s.nrot;
}

// One visit of block pair (bi, bj). Returns the rotation count, or -1 if a wait gave up.
__device__ int bvisit(const SweepDims& D, float* X, int bi, int bj, bool first, BVisitShared& s,
                      unsigned char* dsm, DevState* st)
{
    const int tid = threadIdx.x;
    if (tid < kB2) {
        const int blk = (tid < kBW) ? bi : bj;
        const int c = blk * kBW + (tid & (kBW - 1));
        s.gidx[tid] = (c < D.n) ? c : -1;
    }
    __syncthreads();
    float* G = (float*)(dsm + kRegStage);
    float* W = (float*)(dsm + kRegStage + kRegG);
    if (!gram_tf32(X, D.ldX, D.mX, s, dsm, G, st)) return -1;
    MPJ_TC_PROBE(1)
    const int nrot = rotate_gram(G, W, first, (float)D.tol, s,
                                 (const unsigned short*)(dsm + kRegStage + kRegG + kRegW));
    MPJ_TC_PROBE(2)
    if (nrot > 0 && !apply_tf32(X, D.ldX, D.mX, s, dsm, W, st)) return -1;
    MPJ_TC_PROBE(3)
    return nrot;
}

__device__ int bsweeps_flow(const Group& g, const SweepDims& D, float* X, unsigned long long* rot_sweep,
                            unsigned* mxc, unsigned* mxt, BVisitShared& s, unsigned char* dsm, bool* converged)
{
    const int k = D.k, half = k / 2, rounds = k - 1;
    const long long per_sweep = (long long)rounds * half;
    int sweep = 0;
    *converged = false;
    for (; sweep < D.maxsweep; ++sweep) {
        for (long long f = g.rank; f < per_sweep; f += g.size) {
            const int r = (int)(f / half), i = (int)(f - (long long)r * half);
            int bi, bj;
            rr_pair(k, r, i, bi, bj);
            if (bi > bj) { const int t = bi; bi = bj; bj = t; }
            const unsigned R = (unsigned)(sweep * rounds + r);
            MPJ_TC_PROBE_BEGIN
            if (!wait_blocks(D.ver, bi, bj, R, g.st)) return -1;
            MPJ_TC_PROBE(0)
            const int nrot = bvisit(D, X, bi, bj, r == 0, s, dsm, g.st);
            if (nrot < 0) return -1;
            __syncthreads();
            if (threadIdx.x == 0) {
                if (nrot) {
                    atomicAdd(&rot_sweep[sweep], (unsigned long long)nrot);
                    atomicMax(mxc + sweep, s.mxc);
                    atomicMax(mxt + sweep, s.mxt);
                }
                __threadfence();
                st_release_u32(D.ver + bi, R + 1);
                st_release_u32(D.ver + bj, R + 1);
            }
        }
        if (!g.sync()) return -1;
        if (__ldcg(&rot_sweep[sweep]) == 0 || negligible_sweep(D, mxc, mxt, sweep)) {
            *converged = true;
            ++sweep;
            break;
        }
    }
    return sweep;
}

// The whole binary32 stage in one cooperative launch (one CTA per SM). Returns at once if the
// call already failed or the gate says the stage is skipped.
__global__ void __launch_bounds__(kBThreads, 1) k_bsweeps_tf32(SweepDims D, float* X, DevState* st, int phase,
                                                               int gate_want)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ BVisitShared s;
    if (call_failed(st)) return;
    if (!gate_open(st, gate_want)) return;
    const Group g{(int)blockIdx.x, (int)gridDim.x, st};
    if (threadIdx.x < 32) tmem_alloc(&s.tmem, kTmemCols);
    if (threadIdx.x == 0) {
        mbar_init(&s.mbar[0]);
        mbar_init(&s.mbar[1]);
        s.pend[0] = s.pend[1] = 0u;
        s.par[0] = s.par[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.k; b += gridDim.x * blockDim.x) D.ver[b] = 0u;
    intra_table((unsigned short*)(dsm + kRegStage + kRegG + kRegW));
    int sweeps = -1;
    bool conv = false;
    if (g.sync())
        sweeps = bsweeps_flow(g, D, X, st->rot_sweep[phase], st->mx_cos[phase], st->mx_tan[phase], s, dsm, &conv);
    if (sweeps < 0) {
        // a wait gave up: MMAs this CTA issued may still be running; wait for them (bounded)
        // before the tensor memory is released
        if (threadIdx.x == 0) {
            const uint64_t t0 = globaltimer_ns();
            for (int i = 0; i < 2; ++i)
                while (s.pend[i] && !mbar_test(&s.mbar[i], s.par[i]) && globaltimer_ns() - t0 < 100000000ull) {}
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_free(s.tmem, kTmemCols);
    if (sweeps < 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int sw = 0; sw < sweeps; ++sw) tot += __ldcg(&st->rot_sweep[phase][sw]);
        if (phase == 0) { st->sweeps_low = sweeps; st->rot_low = tot; }
        else { st->sweeps_work = sweeps; st->rot_work = tot; }
        if (!conv) atomicOr(&st->status, MPJSVD_STATUS_NOT_CONVERGED);
    }
}

int launch_bsweeps_tf32(mpjsvd_ctx* h, const SweepDims& D0, float* X, DevState* st, int phase, int gate_want)
{
    SweepDims D = D0;
    if (D.w != kBW) return cuda_fail("blocked binary32 sweeps: block width must be 64", cudaErrorInvalidValue);
    cudaError_t e = cudaFuncSetAttribute((void*)k_bsweeps_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBSmem);
    if (e != cudaSuccess) return cuda_fail("blocked sweeps smem attribute", e);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bsweeps_tf32, kBThreads, kBSmem);
    if (e != cudaSuccess) return cuda_fail("blocked sweeps occupancy", e);
    if (occ < 1) return cuda_fail("blocked sweeps occupancy (0 blocks fit)", cudaErrorInvalidConfiguration);
    int grid = std::max(1, std::min(D.k, h->num_sms));
    void* args[] = {&D, &X, &st, &phase, &gate_want};
    e = cudaLaunchCooperativeKernel((void*)k_bsweeps_tf32, grid, kBThreads, args, kBSmem, h->stream);
    if (e != cudaSuccess) return cuda_fail("blocked sweeps launch", e);
    ++h->launch_count;
    return 0;
}

// ---- standalone building blocks (one CTA): G = Z^T Z and Z <- Z W for a 128-column Z

__global__ void __launch_bounds__(kBThreads, 1) k_tc_block(int mX, float* Z, int ldz, float* Gout,
                                                           const float* Win, DevState* st)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ BVisitShared s;
    if (threadIdx.x < 32) tmem_alloc(&s.tmem, kTmemCols);
    if (threadIdx.x == 0) {
        mbar_init(&s.mbar[0]);
        mbar_init(&s.mbar[1]);
        s.pend[0] = s.pend[1] = 0u;
        s.par[0] = s.par[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < kB2) s.gidx[threadIdx.x] = threadIdx.x;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    float* G = (float*)(dsm + kRegStage);
    float* W = (float*)(dsm + kRegStage + kRegG);
    bool ok = true;
    if (Gout) {
        ok = gram_tf32(Z, ldz, mX, s, dsm, G, st);
        if (ok)
            for (int e = threadIdx.x; e < kB2 * kB2; e += kBThreads) Gout[e] = G[(e & 127) * kGP + (e >> 7)];
    }
    if (ok && Win) {
        for (int e = threadIdx.x; e < kB2 * kB2; e += kBThreads) W[(e & 127) * kGP + (e >> 7)] = Win[e];
        __syncthreads();
        ok = apply_tf32(Z, ldz, mX, s, dsm, W, st);
    }
    if (!ok && threadIdx.x == 0) {
        const uint64_t t0 = globaltimer_ns();
        for (int i = 0; i < 2; ++i)
            while (s.pend[i] && !mbar_test(&s.mbar[i], s.par[i]) && globaltimer_ns() - t0 < 100000000ull) {}
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_free(s.tmem, kTmemCols);
}

int tc_block_call(mpjsvd_ctx* h, int m, float* Z, int ldz, float* G, const float* W)
{
    h->launch_count = 0;
    int rc = state_reset(h, h->dstate);
    if (rc) return rc;
    cudaError_t e = cudaFuncSetAttribute((void*)k_tc_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem);
    if (e != cudaSuccess) return cuda_fail("tc block smem attribute", e);
    k_tc_block<<<1, kBThreads, kBSmem, h->stream>>>(m, Z, ldz, G, W, (DevState*)h->dstate);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("tc block launch", e);
    ++h->launch_count;
    return 0;
}

}  // namespace mpj

extern "C" int mpjsvd_tc_block_f32(mpjsvd_handle h, int m, float* Z, int ldz, float* G, const float* W)
{
    if (!h) return -1;
    if (m < 1 || m > (1 << 24)) return -2;
    if (!Z) return -3;
    if (ldz < m) return -4;
    if (!G && !W) return -5;
    return mpj::tc_block_call(h, m, Z, ldz, G, W);
}
