// sweep.cuh -- one-sided Jacobi sweeps (Alg. 1 of the paper, Section 2.1) over a parallel
// round-robin ordering of column blocks.
//
// Ordering. The n columns are cut into k blocks of W columns (k even; a phantom block
// pads odd counts). A sweep is k-1 rounds of the circle-method tournament; in round r the
// k/2 block pairs are disjoint, so their visits run concurrently on different CTAs. A
// visit of blocks (I, J) rotates every cross pair (i in I, j in J) once (W inner rounds of
// W disjoint pairs); in round 0 it also rotates the pairs inside I and inside J. Over a
// sweep every column pair is visited exactly once, as in the cyclic order of eq. (cyclic),
// but in a different sequence.
//
// Rotation (Section 2.1). For a pair (p, q) with alpha = |x_p|^2, beta = |x_q|^2 and
// gamma = x_p^T x_q, the pair is rotated when |gamma| > tol sqrt(alpha) sqrt(beta); then
// zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), x_p' = c (x_p - t x_q), x_q' = c (x_q + t x_p),
// alpha' = alpha - t gamma, beta' = beta + t gamma. The kernels evaluate the same t as
// sign(zeta) 2|gamma| / (|beta - alpha| + sqrt((beta - alpha)^2 + 4 gamma^2)) on operands
// scaled by a power of two (rot_params): one reciprocal square root and one reciprocal
// instead of two divisions and a square root, which matters because every binary64
// operation on this chain costs a full FP64 pipe latency.
//
// Scaled ("fast") form. Each column is kept as x = d * xh with a scale d that persists
// across visits (global arrays dsc, alph hold d and the tracked alpha of every column).
// The update becomes xh_p -= (t d_q / d_p) xh_q, xh_q += (t d_p / d_q) xh_p, d_p *= c,
// d_q *= c: two FMAs per row instead of two multiplies and two FMAs. V shares the scales.
// A column is folded (xh *= d, d = 1) only when d gets small; the caller folds the rest
// once after the last sweep. The tracked norms are recomputed from the data in round 0 of
// every sweep (each column is visited exactly once there) and whenever a cancellation
// makes a tracked value unreliable.
//
// Execution. A visit keeps its 2W columns in REGISTERS: thread t owns rows t, t + T, ...
// (RPT of them, T threads). Inner rounds are fully unrolled, so every column index is a
// compile-time constant: the dot products and updates touch no shared memory. The W dot
// products of a round are combined by one multi-value warp reduction and W lanes of warp 0
// compute the W rotations. Their parameters go to a dense per-round table; V's rows are
// then streamed through registers and each thread replays the table on its rows.
//
// Scheduling (single-matrix path). Rounds are not separated by grid barriers: each block has
// a version counter (the number of rounds that have finished with it), and a visit of round
// R waits only until its two blocks have reached version R, i.e. until the two visits of
// round R-1 that produced them have stored their columns. Several CTAs per SM then overlap
// one visit's latency-bound steps (reductions, rotation parameters) with another visit's
// FP64 arithmetic. One grid barrier per sweep decides convergence.
#pragma once

#include "common.cuh"

namespace mpj {

// Circle-method round-robin: block k-1 is fixed, the others rotate. Pairs (a, b) of round
// r for i = 0 .. k/2-1 are disjoint, and over r = 0 .. k-2 every pair of blocks meets once.
__host__ __device__ __forceinline__ constexpr void rr_pair(int k, int r, int i, int& a, int& b)
{
    if (i == 0) {
        a = k - 1;
        b = r;
    } else {
        a = (r + i) % (k - 1);
        b = (r - i + (k - 1)) % (k - 1);
    }
}

// 2^-e for the larger binary exponent e of |a| and |b| (clamped so the result is normal):
// multiplying by it brings max(|a|, |b|) into [1, 2) exactly. Integer work only.
__device__ __forceinline__ double pow2_down(double a, double b)
{
    int ea = (__double2hiint(a) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
    int e = min(max(max(ea, eb), 1), 2045);
    return __hiloint2double((2046 - e) << 20, 0);
}
__device__ __forceinline__ float pow2_down(float a, float b)
{
    int ea = (__float_as_int(a) >> 23) & 0xff, eb = (__float_as_int(b) >> 23) & 0xff;
    int e = min(max(max(ea, eb), 1), 253);
    return __int_as_float((254 - e) << 23);
}

// Rotation of Section 2.1 for (alpha, beta, gamma), gamma != 0: t (the root of
// t^2 + 2 zeta t - 1 = 0 with |t| <= 1, zeta = (beta - alpha) / (2 gamma); t > 0 when
// zeta = 0), c = 1 / sqrt(1 + t^2) and 1 / c. With dd = beta - alpha, g2 = 2 gamma,
// D = sqrt(dd^2 + g2^2) and S = |dd| + D: |t| = |g2| / S, sign(t) = sign(dd) sign(gamma).
// t depends only on the ratio dd : g2, so both are first scaled by a power of two: no
// intermediate overflows or underflows for any finite input.
template <typename T>
__device__ __forceinline__ void rot_params(T alpha, T beta, T gamma, T& t, T& c, T& ic)
{
    const T dd = beta - alpha, g2 = T(2) * gamma;
    const T sc = pow2_down(dd, g2);
    const T ds = dd * sc, gs = g2 * sc;
    const T D2 = fma(ds, ds, gs * gs);
    const T D = D2 * rsqrt(D2);
    const T r = T(1) / (fabs(ds) + D);
    const T num = (dd == T(0)) ? fabs(gs) : ((dd > T(0)) ? gs : -gs);
    t = num * r;
    const T q1 = fma(t, t, T(1));
    c = rsqrt(q1);
    ic = q1 * c;
}

// gamma / dd for the rare case below (not inlined: keeps the division off the common path).
static __device__ __noinline__ double ratio_slow(double gamma, double dd) { return gamma / dd; }

// binary64 variant: t is evaluated in binary32 from the scaled operands and then used exactly
// as a binary64 number. The transformation [c, c t; -c t, c] is orthogonal to binary64
// precision for ANY t as long as c = 1 / sqrt(1 + t^2) is accurate for that t, which is
// computed in binary64; only how completely the pair is annihilated (to ~2^-23 of gamma)
// depends on t, and the next sweep removes the remainder. The binary32 chain is about a
// fifth as long as the binary64 one (each binary64 operation costs a full FP64 pipe
// latency on this part). If the scaled gamma underflows binary32 (|gamma| < 2^-126 |dd|),
// t = gamma / dd is taken in binary64.
template <>
__device__ __forceinline__ void rot_params<double>(double alpha, double beta, double gamma, double& t,
                                                   double& c, double& ic)
{
    const double dd = beta - alpha;
    const double sc = pow2_down(dd, gamma);
    const float ds = (float)(dd * sc), gs = 2.0f * (float)(gamma * sc);
    const float D2 = fmaf(ds, ds, gs * gs);
    const float D = D2 * rsqrtf(D2);
    const float num = (ds == 0.0f) ? fabsf(gs) : ((ds > 0.0f) ? gs : -gs);
    const float tf = __fdividef(num, fabsf(ds) + D);
    t = (double)tf;
    if (tf == 0.0f) t = ratio_slow(gamma, dd);
    const double q1 = fma(t, t, 1.0);
    c = rsqrt(q1);
    ic = q1 * c;
}

// binary32 variant (the lower-precision stage): the reciprocal by the fast division
// intrinsic (a tangent off by a few ulps only changes how completely the pair is
// annihilated); the cosine is rsqrtf(1 + t^2) for that t, orthogonal to binary32 precision.
template <>
__device__ __forceinline__ void rot_params<float>(float alpha, float beta, float gamma, float& t, float& c,
                                                  float& ic)
{
    const float dd = beta - alpha, g2 = 2.0f * gamma;
    const float sc = pow2_down(dd, g2);
    const float ds = dd * sc, gs = g2 * sc;
    const float D2 = fmaf(ds, ds, gs * gs);
    const float D = D2 * rsqrtf(D2);
    const float num = (dd == 0.0f) ? fabsf(gs) : ((dd > 0.0f) ? gs : -gs);
    t = __fdividef(num, fabsf(ds) + D);
    const float q1 = fmaf(t, t, 1.0f);
    c = rsqrtf(q1);
    ic = q1 * c;
}

// True when x <= 0 or x < y / 16 up to a factor of two (y > 0), from the sign and binary
// exponents (no floating-point instruction): flags a tracked norm that lost about four bits
// to cancellation.
__device__ __forceinline__ bool lost_bits(double x, double y)
{
    const int hx = __double2hiint(x);
    if (hx <= 0) return true;  // negative, zero, or far below any normal y
    return ((hx >> 20) & 0x7ff) + 4 < ((__double2hiint(y) >> 20) & 0x7ff);
}
__device__ __forceinline__ bool lost_bits(float x, float y)
{
    const int bx = __float_as_int(x);
    if (bx <= 0) return true;  // negative or zero
    return ((bx >> 23) & 0xff) + 4 < ((__float_as_int(y) >> 23) & 0xff);
}

// The rotation test of Section 2.1, |gamma| > tol |x_a| |x_b|, from gamma and the squared
// norms alpha = |x_a|^2, beta = |x_b|^2. binary32 takes the square roots: compared as squares,
// alpha beta underflows once both columns are below about 1e-10 of unit size, and those pairs
// would never be rotated (their directions would stay unresolved in the lower-precision
// stage). binary64 compares squares, gamma^2 > tol^2 alpha beta (no square root on the scarce
// FP64 pipe), which stays in range for column norms down to about 1e-75.
template <typename T>
__device__ __forceinline__ bool above_tol(T gamma, T al, T be, T tol, T tol2);
template <>
__device__ __forceinline__ bool above_tol<double>(double gamma, double al, double be, double, double tol2)
{
    return gamma * gamma > tol2 * (al * be);
}
template <>
__device__ __forceinline__ bool above_tol<float>(float gamma, float al, float be, float tol, float)
{
    return fabsf(gamma) > tol * (sqrtf(al) * sqrtf(be));
}

// Cosine |gamma| / (|x_a| |x_b|) of a rotated pair as binary32, for the stopping rule. binary64:
// from the significands and exponents of gamma, alpha, beta (integer arithmetic and binary32
// only, nothing on the FP64 pipe); 0 when it is below 2^-63, 1 for non-normal norms (a
// conservative value: it never ends the iteration early).
__device__ __forceinline__ float pair_cos(double gamma, double al, double be)
{
    const long long ig = __double_as_longlong(gamma) & 0x7fffffffffffffffll;
    const long long ia = __double_as_longlong(al), ib = __double_as_longlong(be);
    const int eg = (int)(ig >> 52), ea = (int)((ia >> 52) & 0x7ff), eb = (int)((ib >> 52) & 0x7ff);
    if (eg == 0) return 0.0f;
    if (ea == 0 || eb == 0 || ea == 0x7ff || eb == 0x7ff || eg == 0x7ff) return 1.0f;
    const float mg = __int_as_float(0x3f800000 | (int)((ig >> 29) & 0x7fffff));  // [1, 2)
    const float ma = __int_as_float(0x3f800000 | (int)((ia >> 29) & 0x7fffff));
    const float mb = __int_as_float(0x3f800000 | (int)((ib >> 29) & 0x7fffff));
    const int k2 = 2 * eg - ea - eb;  // cos^2 = mg^2 / (ma mb) * 2^k2
    if (k2 < -126) return 0.0f;
    if (k2 > 126) return 1.0f;
    const float c2 = (mg * mg) / (ma * mb) * __int_as_float((k2 + 127) << 23);
    return sqrtf(c2);
}
__device__ __forceinline__ float pair_cos(float gamma, float al, float be)
{
    return fabsf(gamma) / (sqrtf(al) * sqrtf(be));
}

// Sum of n >= 1 values with a dependency depth of about log2(4) + n / 4 instead of n.
template <typename T>
__device__ __forceinline__ T short_sum(const T* v, int n)
{
    T s0 = v[0], s1 = T(0), s2 = T(0), s3 = T(0);
    if (n > 1) s1 = v[1];
    if (n > 2) s2 = v[2];
    if (n > 3) s3 = v[3];
    int k = 4;
    for (; k + 3 < n; k += 4) {
        s0 += v[k];
        s1 += v[k + 1];
        s2 += v[k + 2];
        s3 += v[k + 3];
    }
    for (; k < n; ++k) s0 += v[k];
    return (s0 + s1) + (s2 + s3);
}

// Acquire load / release store of a version counter (cross-CTA hand-off of a block).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct SweepDims {
    int n;       // columns of X (and of V)
    int mX;      // rows of X (<= RPT * blockDim.x)
    int ldX;
    int nV;      // rows of V (0: no V)
    int ldV;
    int w;       // block width (== W of the kernel)
    int k;       // number of blocks (even)
    int maxsweep;
    int stop;    // MPJSVD_STOP_*: also stop after a negligible sweep (0) or not (1)
    double tol;  // rotation threshold
    void* dsc;   // T[n]: column scales, 1 at the start of the stage
    void* alph;  // T[n]: tracked squared norms (true scale)
    unsigned* ver;  // 2k block versions, X then V (cooperative single-matrix launch only)
    // pair filter (the Y1/Y2 safeguard of Section 3.4): 0 every pair; 1 only pairs of columns
    // >= *j0 (Alg. 1 on Y2); 2 only pairs with one column < *j0 and one >= *j0 (one pass over
    // the pairs between Y1 and Y2). j0: device int, read when a visit starts.
    int filter = 0;
    const int* j0 = nullptr;
};

constexpr int kMaxWarps = 32;

// Shared memory of a visit (static per instantiation).
template <typename T, int W>
struct VisitShared {
    T part[2 * W][kMaxWarps];   // per-warp partial sums
    T alpha[2 * W];
    T d[2 * W];
    T dinv[2 * W];
    T tab[2 * W][W];            // rotation parameters per inner round (<= 2W - 1 rounds)
    T tba[2 * W][W];
    T fold[2 * W];              // 1, or the factor a column was folded by at the store
    int gidx[2 * W];
    unsigned act[2 * W];        // active-pair mask per inner round
    int flags[4];               // [0] rotations, [1] norms need recomputing
    unsigned mxc, mxt;          // binary32 bits: largest cosine and |tan| rotated in the visit
    unsigned char side[2 * W];  // pair filter 2: 1 for a column < j0
    int cross_only;             // pair filter 2 active
};

// Pair p of an inner round. Cross rounds: (p, W + (p + q) % W). Intra rounds (W even,
// round-robin inside each block): pairs 0..W/2-1 inside I, W/2..W-1 inside J.
template <int W>
__device__ __forceinline__ constexpr int pair_a(bool intra, int q, int p)
{
    if (!intra) return p;
    int half = W / 2, base = (p < half) ? 0 : W, ii = (p < half) ? p : p - half;
    int a = 0, b = 0;
    rr_pair(W, q, ii, a, b);
    return base + a;
}
template <int W>
__device__ __forceinline__ constexpr int pair_b(bool intra, int q, int p)
{
    if (!intra) return W + (p + q) % W;
    int half = W / 2, base = (p < half) ? 0 : W, ii = (p < half) ? p : p - half;
    int a = 0, b = 0;
    rr_pair(W, q, ii, a, b);
    return base + b;
}

// Squared norms of the 2W register columns into sm.alpha (true scale). Ends synchronized.
template <typename T, int W, int RPT>
__device__ __forceinline__ void reg_norms(const T (&x)[RPT][2 * W], VisitShared<T, W>& sm)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    T acc[2 * W];
#pragma unroll
    for (int c = 0; c < 2 * W; ++c) {
        acc[c] = T(0);
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[c] = fma(x[k][c], x[k][c], acc[c]);
    }
    warp_reduce_multi<2 * W>(acc, lane);
    constexpr int sh = 5 - ilog2c(2 * W);
    if ((lane & ((1 << sh) - 1)) == 0) sm.part[lane >> sh][wid] = acc[0];
    __syncthreads();
    if (tid < 2 * W) {
        const T s = short_sum(sm.part[tid], nw);
        T dc = sm.d[tid];
        sm.alpha[tid] = (sm.gidx[tid] >= 0) ? s * dc * dc : T(0);
    }
    __syncthreads();
}

// One inner round (pairs given by intra/q), slot = its index in the visit's table.
template <typename T, bool WITH_V, int W, int RPT>
__device__ __forceinline__ void inner_round(T (&x)[RPT][2 * W], bool intra, int q, int slot,
                                            VisitShared<T, W>& sm, T tol, T tol2)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    constexpr int SH = 5 - ilog2c(W);
    // phase A: partial dot products of the W pairs over this thread's rows
    T acc[W];
#pragma unroll
    for (int p = 0; p < W; ++p) {
        const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
        acc[p] = T(0);
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[p] = fma(x[k][a], x[k][b], acc[p]);
    }
    warp_reduce_multi<W>(acc, lane);
    if ((lane & ((1 << SH) - 1)) == 0) sm.part[lane >> SH][wid] = acc[0];
    __syncthreads();
    // phase B: rotation parameters, lane p of warp 0 for pair p
    if (tid < W) {
        const int p = tid;
        const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
        unsigned act = 0;
        float cs = 0.0f, ta = 0.0f;  // cosine and |tan| of this pair's rotation (stopping rule)
        if (sm.gidx[a] >= 0 && sm.gidx[b] >= 0 && (!sm.cross_only || sm.side[a] != sm.side[b])) {
            const T gh = short_sum(sm.part[p], nw);
            const T da = sm.d[a], db = sm.d[b];
            const T ia = sm.dinv[a], ib = sm.dinv[b];
            const T al = sm.alpha[a], be = sm.alpha[b];
            const T gamma = gh * (da * db);
            if (above_tol<T>(gamma, al, be, tol, tol2)) {
                T t, c, ic;  // tangent, cosine and 1 / cosine of the rotation
                rot_params(al, be, gamma, t, c, ic);
                cs = pair_cos(gamma, al, be);
                ta = fabsf((float)t);
                sm.tab[slot][p] = t * (db * ia);
                sm.tba[slot][p] = t * (da * ib);
                sm.d[a] = da * c;
                sm.d[b] = db * c;
                sm.dinv[a] = ia * ic;
                sm.dinv[b] = ib * ic;
                const T na = fma(-t, gamma, al), nb = fma(t, gamma, be);
                if (lost_bits(na, al) || lost_bits(nb, be)) sm.flags[1] = 1;
                sm.alpha[a] = na;
                sm.alpha[b] = nb;
                act = 1u << p;
            }
        }
        // combine the W bits of warp 0's lanes
        unsigned m = __reduce_or_sync((1u << W) - 1u, act);
        const unsigned mc = __reduce_max_sync((1u << W) - 1u, __float_as_uint(cs));
        const unsigned mt = __reduce_max_sync((1u << W) - 1u, __float_as_uint(ta));
        if (p == 0) {
            sm.act[slot] = m;
            sm.flags[0] += __popc(m);
            sm.mxc = max(sm.mxc, mc);
            sm.mxt = max(sm.mxt, mt);
        }
    }
    __syncthreads();
    // phase C: apply the active rotations to this thread's rows
    const unsigned m = sm.act[slot];
    if (m) {
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (!(m & (1u << p))) continue;
            const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
            const T tab = sm.tab[slot][p], tba = sm.tba[slot][p];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                T ya = x[k][a], yb = x[k][b];
                x[k][a] = fma(-tab, yb, ya);
                x[k][b] = fma(tba, ya, yb);
            }
        }
    }
    if (sm.flags[1]) {  // rare: a tracked norm lost its accuracy; recompute all 2W
        reg_norms<T, W, RPT>(x, sm);
        if (tid == 0) sm.flags[1] = 0;
        __syncthreads();
    }
}

// Replay the visit's rotation table on R rows of V held in v[][] (compile-time column
// indices): rotations in table order, each applied to all R rows.
template <int W, int R, typename T>
__device__ __forceinline__ void replay_rows(double (&v)[R][2 * W], bool first, const VisitShared<T, W>& sm)
{
    const int nintra = first ? W - 1 : 0;
#pragma unroll
    for (int q = 0; q < W - 1; ++q) {
        if (q >= nintra) break;
        const unsigned m = sm.act[q];
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (!(m & (1u << p))) continue;
            const int a = pair_a<W>(true, q, p), b = pair_b<W>(true, q, p);
            const double ta = (double)sm.tab[q][p], tb = (double)sm.tba[q][p];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const double va = v[k][a], vb = v[k][b];
                v[k][a] = fma(-ta, vb, va);
                v[k][b] = fma(tb, va, vb);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const int slot = nintra + q;
        const unsigned m = sm.act[slot];
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (!(m & (1u << p))) continue;
            const int a = pair_a<W>(false, q, p), b = pair_b<W>(false, q, p);
            const double ta = (double)sm.tab[slot][p], tb = (double)sm.tba[slot][p];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const double va = v[k][a], vb = v[k][b];
                v[k][a] = fma(-ta, vb, va);
                v[k][b] = fma(tb, va, vb);
            }
        }
    }
}

// X part of one visit of block pair (bi, bj): load to registers, rotate, store X, scales
// and tracked norms. Returns the rotation count (all threads) and leaves the visit's rotation
// table, fold factors and column indices in sm for replay_v. All threads of the CTA must
// call it; mX <= RPT * blockDim.x.
template <typename T, bool WITH_V, int W, int RPT>
__device__ int jacobi_visit_x(const SweepDims& D, T* X, int bi, int bj, bool first,
                              VisitShared<T, W>& sm)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int W2 = 2 * W;
    const T tol1 = T(D.tol), tol2 = T(D.tol * D.tol);
    T* dsc = (T*)D.dsc;
    T* alph = (T*)D.alph;
    // fold a column into its data once its scale is this small (persistent scales only
    // shrink: c <= 1); binary32 needs it long before underflow
    const T fold_min = sizeof(T) == 8 ? T(1e-120) : T(1e-12);

    if (tid < W2) {
        int blk = (tid < W) ? bi : bj;
        int c = blk * W + (tid < W ? tid : tid - W);
        bool ok = (blk * W < D.n) && (c < D.n);
        if (D.filter != 0) {
            const int j0 = *(volatile const int*)D.j0;
            if (D.filter == 1 && c < j0) ok = false;  // Y1 columns stay as they are
            sm.side[tid] = (unsigned char)(c < j0);
        }
        sm.gidx[tid] = ok ? c : -1;
        T dc = ok ? __ldcg(dsc + c) : T(1);
        sm.d[tid] = dc;
        sm.dinv[tid] = T(1) / dc;
        sm.alpha[tid] = ok ? __ldcg(alph + c) : T(0);
        sm.fold[tid] = T(1);
    }
    if (tid == 0) {
        sm.flags[0] = 0;
        sm.flags[1] = 0;
        sm.mxc = 0u;
        sm.mxt = 0u;
        sm.cross_only = (D.filter == 2);
    }
    __syncthreads();

    // ---- load the rows of the 2W columns (through L2: other CTAs wrote them)
    T x[RPT][W2];
#pragma unroll
    for (int c = 0; c < W2; ++c) {
        const int gc = sm.gidx[c];
        const T* col = X + (size_t)(gc < 0 ? 0 : gc) * D.ldX;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = tid + k * nthr;
            x[k][c] = (gc >= 0 && r < D.mX) ? __ldcg(col + r) : T(0);
        }
    }
    // binary32 norms are recomputed at every visit: tracked over a whole sweep (about n
    // updates per column) they drift enough to misjudge convergence; binary64 ones only in
    // round 0 of each sweep
    const bool fresh = first || sizeof(T) == 4;
    if (fresh) reg_norms<T, W, RPT>(x, sm);

    // ---- inner rounds (unrolled: compile-time column indices)
    if (first) {
#pragma unroll
        for (int q = 0; q < W - 1; ++q) inner_round<T, WITH_V, W, RPT>(x, true, q, q, sm, tol1, tol2);
    }
    const int base = first ? W - 1 : 0;
#pragma unroll
    for (int q = 0; q < W; ++q) inner_round<T, WITH_V, W, RPT>(x, false, q, base + q, sm, tol1, tol2);

    const int nrot = sm.flags[0];
    if (nrot > 0) {
        // ---- fold tiny scales, store the columns, scales and tracked norms
        if (tid < W2 && sm.gidx[tid] >= 0 && sm.d[tid] < fold_min) {
            sm.fold[tid] = sm.d[tid];
            sm.d[tid] = T(1);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = sm.gidx[c];
            if (gc < 0) continue;
            const T f = sm.fold[c];
            T* col = X + (size_t)gc * D.ldX;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = tid + k * nthr;
                if (r < D.mX) col[r] = (f == T(1)) ? x[k][c] : x[k][c] * f;
            }
        }
        if (tid < W2 && sm.gidx[tid] >= 0) {
            dsc[sm.gidx[tid]] = sm.d[tid];
            alph[sm.gidx[tid]] = sm.alpha[tid];
        }
    } else if (fresh) {
        // no rotation: only the recomputed norms change
        if (tid < W2 && sm.gidx[tid] >= 0) alph[sm.gidx[tid]] = sm.alpha[tid];
    }
    __syncthreads();
    return nrot;
}

// Replay the rotation table of the last jacobi_visit_x (first: it had intra rounds) on the
// rows of V, RPT rows per thread at a time: all loads of a pass are issued before the
// first is used (one L2 round trip per pass instead of one per row). Ends synchronized.
template <typename T, int W, int RPT>
__device__ void replay_v(const SweepDims& D, double* V, bool first, const VisitShared<T, W>& sm)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int W2 = 2 * W;
    for (int r0 = tid; r0 < D.nV; r0 += RPT * nthr) {
        double v[RPT][W2];
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = sm.gidx[c];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = r0 + k * nthr;
                v[k][c] = (gc >= 0 && r < D.nV) ? __ldcg(V + cm(r, gc, D.ldV)) : 0.0;
            }
        }
        replay_rows<W, RPT, T>(v, first, sm);
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = sm.gidx[c];
            if (gc < 0) continue;
            const double f = (double)sm.fold[c];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = r0 + k * nthr;
                if (r < D.nV) V[cm(r, gc, D.ldV)] = (f == 1.0) ? v[k][c] : v[k][c] * f;
            }
        }
    }
    __syncthreads();
}

// One whole visit: X part, then (with V and at least one rotation) the replay on V.
template <typename T, bool WITH_V, int W, int RPT>
__device__ int jacobi_visit(const SweepDims& D, T* X, double* V, int bi, int bj, bool first,
                            VisitShared<T, W>& sm)
{
    const int nrot = jacobi_visit_x<T, WITH_V, W, RPT>(D, X, bi, bj, first, sm);
    if (WITH_V && nrot > 0) replay_v<T, W, RPT>(D, V, first, sm);
    return nrot;
}

// Full Alg. 1 iteration on X (and V) by a group of CTAs: sweeps of k-1 rounds until a sweep
// performs no rotation or maxsweep sweeps ran. rot_sweep (global, zeroed, >= maxsweep
// entries) accumulates the rotations of each sweep. D.dsc must hold 1 and D.alph anything
// (round 0 recomputes it). Returns the number of sweeps run, or -1 if a barrier failed;
// *converged tells whether the last sweep rotated nothing.
// The stopping rule of MPJSVD_STOP_XGESVJ after sweep `sweep` (not the first) with rotations:
// every rotation of the sweep was negligible (largest cosine among the rotated pairs below
// sqrt(n) tol, and n times it times the largest |tan| below tol). Reads the sweep's maxima
// after the barrier that ends it, so every CTA takes the same decision.
__device__ __forceinline__ bool negligible_sweep(const SweepDims& D, const unsigned* mxc, const unsigned* mxt,
                                                 int sweep)
{
    if (D.stop != 0 || sweep == 0) return false;
    const double cmax = (double)__uint_as_float(__ldcg(mxc + sweep));
    const double tmax = (double)__uint_as_float(__ldcg(mxt + sweep));
    return cmax < sqrt((double)D.n) * D.tol && (double)D.n * cmax * tmax < D.tol;
}

template <typename T, bool WITH_V, int W, int RPT>
__device__ int jacobi_sweeps(const Group& g, const SweepDims& D, T* X, double* V,
                             unsigned long long* rot_sweep, unsigned* mxc, unsigned* mxt,
                             VisitShared<T, W>& sm, bool* converged)
{
    const int k = D.k;
    int sweep = 0;
    *converged = false;
    for (; sweep < D.maxsweep; ++sweep) {
        for (int r = 0; r < k - 1; ++r) {
            unsigned long long local = 0;
            for (int v = g.rank; v < k / 2; v += g.size) {
                int bi, bj;
                rr_pair(k, r, v, bi, bj);
                if (bi > bj) { int t = bi; bi = bj; bj = t; }
                const int nr = jacobi_visit<T, WITH_V, W, RPT>(D, X, V, bi, bj, r == 0, sm);
                local += (unsigned long long)nr;
                if (threadIdx.x == 0 && nr) {
                    atomicMax(mxc + sweep, sm.mxc);
                    atomicMax(mxt + sweep, sm.mxt);
                }
            }
            if (threadIdx.x == 0 && local) atomicAdd(&rot_sweep[sweep], local);
            if (!g.sync()) return -1;
        }
        unsigned long long total = __ldcg(&rot_sweep[sweep]);
        if (total == 0 || negligible_sweep(D, mxc, mxt, sweep)) {
            *converged = true;
            ++sweep;
            break;
        }
    }
    return sweep;
}

// Thread 0 waits (bounded) until blocks bi and bj have version >= R; false for every thread
// if the wait gave up (MPJSVD_STATUS_TIMEOUT recorded) or the call failed elsewhere.
__device__ __forceinline__ bool wait_blocks(const unsigned* ver, int bi, int bj, unsigned R, DevState* st)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
        unsigned spins = 0;
        // tight acquire spin (the wait is usually a few microseconds), time-bounded
        while (ld_acquire_u32(ver + bi) < R || ld_acquire_u32(ver + bj) < R) {
            if ((++spins & 255u) == 0) {
                if (call_failed(st)) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > lim) {
                    atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// jacobi_sweeps for a cooperative group of CTAs, scheduled by block versions instead of a
// barrier per round. ver: 2k zeroed counters (X versions, then V versions). The visits of a sweep are numbered round-major
// (f = r * k/2 + i) and CTA c takes f = c, c + G, ...: every visit waits only on visits with
// smaller numbers, so the smallest unfinished one can always run (all CTAs are resident).
template <typename T, bool WITH_V, int W, int RPT>
__device__ int jacobi_sweeps_flow(const Group& g, const SweepDims& D, T* X, double* V,
                                  unsigned long long* rot_sweep, unsigned* mxc, unsigned* mxt,
                                  unsigned* ver, VisitShared<T, W>& sm, bool* converged)
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
            if (bi > bj) { int t = bi; bi = bj; bj = t; }
            const unsigned R = (unsigned)(sweep * rounds + r);
            if (!wait_blocks(ver, bi, bj, R, g.st)) return -1;
            const int nrot = jacobi_visit_x<T, WITH_V, W, RPT>(D, X, bi, bj, r == 0, sm);
            // jacobi_visit_x ends with a CTA barrier: every store of X precedes the release,
            // so the next round's visits of bi and bj can start while this CTA updates V
            if (threadIdx.x == 0) {
                if (nrot) {
                    atomicAdd(&rot_sweep[sweep], (unsigned long long)nrot);
                    atomicMax(mxc + sweep, sm.mxc);
                    atomicMax(mxt + sweep, sm.mxt);
                }
                __threadfence();
                st_release_u32(ver + bi, R + 1);
                st_release_u32(ver + bj, R + 1);
            }
            if (WITH_V) {
                // V has its own versions (ver + k): replays of a block stay in round order
                unsigned* vv = ver + k;
                if (!wait_blocks(vv, bi, bj, R, g.st)) return -1;
                if (nrot > 0) replay_v<T, W, RPT>(D, V, r == 0, sm);
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release_u32(vv + bi, R + 1);
                    st_release_u32(vv + bj, R + 1);
                }
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

// x[:, j] *= dsc[j], dsc[j] = 1 for every column (end of a sweep stage), optionally V too.
template <typename T>
__device__ __forceinline__ void fold_scales_cols(const Group& g, int rows, int ncols, T* X, int ldX,
                                                 int nV, double* V, int ldV, T* dsc)
{
    for (int j = g.rank; j < ncols; j += g.size) {
        const T d = dsc[j];
        if (d != T(1)) {
            T* col = X + (size_t)j * ldX;
            for (int i = threadIdx.x; i < rows; i += blockDim.x) col[i] *= d;
            if (V) {
                double* vc = V + (size_t)j * ldV;
                for (int i = threadIdx.x; i < nV; i += blockDim.x) vc[i] *= (double)d;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) dsc[j] = T(1);
    }
}

}  // namespace mpj
