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
// alpha' = alpha - t gamma, beta' = beta + t gamma.
//
// Scaled ("fast") form. Inside a visit each column is kept as x = d * xh with a scale d
// (1 at the start of the visit). The update becomes xh_p -= (t d_q / d_p) xh_q,
// xh_q += (t d_p / d_q) xh_p, d_p *= c, d_q *= c: two FMAs per row instead of two
// multiplies and two FMAs. The scales are folded back into the columns when the visit
// stores them. V (when accumulated) shares the same scales and receives the same updates.
//
// Execution. The visit's 2W columns of X live in shared memory (column-major), loaded and
// stored with batched vector accesses. In an inner round every thread works on all W pairs
// over its own rows; the W partial dot products are combined with one multi-value warp
// reduction (W - 1 + 5 - log2 W additions per lane instead of 5 W) and W lanes of warp 0
// compute the W rotations together. The rotations are recorded in order; V's rows are then
// streamed through shared memory in chunks and each thread replays the whole record on
// one row (rows are independent).
#pragma once

#include "common.cuh"

namespace mpj {

// Circle-method round-robin: block k-1 is fixed, the others rotate. Pairs (a, b) of round
// r for i = 0 .. k/2-1 are disjoint, and over r = 0 .. k-2 every pair of blocks meets once.
__host__ __device__ __forceinline__ void rr_pair(int k, int r, int i, int& a, int& b)
{
    if (i == 0) {
        a = k - 1;
        b = r;
    } else {
        a = (r + i) % (k - 1);
        b = (r - i + (k - 1)) % (k - 1);
    }
}

template <typename T>
__device__ __forceinline__ T rot_tangent(T alpha, T beta, T gamma)
{
    T zeta = (beta - alpha) / (T(2) * gamma);
    T az = fabs(zeta);
    T big = sizeof(T) == 8 ? T(1e150) : T(1e18);
    T t = (az > big) ? T(1) / (T(2) * az) : T(1) / (az + sqrt(T(1) + az * az));
    return zeta >= T(0) ? t : -t;
}

struct SweepDims {
    int n;       // columns of X (and of V)
    int mX;      // rows of X
    int ldX;
    int nV;      // rows of V (0: no V)
    int ldV;
    int w;       // block width (== W of the kernel)
    int k;       // number of blocks (even)
    int maxsweep;
    double tol;  // rotation threshold
};

constexpr int kVChunkRows = 256;
constexpr int kMaxWarps = 32;

// Shared-memory layout of a visit for block width W.
template <typename T, int W>
struct VisitSmem {
    T* Xs;          // [2W][ldsm]
    double* Vs;     // [kVChunkRows][2W+1]
    T* part;        // [2W][kMaxWarps] per-warp partial sums
    T* alpha;       // [2W] tracked squared norms (true scale)
    T* d;           // [2W] scales of the scaled form
    T* dinv;        // [2W] their reciprocals (kept alongside: no division per rotation)
    T* tab;         // [W] rotation parameters of the current inner round
    T* tba;         // [W]
    double* rec_t;  // [2W*W][2] recorded (t_ab, t_ba)
    unsigned char* rec_ab;  // [2W*W][2]
    int* gidx;      // [2W] global column or -1
    int* flags;     // [0]: rotations in this visit; [1]: record length; [2]: dirty
    int* active;    // [W]
    int ldsm;       // column stride of Xs
    int ldv;        // row stride of Vs (2W + 1: conflict-free 8-byte accesses)
};

__host__ __device__ inline int sweep_ldsm(int mX) { return (mX + 3) & ~3; }

template <typename T, int W>
__host__ __device__ inline size_t sweep_smem_bytes(int mX, bool with_v)
{
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 15) & ~size_t(15); };
    add(sizeof(T) * 2 * W * (size_t)sweep_ldsm(mX));
    if (with_v) add(sizeof(double) * kVChunkRows * (2 * W + 1));
    add(sizeof(T) * 2 * W * kMaxWarps);
    add(sizeof(T) * 2 * W);
    add(sizeof(T) * 2 * W);
    add(sizeof(T) * 2 * W);
    add(sizeof(T) * W);
    add(sizeof(T) * W);
    if (with_v) add(sizeof(double) * 2 * W * W * 2);
    if (with_v) add(2 * 2 * W * W);
    add(sizeof(int) * 2 * W);
    add(sizeof(int) * 4);
    add(sizeof(int) * W);
    return b;
}

template <typename T, int W>
__device__ inline VisitSmem<T, W> carve_visit_smem(unsigned char* base, int mX, bool with_v)
{
    VisitSmem<T, W> s;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    s.ldsm = sweep_ldsm(mX);
    s.ldv = 2 * W + 1;
    s.Xs = (T*)take(sizeof(T) * 2 * W * (size_t)s.ldsm);
    s.Vs = with_v ? (double*)take(sizeof(double) * kVChunkRows * (2 * W + 1)) : nullptr;
    s.part = (T*)take(sizeof(T) * 2 * W * kMaxWarps);
    s.alpha = (T*)take(sizeof(T) * 2 * W);
    s.d = (T*)take(sizeof(T) * 2 * W);
    s.dinv = (T*)take(sizeof(T) * 2 * W);
    s.tab = (T*)take(sizeof(T) * W);
    s.tba = (T*)take(sizeof(T) * W);
    s.rec_t = with_v ? (double*)take(sizeof(double) * 2 * W * W * 2) : nullptr;
    s.rec_ab = with_v ? (unsigned char*)take(2 * 2 * W * W) : nullptr;
    s.gidx = (int*)take(sizeof(int) * 2 * W);
    s.flags = (int*)take(sizeof(int) * 4);
    s.active = (int*)take(sizeof(int) * W);
    return s;
}

// Local columns of inner round q. Cross rounds (intra = false): pair i = (i, W + (i+q) % W).
// Intra rounds (intra = true, round-robin inside each block, W even): pairs 0..W/2-1 inside
// block I, pairs W/2..W-1 inside block J.
template <int W>
__device__ __forceinline__ void inner_pair(bool intra, int q, int i, int& a, int& b)
{
    if (!intra) {
        a = i;
        b = W + (i + q) % W;
        return;
    }
    constexpr int half = W / 2;
    int base = (i < half) ? 0 : W;
    int ii = (i < half) ? i : i - half;
    int pa, pb;
    rr_pair(W, q, ii, pa, pb);
    a = base + pa;
    b = base + pb;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// Copy columns gidx[c] (c < ncols, rows 0..rows-1) of a global matrix into shared memory
// dst[c * ldsm + i] (or back with a per-column scale when STORE). Several independent
// accesses are issued per thread before their results are used. Reads go through L2
// (__ldcg): other CTAs wrote these columns in earlier rounds.
template <typename T, bool STORE>
__device__ __forceinline__ void copy_cols(T* g, int ld, T* sm, int ldsm, const int* gidx, int ncols,
                                          int rows, const T* scale)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    constexpr int U = 4;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool vec = (ld % VN == 0) && (rows % VN == 0) && ((((size_t)g) & 15) == 0);
    if (vec) {
        const int nv = rows / VN;
        const int total = ncols * nv;
        for (int base = tid; base < total; base += nthr * U) {
            V r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = base + u * nthr;
                if (e < total) {
                    int c = e / nv, v = e - c * nv;
                    int gc = gidx[c];
                    if (gc >= 0) {
                        if (STORE) r[u] = *(const V*)(sm + (size_t)c * ldsm + v * VN);
                        else r[u] = __ldcg((const V*)(g + (size_t)gc * ld) + v);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = base + u * nthr;
                if (e < total) {
                    int c = e / nv, v = e - c * nv;
                    int gc = gidx[c];
                    if (gc >= 0) {
                        if (STORE) {
                            T s = scale[c];
                            V o = r[u];
                            if constexpr (VN == 2) { o.x *= s; o.y *= s; }
                            else { o.x *= s; o.y *= s; o.z *= s; o.w *= s; }
                            *((V*)(g + (size_t)gc * ld) + v) = o;
                        } else {
                            *(V*)(sm + (size_t)c * ldsm + v * VN) = r[u];
                        }
                    }
                }
            }
        }
    } else {
        const int total = ncols * rows;
        for (int base = tid; base < total; base += nthr * U) {
            T r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = base + u * nthr;
                if (e < total) {
                    int c = e / rows, i = e - c * rows;
                    int gc = gidx[c];
                    if (gc >= 0) r[u] = STORE ? sm[(size_t)c * ldsm + i] : __ldcg(g + (size_t)gc * ld + i);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = base + u * nthr;
                if (e < total) {
                    int c = e / rows, i = e - c * rows;
                    int gc = gidx[c];
                    if (gc >= 0) {
                        if (STORE) g[(size_t)gc * ld + i] = r[u] * scale[c];
                        else sm[(size_t)c * ldsm + i] = r[u];
                    }
                }
            }
        }
    }
}

// Squared norms of the 2W shared-memory columns (scaled data times d^2) into alpha.
// Ends with __syncthreads.
template <typename T, int W>
__device__ __forceinline__ void visit_norms(const VisitSmem<T, W>& sm, int mX)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = nthr >> 5;
    T acc[2 * W];
#pragma unroll
    for (int c = 0; c < 2 * W; ++c) acc[c] = T(0);
    for (int r = tid; r < mX; r += nthr) {
#pragma unroll
        for (int c = 0; c < 2 * W; ++c) {
            T x = sm.Xs[(size_t)c * sm.ldsm + r];
            acc[c] = fma(x, x, acc[c]);
        }
    }
    warp_reduce_multi<2 * W>(acc, lane);
    constexpr int sh = 5 - ilog2c(2 * W);
    if ((lane & ((1 << sh) - 1)) == 0) sm.part[(lane >> sh) * kMaxWarps + wid] = acc[0];
    __syncthreads();
    if (tid < 2 * W) {
        T s = T(0);
        for (int k2 = 0; k2 < nwarps; ++k2) s += sm.part[tid * kMaxWarps + k2];
        T dc = sm.d[tid];
        sm.alpha[tid] = (sm.gidx[tid] >= 0) ? s * dc * dc : T(0);
    }
    __syncthreads();
}

// One visit of block pair (bi, bj): load, rotate, store. Returns the rotation count (all
// threads). All threads of the CTA must call it.
template <typename T, bool WITH_V, int W>
__device__ int jacobi_visit(const SweepDims& D, T* X, double* V, int bi, int bj, bool first,
                            const VisitSmem<T, W>& sm)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = nthr >> 5;
    const int mX = D.mX, ldsm = sm.ldsm;
    const T tol = T(D.tol);
    constexpr int W2 = 2 * W;
    constexpr int SH = 5 - ilog2c(W);  // lanes per value after warp_reduce_multi<W>

    // ---- columns of the visit
    if (tid < W2) {
        int blk = (tid < W) ? bi : bj;
        int c = blk * W + (tid < W ? tid : tid - W);
        bool ok = (blk * W < D.n) && (c < D.n);
        sm.gidx[tid] = ok ? c : -1;
        sm.d[tid] = T(1);
        sm.dinv[tid] = T(1);
    }
    if (tid == 0) {
        sm.flags[0] = 0;
        sm.flags[1] = 0;
        sm.flags[2] = 0;
    }
    __syncthreads();
    copy_cols<T, false>(X, D.ldX, sm.Xs, ldsm, sm.gidx, W2, mX, nullptr);
    __syncthreads();
    visit_norms<T, W>(sm, mX);

    const int nintra = first ? (W - 1) : 0;
    const int nrounds = nintra + W;
    for (int q = 0; q < nrounds; ++q) {
        const bool intra = q < nintra;
        const int qq = intra ? q : q - nintra;
        // phase A: partial dot products of all W pairs over this thread's rows
        T acc[W];
#pragma unroll
        for (int p = 0; p < W; ++p) acc[p] = T(0);
        for (int r = tid; r < mX; r += nthr) {
#pragma unroll
            for (int p = 0; p < W; ++p) {
                int a, b;
                inner_pair<W>(intra, qq, p, a, b);
                acc[p] = fma(sm.Xs[(size_t)a * ldsm + r], sm.Xs[(size_t)b * ldsm + r], acc[p]);
            }
        }
        warp_reduce_multi<W>(acc, lane);
        if ((lane & ((1 << SH) - 1)) == 0) sm.part[(lane >> SH) * kMaxWarps + wid] = acc[0];
        __syncthreads();
        // phase B: rotation parameters, lane p of warp 0 for pair p
        if (tid < W) {
            const int p = tid;
            int a, b;
            inner_pair<W>(intra, qq, p, a, b);
            int act = 0;
            if (sm.gidx[a] >= 0 && sm.gidx[b] >= 0) {
                T gh = T(0);
                for (int k2 = 0; k2 < nwarps; ++k2) gh += sm.part[p * kMaxWarps + k2];
                T da = sm.d[a], db = sm.d[b];
                T gamma = gh * da * db;
                T al = sm.alpha[a], be = sm.alpha[b];
                if (gamma * gamma > tol * tol * al * be) {  // |gamma| > tol |x_a| |x_b|
                    T t = rot_tangent(al, be, gamma);
                    T q1 = T(1) + t * t;
                    T c = rsqrt(q1);      // cos of the rotation
                    T ic = q1 * c;        // 1 / c
                    T ia = sm.dinv[a], ib = sm.dinv[b];
                    T tab = t * db * ia, tba = t * da * ib;
                    sm.tab[p] = tab;
                    sm.tba[p] = tba;
                    sm.d[a] = da * c;
                    sm.d[b] = db * c;
                    sm.dinv[a] = ia * ic;
                    sm.dinv[b] = ib * ic;
                    T na = al - t * gamma, nb = be + t * gamma;
                    // severe cancellation in a tracked norm: recompute the norms after this round
                    if (na < T(0.0625) * al || nb < T(0.0625) * be) sm.flags[2] = 1;
                    sm.alpha[a] = na;
                    sm.alpha[b] = nb;
                    act = 1;
                    atomicAdd(&sm.flags[0], 1);
                    if (WITH_V) {
                        int slot = atomicAdd(&sm.flags[1], 1);
                        sm.rec_t[2 * slot] = (double)tab;
                        sm.rec_t[2 * slot + 1] = (double)tba;
                        sm.rec_ab[2 * slot] = (unsigned char)a;
                        sm.rec_ab[2 * slot + 1] = (unsigned char)b;
                    }
                }
            }
            sm.active[p] = act;
        }
        __syncthreads();
        // phase C: apply the active rotations to this thread's rows
        int actm = 0;
        T tab[W], tba[W];
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (sm.active[p]) actm |= 1 << p;
            tab[p] = sm.tab[p];
            tba[p] = sm.tba[p];
        }
        if (actm) {
            for (int r = tid; r < mX; r += nthr) {
#pragma unroll
                for (int p = 0; p < W; ++p) {
                    if (!(actm & (1 << p))) continue;
                    int a, b;
                    inner_pair<W>(intra, qq, p, a, b);
                    T* xa = sm.Xs + (size_t)a * ldsm + r;
                    T* xb = sm.Xs + (size_t)b * ldsm + r;
                    T ya = *xa, yb = *xb;
                    *xa = fma(-tab[p], yb, ya);
                    *xb = fma(tba[p], ya, yb);
                }
            }
        }
        __syncthreads();
        if (sm.flags[2]) {  // rare: a tracked norm lost its accuracy
            visit_norms<T, W>(sm, mX);
            if (tid == 0) sm.flags[2] = 0;
            __syncthreads();
        }
    }

    const int nrot = sm.flags[0];
    // ---- store X with the scales folded in
    if (nrot > 0) copy_cols<T, true>(X, D.ldX, sm.Xs, ldsm, sm.gidx, W2, mX, sm.d);

    // ---- replay the rotations on the rows of V
    if (WITH_V && nrot > 0) {
        const int nrec = sm.flags[1];
        const int ldv = sm.ldv;
        for (int r0 = 0; r0 < D.nV; r0 += kVChunkRows) {
            const int rows = min(kVChunkRows, D.nV - r0);
            __syncthreads();
            for (int i = tid; i < rows; i += nthr) {
                double r[W2];
#pragma unroll
                for (int c = 0; c < W2; ++c)
                    if (sm.gidx[c] >= 0) r[c] = __ldcg(V + cm(r0 + i, sm.gidx[c], D.ldV));
#pragma unroll
                for (int c = 0; c < W2; ++c)
                    if (sm.gidx[c] >= 0) sm.Vs[i * ldv + c] = r[c];
            }
            __syncthreads();
            for (int i = tid; i < rows; i += nthr) {
                double* row = sm.Vs + i * ldv;
                for (int e = 0; e < nrec; ++e) {
                    int a = sm.rec_ab[2 * e], b = sm.rec_ab[2 * e + 1];
                    double ta = sm.rec_t[2 * e], tb = sm.rec_t[2 * e + 1];
                    double va = row[a], vb = row[b];
                    row[a] = fma(-ta, vb, va);
                    row[b] = fma(tb, va, vb);
                }
            }
            __syncthreads();
            for (int i = tid; i < rows; i += nthr) {
#pragma unroll
                for (int c = 0; c < W2; ++c)
                    if (sm.gidx[c] >= 0)
                        V[cm(r0 + i, sm.gidx[c], D.ldV)] = sm.Vs[i * ldv + c] * (double)sm.d[c];
            }
        }
    }
    __syncthreads();
    return nrot;
}

// Full Alg. 1 iteration on X (and V) by a group of CTAs: sweeps of k-1 rounds until a sweep
// performs no rotation or maxsweep sweeps ran. rot_sweep (global, zeroed, >= maxsweep
// entries) accumulates the rotations of each sweep. Returns the number of sweeps run, or
// -1 if a barrier failed; *converged tells whether the last sweep rotated nothing.
template <typename T, bool WITH_V, int W>
__device__ int jacobi_sweeps(const Group& g, const SweepDims& D, T* X, double* V,
                             unsigned long long* rot_sweep, const VisitSmem<T, W>& sm,
                             bool* converged)
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
                local += (unsigned long long)jacobi_visit<T, WITH_V, W>(D, X, V, bi, bj, r == 0, sm);
            }
            if (threadIdx.x == 0 && local) atomicAdd(&rot_sweep[sweep], local);
            if (!g.sync()) return -1;
        }
        unsigned long long total = __ldcg(&rot_sweep[sweep]);
        if (total == 0) {
            *converged = true;
            ++sweep;
            break;
        }
    }
    return sweep;
}

}  // namespace mpj
