// sweep.cuh -- one-sided Jacobi sweeps (Alg. 1 of the paper, Section 2.1) over a parallel
// round-robin ordering of column blocks.
//
// Ordering. The n columns are cut into k blocks of w columns (k even; a phantom block
// pads odd counts). A sweep is k-1 rounds of the circle-method tournament; in round r the
// k/2 block pairs are disjoint, so their visits run concurrently on different CTAs. A
// visit of blocks (I, J) rotates every cross pair (i in I, j in J) once (w inner rounds of
// w disjoint pairs); in round 0 it also rotates the pairs inside I and inside J. Over a
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
// Data. The visit's 2w columns of X live in shared memory (column-major). The rotations
// are recorded in order; V's rows are then streamed through shared memory in chunks and
// each thread replays the whole record on one row (rows of V are independent).
#pragma once

#include "common.cuh"

namespace mpj {

// Circle-method round-robin: block k-1 is fixed, the others rotate. Pairs (a, b) of round
// r for i = 0 .. k/2-1 are disjoint, and over r = 0 .. k-2 every pair of blocks meets once.
__device__ __forceinline__ void rr_pair(int k, int r, int i, int& a, int& b)
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
    int w;       // block width (<= WMAX)
    int k;       // number of blocks (even)
    int maxsweep;
    double tol;  // rotation threshold
};

// Shared-memory layout of a visit (sizes in elements; the host computes the byte size
// with sweep_smem_bytes()).
template <typename T, int WMAX>
struct VisitSmem {
    static constexpr int kVChunkRows = 256;
    static constexpr int kMaxTeamWarps = 32;
    T* Xs;          // [2*w][ldsm]
    double* Vs;     // [kVChunkRows][2*w+1]
    T* gpart;       // [WMAX][kMaxTeamWarps]
    T* alpha;       // [2*WMAX]
    T* d;           // [2*WMAX]
    T* tab;         // [WMAX] per pair of the current inner round
    T* tba;         // [WMAX]
    double* rec_t;  // [2*WMAX*WMAX][2] recorded (t_ab, t_ba)
    unsigned char* rec_ab;  // [2*WMAX*WMAX][2]
    int* gidx;      // [2*WMAX] global column or -1
    int* flags;     // [0]: rotations in this visit; [1]: record length; [2]: dirty count
    int* active;    // [WMAX]
    int* dirty;     // [2*WMAX]
    int ldsm;       // column stride of Xs
    int ldv;        // row stride of Vs (2w + 1: conflict-free 8-byte accesses)
};

__host__ __device__ inline int sweep_ldsm(int mX) { return (mX + 3) & ~3; }

// Sizes depend on the runtime block width w (<= WMAX) for the big tiles.
template <typename T, int WMAX>
__host__ __device__ inline size_t sweep_smem_bytes(int mX, int w, bool with_v)
{
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 15) & ~size_t(15); };
    add(sizeof(T) * 2 * w * (size_t)sweep_ldsm(mX));
    if (with_v) add(sizeof(double) * VisitSmem<T, WMAX>::kVChunkRows * (2 * w + 1));
    add(sizeof(T) * WMAX * VisitSmem<T, WMAX>::kMaxTeamWarps);
    add(sizeof(T) * 2 * WMAX);
    add(sizeof(T) * 2 * WMAX);
    add(sizeof(T) * WMAX);
    add(sizeof(T) * WMAX);
    if (with_v) add(sizeof(double) * 2 * WMAX * WMAX * 2);
    if (with_v) add(2 * 2 * WMAX * WMAX);
    add(sizeof(int) * 2 * WMAX);
    add(sizeof(int) * 4);
    add(sizeof(int) * WMAX);
    add(sizeof(int) * 2 * WMAX);
    return b;
}

template <typename T, int WMAX>
__device__ inline VisitSmem<T, WMAX> carve_visit_smem(unsigned char* base, int mX, int w, bool with_v)
{
    VisitSmem<T, WMAX> s;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    s.ldsm = sweep_ldsm(mX);
    s.ldv = 2 * w + 1;
    s.Xs = (T*)take(sizeof(T) * 2 * w * (size_t)s.ldsm);
    s.Vs = with_v ? (double*)take(sizeof(double) * VisitSmem<T, WMAX>::kVChunkRows * (2 * w + 1)) : nullptr;
    s.gpart = (T*)take(sizeof(T) * WMAX * VisitSmem<T, WMAX>::kMaxTeamWarps);
    s.alpha = (T*)take(sizeof(T) * 2 * WMAX);
    s.d = (T*)take(sizeof(T) * 2 * WMAX);
    s.tab = (T*)take(sizeof(T) * WMAX);
    s.tba = (T*)take(sizeof(T) * WMAX);
    s.rec_t = with_v ? (double*)take(sizeof(double) * 2 * WMAX * WMAX * 2) : nullptr;
    s.rec_ab = with_v ? (unsigned char*)take(2 * 2 * WMAX * WMAX) : nullptr;
    s.gidx = (int*)take(sizeof(int) * 2 * WMAX);
    s.flags = (int*)take(sizeof(int) * 4);
    s.active = (int*)take(sizeof(int) * WMAX);
    s.dirty = (int*)take(sizeof(int) * 2 * WMAX);
    return s;
}

// Local columns of inner round q. Cross rounds (intra = false): pair i = (i, w + (i+q) % w).
// Intra rounds (intra = true, round-robin inside each block, w even): pairs 0..w/2-1 inside
// block I, pairs w/2..w-1 inside block J.
__device__ __forceinline__ void inner_pair(bool intra, int w, int q, int i, int& a, int& b)
{
    if (!intra) {
        a = i;
        b = w + (i + q) % w;
        return;
    }
    int half = w >> 1;
    int base = (i < half) ? 0 : w;
    int ii = (i < half) ? i : i - half;
    int pa, pb;
    rr_pair(w, q, ii, pa, pb);
    a = base + pa;
    b = base + pb;
}

// One visit of block pair (bi, bj): load, rotate, store. Returns the rotation count
// (meaningful in thread 0). All threads of the CTA must call it.
template <typename T, bool WITH_V, int WMAX>
__device__ int jacobi_visit(const SweepDims& D, T* X, double* V, int bi, int bj, bool first,
                            const VisitSmem<T, WMAX>& sm)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = nthr >> 5;
    const int w = D.w, w2 = 2 * w, mX = D.mX, ldsm = sm.ldsm;
    const T tol = T(D.tol);

    // ---- columns of the visit
    if (tid < w2) {
        int blk = (tid < w) ? bi : bj;
        int c = blk * w + (tid < w ? tid : tid - w);
        bool ok = (blk * w < D.n) && (c < D.n);
        sm.gidx[tid] = ok ? c : -1;
        sm.d[tid] = T(1);
        sm.dirty[tid] = 0;
    }
    if (tid == 0) {
        sm.flags[0] = 0;
        sm.flags[1] = 0;
        sm.flags[2] = 0;
    }
    __syncthreads();

    // ---- load X columns (through L2: other CTAs wrote them in earlier rounds)
    for (int c = 0; c < w2; ++c) {
        int gc = sm.gidx[c];
        T* dst = sm.Xs + (size_t)c * ldsm;
        if (gc < 0) continue;
        const T* src = X + cm(0, gc, D.ldX);
        for (int i = tid; i < mX; i += nthr) dst[i] = __ldcg(src + i);
    }
    __syncthreads();

    // ---- fresh squared norms
    for (int c = wid; c < w2; c += nwarps) {
        T s = T(0);
        if (sm.gidx[c] >= 0) {
            const T* col = sm.Xs + (size_t)c * ldsm;
            for (int i = lane; i < mX; i += 32) s = fma(col[i], col[i], s);
            s = warp_sum(s);
        }
        if (lane == 0) sm.alpha[c] = s;
    }
    __syncthreads();

    // ---- inner rounds
    const int nintra = first ? (w - 1) : 0;
    const int nrounds = nintra + w;
    const int npairs = w;  // pairs per inner round
    // teams of warps per pair
    const int team_warps = max(1, nwarps / npairs);
    const int nteams = nwarps / team_warps;
    const int team = wid / team_warps;
    const int wit = wid % team_warps;  // warp index in team
    const int team_lane = wit * 32 + lane;
    const int team_thr = team_warps * 32;

    for (int q = 0; q < nrounds; ++q) {
        const bool intra = q < nintra;
        const int qq = intra ? q : q - nintra;
        if (intra && w < 2) continue;
        // phase A: partial dot products
        for (int pp = team; pp < npairs && team < nteams; pp += nteams) {
            int a, b;
            inner_pair(intra, w, qq, pp, a, b);
            T s = T(0);
            if (sm.gidx[a] >= 0 && sm.gidx[b] >= 0) {
                const T* xa = sm.Xs + (size_t)a * ldsm;
                const T* xb = sm.Xs + (size_t)b * ldsm;
                for (int i = team_lane; i < mX; i += team_thr) s = fma(xa[i], xb[i], s);
            }
            s = warp_sum(s);
            if (lane == 0) sm.gpart[pp * VisitSmem<T, WMAX>::kMaxTeamWarps + wit] = s;
        }
        __syncthreads();
        // phase B: rotation parameters, one thread per pair
        if (tid < npairs) {
            int a, b;
            inner_pair(intra, w, qq, tid, a, b);
            int act = 0;
            if (sm.gidx[a] >= 0 && sm.gidx[b] >= 0) {
                T gh = T(0);
                for (int k2 = 0; k2 < team_warps; ++k2) gh += sm.gpart[tid * VisitSmem<T, WMAX>::kMaxTeamWarps + k2];
                T da = sm.d[a], db = sm.d[b];
                T gamma = gh * da * db;
                T al = sm.alpha[a], be = sm.alpha[b];
                if (fabs(gamma) > tol * sqrt(al) * sqrt(be)) {
                    T t = rot_tangent(al, be, gamma);
                    T c = T(1) / sqrt(T(1) + t * t);
                    T tab = t * (db / da), tba = t * (da / db);
                    sm.tab[tid] = tab;
                    sm.tba[tid] = tba;
                    sm.d[a] = da * c;
                    sm.d[b] = db * c;
                    T na = al - t * gamma, nb = be + t * gamma;
                    // severe cancellation in the tracked norm: recompute it from the data
                    if (na < T(0.0625) * al) { sm.dirty[a] = 1; atomicAdd(&sm.flags[2], 1); }
                    if (nb < T(0.0625) * be) { sm.dirty[b] = 1; atomicAdd(&sm.flags[2], 1); }
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
            sm.active[tid] = act;
        }
        __syncthreads();
        // phase C: apply the rotations to the X columns
        for (int pp = team; pp < npairs && team < nteams; pp += nteams) {
            if (!sm.active[pp]) continue;
            int a, b;
            inner_pair(intra, w, qq, pp, a, b);
            T* xa = sm.Xs + (size_t)a * ldsm;
            T* xb = sm.Xs + (size_t)b * ldsm;
            T tab = sm.tab[pp], tba = sm.tba[pp];
            for (int i = team_lane; i < mX; i += team_thr) {
                T ya = xa[i], yb = xb[i];
                xa[i] = fma(-tab, yb, ya);
                xb[i] = fma(tba, ya, yb);
            }
        }
        __syncthreads();
        // recompute tracked norms that lost accuracy
        if (sm.flags[2] > 0) {
            for (int c = wid; c < w2; c += nwarps) {
                if (!sm.dirty[c]) continue;
                const T* col = sm.Xs + (size_t)c * ldsm;
                T s = T(0);
                for (int i = lane; i < mX; i += 32) s = fma(col[i], col[i], s);
                s = warp_sum(s);
                if (lane == 0) {
                    T dc = sm.d[c];
                    sm.alpha[c] = s * dc * dc;
                    sm.dirty[c] = 0;
                }
            }
            __syncthreads();
            if (tid == 0) sm.flags[2] = 0;
            __syncthreads();
        }
    }

    const int nrot = sm.flags[0];
    // ---- store X with the scales folded in
    if (nrot > 0) {
        for (int c = 0; c < w2; ++c) {
            int gc = sm.gidx[c];
            if (gc < 0) continue;
            const T* src = sm.Xs + (size_t)c * ldsm;
            T* dst = X + cm(0, gc, D.ldX);
            T dc = sm.d[c];
            for (int i = tid; i < mX; i += nthr) dst[i] = src[i] * dc;
        }
    }

    // ---- replay the rotations on the rows of V
    if (WITH_V && nrot > 0) {
        const int nrec = sm.flags[1];
        const int ldv = sm.ldv;
        constexpr int CH = VisitSmem<T, WMAX>::kVChunkRows;
        for (int r0 = 0; r0 < D.nV; r0 += CH) {
            int rows = min(CH, D.nV - r0);
            __syncthreads();
            for (int c = 0; c < w2; ++c) {
                int gc = sm.gidx[c];
                if (gc < 0) continue;
                const double* src = V + cm(r0, gc, D.ldV);
                for (int i = tid; i < rows; i += nthr) sm.Vs[i * ldv + c] = __ldcg(src + i);
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
            for (int c = 0; c < w2; ++c) {
                int gc = sm.gidx[c];
                if (gc < 0) continue;
                double dc = (double)sm.d[c];
                double* dst = V + cm(r0, gc, D.ldV);
                for (int i = tid; i < rows; i += nthr) dst[i] = sm.Vs[i * ldv + c] * dc;
            }
        }
    }
    __syncthreads();
    return nrot;
}

// Full Alg. 1 iteration on X (and V) by a group of CTAs: sweeps of k-1 rounds until a sweep
// performs no rotation or maxsweep sweeps ran. rot_sweep (global, zeroed, >= maxsweep
// entries) accumulates the rotations of each sweep. Returns the number of sweeps run
// (> maxsweep - 1 and last count nonzero means not converged), or -1 if a barrier failed.
template <typename T, bool WITH_V, int WMAX>
__device__ int jacobi_sweeps(const Group& g, const SweepDims& D, T* X, double* V,
                             unsigned long long* rot_sweep, const VisitSmem<T, WMAX>& sm,
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
                local += (unsigned long long)jacobi_visit<T, WITH_V, WMAX>(D, X, V, bi, bj, r == 0, sm);
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
