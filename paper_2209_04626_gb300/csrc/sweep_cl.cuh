// sweep_cl.cuh -- binary64 sweeps of Alg. 1 (Section 2.1) for tall matrices: every visit of a
// block pair is split by rows over a thread-block cluster of CS CTAs.
//
// The register-resident visit of sweep.cuh keeps the 2W columns of a block pair in one CTA's
// registers, so for tall matrices (8192 rows) only W = 1 fits: every round then loads and
// stores each column of Y and V, and the FP64 work of a visit (one pair) is separated by the
// latencies of the loads and of the reduction and rotation-parameter chain. Here CTA r of a
// cluster holds rows [r rpc, (r + 1) rpc) of the 2W columns (rpc = ceil(mX / CS)), so W = 4
// fits at 8192 rows (CS = 8: 1024 rows and 128 threads per CTA, two CTAs of different visits
// per SM) and each CTA runs the work of the W = 4 visit on a 1024-row matrix. Per inner round,
// each CTA reduces its partial dot products, writes them into every CTA's shared memory
// (distributed shared memory) and passes one cluster barrier; then every CTA sums the CS
// partials in rank order and computes the same rotations (the same bits: same operands, same
// order), so all CTAs of a cluster take the same decisions without further exchange. V's rows
// are split over the cluster the same way.
//
// Late sweeps. Once a sweep's largest rotated cosine is below kClBatchCos, the next sweep's
// rotations are of the order of its square and almost no visit rotates: each visit then
// computes the dot products of all its pairs at once and passes a single cluster exchange
// (cl_batch_quiet); only a visit with a pair to rotate runs the inner rounds.
//
// Uniform control flow. A cluster barrier waits for every CTA of the cluster, without a time
// limit, so no CTA may leave while another waits at one. Every decision that reads state other
// CTAs write (the bounded waits on block versions, the grid barrier, the failure flag, the
// convergence test) is taken by each CTA and then agreed on through one exchange and barrier
// (cl_agree): all CTAs continue, or all return. Everything else is computed from identical
// data in identical order.
//
// Scheduling is that of jacobi_sweeps_flow: per-block version counters (acquired by every CTA
// of the cluster for itself), released by rank 0 after a cluster barrier that follows every
// rank's stores; one grid barrier per sweep for the convergence test.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"

namespace cg = cooperative_groups;

namespace mpj {

// Block widths W in {2, 4, 8}: each thread holds RPT = 32 / W rows of the 2W columns (64
// doubles in registers), at most kClMaxThreads threads per CTA.
constexpr int kClMaxThreads = 256;
__host__ __device__ constexpr int cl_rpt(int w) { return 32 / w; }
__host__ __device__ constexpr int cl_rows_per_cta(int w) { return cl_rpt(w) * kClMaxThreads; }

// The batched test of a visit (sweeps whose rotations have become rare): the values it reduces,
// in this order: the 2W squared norms and the W (W - 1) intra-block pairs (first round of a
// sweep only), then the W^2 cross pairs, each pair as the sequential inner rounds take it.
template <int W>
struct ClBatch {
    static constexpr int NI = (W - 1) * W;
    static constexpr int NC = W * W;
    static constexpr int NF = 2 * W + NI + NC;
};
// A sweep takes the batched test when the previous one rotated no pair with a cosine above
// this (the next sweep's rotations are then of the order of its square: almost no visit
// rotates).
constexpr float kClBatchCos = 1e-6f;

template <int W, int CS>
struct ClShared {
    VisitShared<double, W> v;   // the visit's state: identical in every CTA of the cluster
    double xch[2][CS][2 * W];   // partial sums of each rank (double-buffered by exchange parity)
    int agree[2][CS][2];        // per rank: ok flag, rank 0's value (parity-buffered)
    double bpart[ClBatch<W>::NF][kClMaxThreads / 32];  // batched test: per-warp partial sums
    double xchb[2][CS][ClBatch<W>::NF];                // batched test: each rank's partial sums
    int brot;                                           // batched test: pairs that would rotate
};

// Parities of the two exchange buffers. Every CTA of a cluster runs the same sequence of
// exchanges, so the parities agree; two uses of one buffer are separated by a cluster barrier
// that every CTA reaches only after reading the earlier use.
struct ClPar {
    int x = 0;
    int a = 0;
    int b = 0;
};

// Every CTA contributes ok; afterwards every thread of every CTA of the cluster holds the AND
// of all, and *lead the value rank 0 contributed. One cluster barrier.
template <int W, int CS>
__device__ __forceinline__ bool cl_agree(const cg::cluster_group& cl, ClShared<W, CS>& sm, ClPar& par, int rank,
                                         bool ok, int lead_val, int* lead)
{
    if (threadIdx.x == 0) {
#pragma unroll
        for (int rr = 0; rr < CS; ++rr) {
            int* p = cl.map_shared_rank(&sm.agree[par.a][rank][0], rr);
            p[0] = ok ? 1 : 0;
            p[1] = lead_val;
        }
    }
    cl.sync();
    bool all = true;
#pragma unroll
    for (int rr = 0; rr < CS; ++rr) all = all && (sm.agree[par.a][rr][0] != 0);
    if (lead) *lead = sm.agree[par.a][0][1];
    par.a ^= 1;
    return all;
}

// Warp 0's lanes i < N write their CTA's partial sum of value i (the sum over the CTA's warps
// of sm.v.part[i][*]) into every rank's exchange buffer; ends with the cluster barrier. Call
// after a CTA barrier that follows the writes of part.
template <int N, int W, int CS>
__device__ __forceinline__ void cl_exchange(const cg::cluster_group& cl, ClShared<W, CS>& sm, int xp, int rank,
                                            int nw)
{
    if (threadIdx.x < N) {
        const double s = short_sum(sm.v.part[threadIdx.x], nw);
#pragma unroll
        for (int rr = 0; rr < CS; ++rr) *cl.map_shared_rank(&sm.xch[xp][rank][threadIdx.x], rr) = s;
    }
    cl.sync();
}

// The cluster-wide total of value i (ranks summed in order: the same bits in every CTA).
template <int W, int CS>
__device__ __forceinline__ double cl_sum(const ClShared<W, CS>& sm, int xp, int i)
{
    double s = sm.xch[xp][0][i];
#pragma unroll
    for (int rr = 1; rr < CS; ++rr) s += sm.xch[xp][rr][i];
    return s;
}

// Row range of this CTA and the rows of this thread: r = lo + tid + k T for k < RPT, r < hi.
struct ClRows {
    int lo, hi;
};

// Squared norms of the 2W columns over the whole cluster into sm.v.alpha. Ends synchronized.
template <int W, int RPT, int CS>
__device__ __forceinline__ void cl_norms(const cg::cluster_group& cl, const double (&x)[RPT][2 * W],
                                         ClShared<W, CS>& sm, ClPar& par, int rank)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    double acc[2 * W];
#pragma unroll
    for (int c = 0; c < 2 * W; ++c) {
        acc[c] = 0.0;
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[c] = fma(x[k][c], x[k][c], acc[c]);
    }
    warp_reduce_multi<2 * W>(acc, lane);
    constexpr int sh = 5 - ilog2c(2 * W);
    if ((lane & ((1 << sh) - 1)) == 0) sm.v.part[lane >> sh][wid] = acc[0];
    __syncthreads();
    cl_exchange<2 * W, W, CS>(cl, sm, par.x, rank, nw);
    if (tid < 2 * W) {
        const double s = cl_sum<W, CS>(sm, par.x, tid);
        const double dc = sm.v.d[tid];
        sm.v.alpha[tid] = (sm.v.gidx[tid] >= 0) ? s * dc * dc : 0.0;
    }
    par.x ^= 1;
    __syncthreads();
}

// One inner round on the cluster: as inner_round of sweep.cuh, with the dot products summed
// over the cluster before the rotation step.
template <int W, int RPT, int CS>
__device__ __forceinline__ void cl_inner_round(const cg::cluster_group& cl, double (&x)[RPT][2 * W], bool intra,
                                               int q, int slot, ClShared<W, CS>& sm, ClPar& par, int rank,
                                               double tol2)
{
    VisitShared<double, W>& s = sm.v;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    constexpr int SH = 5 - ilog2c(W);
    double acc[W];
#pragma unroll
    for (int p = 0; p < W; ++p) {
        const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
        acc[p] = 0.0;
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[p] = fma(x[k][a], x[k][b], acc[p]);
    }
    warp_reduce_multi<W>(acc, lane);
    if ((lane & ((1 << SH) - 1)) == 0) s.part[lane >> SH][wid] = acc[0];
    __syncthreads();
    cl_exchange<W, W, CS>(cl, sm, par.x, rank, nw);
    if (tid < W) {
        const int p = tid;
        const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
        unsigned act = 0;
        float cs = 0.0f, ta = 0.0f;
        if (s.gidx[a] >= 0 && s.gidx[b] >= 0 && (!s.cross_only || s.side[a] != s.side[b])) {
            const double gh = cl_sum<W, CS>(sm, par.x, p);
            const double da = s.d[a], db = s.d[b];
            const double ia = s.dinv[a], ib = s.dinv[b];
            const double al = s.alpha[a], be = s.alpha[b];
            const double gamma = gh * (da * db);
            if (above_tol<double>(gamma, al, be, 0.0, tol2)) {
                double t, c, ic;
                rot_params(al, be, gamma, t, c, ic);
                cs = pair_cos(gamma, al, be);
                ta = fabsf((float)t);
                s.tab[slot][p] = t * (db * ia);
                s.tba[slot][p] = t * (da * ib);
                s.d[a] = da * c;
                s.d[b] = db * c;
                s.dinv[a] = ia * ic;
                s.dinv[b] = ib * ic;
                const double na = fma(-t, gamma, al), nb = fma(t, gamma, be);
                if (lost_bits(na, al) || lost_bits(nb, be)) s.flags[1] = 1;
                s.alpha[a] = na;
                s.alpha[b] = nb;
                act = 1u << p;
            }
        }
        const unsigned m = __reduce_or_sync((1u << W) - 1u, act);
        const unsigned mc = __reduce_max_sync((1u << W) - 1u, __float_as_uint(cs));
        const unsigned mt = __reduce_max_sync((1u << W) - 1u, __float_as_uint(ta));
        if (p == 0) {
            s.act[slot] = m;
            s.flags[0] += __popc(m);
            s.mxc = max(s.mxc, mc);
            s.mxt = max(s.mxt, mt);
        }
    }
    par.x ^= 1;
    __syncthreads();
    const unsigned m = s.act[slot];
    if (m) {
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (!(m & (1u << p))) continue;
            const int a = pair_a<W>(intra, q, p), b = pair_b<W>(intra, q, p);
            const double tab = s.tab[slot][p], tba = s.tba[slot][p];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const double ya = x[k][a], yb = x[k][b];
                x[k][a] = fma(-tab, yb, ya);
                x[k][b] = fma(tba, ya, yb);
            }
        }
    }
    if (s.flags[1]) {  // the same in every CTA: recompute the 2W norms over the cluster
        cl_norms<W, RPT, CS>(cl, x, sm, par, rank);
        if (tid == 0) s.flags[1] = 0;
        __syncthreads();
    }
}

// Columns (a, b) of value idx of the batched test (FIRST: norms, intra pairs, cross pairs; else
// cross pairs only). Compile-time in the unrolled loops below.
template <bool FIRST, int W>
__device__ __forceinline__ constexpr int batch_a(int idx)
{
    return (FIRST && idx < 2 * W) ? idx
         : (FIRST && idx < 2 * W + ClBatch<W>::NI) ? pair_a<W>(true, (idx - 2 * W) / W, (idx - 2 * W) % W)
         : pair_a<W>(false, (idx - (FIRST ? 2 * W + ClBatch<W>::NI : 0)) / W,
                     (idx - (FIRST ? 2 * W + ClBatch<W>::NI : 0)) % W);
}
template <bool FIRST, int W>
__device__ __forceinline__ constexpr int batch_b(int idx)
{
    return (FIRST && idx < 2 * W) ? idx
         : (FIRST && idx < 2 * W + ClBatch<W>::NI) ? pair_b<W>(true, (idx - 2 * W) / W, (idx - 2 * W) % W)
         : pair_b<W>(false, (idx - (FIRST ? 2 * W + ClBatch<W>::NI : 0)) / W,
                     (idx - (FIRST ? 2 * W + ClBatch<W>::NI : 0)) % W);
}

// Per-warp partial sums of values OFF .. OFF + REM - 1 into bpart, at most 16 at a time (the
// rows stay in registers; only one chunk of sums is live).
template <bool FIRST, int OFF, int REM, int W, int RPT, int CS>
__device__ __forceinline__ void cl_batch_parts(const double (&x)[RPT][2 * W], ClShared<W, CS>& sm, int lane, int wid)
{
    if constexpr (REM > 0) {
        constexpr int C = REM >= 16 ? 16 : (REM >= 8 ? 8 : (REM >= 4 ? 4 : (REM >= 2 ? 2 : 1)));
        double t[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int a = batch_a<FIRST, W>(OFF + i), b = batch_b<FIRST, W>(OFF + i);
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < RPT; ++k) acc = fma(x[k][a], x[k][b], acc);
            t[i] = acc;
        }
        warp_reduce_multi<C>(t, lane);
        constexpr int sh = 5 - ilog2c(C);
        if ((lane & ((1 << sh) - 1)) == 0) sm.bpart[OFF + (lane >> sh)][wid] = t[0];
        cl_batch_parts<FIRST, OFF + C, REM - C, W, RPT, CS>(x, sm, lane, wid);
    }
}

// The batched test of a visit: every pair's dot product from the unrotated columns (and, in
// the first round of a sweep, the fresh squared norms, written to sm.v.alpha), summed over the
// cluster in one exchange, then the rotation test of the inner rounds on all of them. True
// (every CTA alike) when no pair would rotate. Ends synchronized.
template <bool FIRST, int W, int RPT, int CS>
__device__ bool cl_batch_quiet(const cg::cluster_group& cl, const double (&x)[RPT][2 * W], ClShared<W, CS>& sm,
                               ClPar& par, int rank, double tol2)
{
    using B = ClBatch<W>;
    constexpr int NV = FIRST ? B::NF : B::NC;
    constexpr int OC = FIRST ? 2 * W + B::NI : 0;
    VisitShared<double, W>& s = sm.v;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    cl_batch_parts<FIRST, 0, NV, W, RPT, CS>(x, sm, lane, wid);
    __syncthreads();
    if (tid < 32) {
        for (int i = lane; i < NV; i += 32) {
            const double sv = short_sum(sm.bpart[i], nw);
#pragma unroll
            for (int rr = 0; rr < CS; ++rr) *cl.map_shared_rank(&sm.xchb[par.b][rank][i], rr) = sv;
        }
    }
    cl.sync();
    if (tid < 32) {
        auto total = [&](int i) {
            double t = sm.xchb[par.b][0][i];
#pragma unroll
            for (int rr = 1; rr < CS; ++rr) t += sm.xchb[par.b][rr][i];
            return t;
        };
        if (FIRST && lane < 2 * W) {
            const double dc = s.d[lane];
            s.alpha[lane] = (s.gidx[lane] >= 0) ? total(lane) * dc * dc : 0.0;
        }
        __syncwarp();
        int cnt = 0;
        for (int i = lane; i < NV - (FIRST ? 2 * W : 0); i += 32) {
            const int idx = i + (FIRST ? 2 * W : 0);
            int a, b;
            if (FIRST && idx < OC) {
                a = pair_a<W>(true, (idx - 2 * W) / W, (idx - 2 * W) % W);
                b = pair_b<W>(true, (idx - 2 * W) / W, (idx - 2 * W) % W);
            } else {
                a = pair_a<W>(false, (idx - OC) / W, (idx - OC) % W);
                b = pair_b<W>(false, (idx - OC) / W, (idx - OC) % W);
            }
            if (s.gidx[a] >= 0 && s.gidx[b] >= 0 && (!s.cross_only || s.side[a] != s.side[b])) {
                const double gamma = total(idx) * (s.d[a] * s.d[b]);
                if (above_tol<double>(gamma, s.alpha[a], s.alpha[b], 0.0, tol2)) ++cnt;
            }
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) sm.brot = cnt;
    }
    par.b ^= 1;
    __syncthreads();
    return sm.brot == 0;
}

// X part of a visit on this CTA's rows: load, rotate, store. Rank 0 stores the columns' scales
// and tracked norms. Returns the rotation count (the same in every CTA). Ends with a CTA
// barrier after this CTA's stores.
template <int W, int RPT, int CS>
__device__ int cl_visit_x(const cg::cluster_group& cl, const SweepDims& D, double* X, int bi, int bj, bool first,
                          ClShared<W, CS>& sm, ClPar& par, int rank, ClRows rows, bool batch)
{
    VisitShared<double, W>& s = sm.v;
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int W2 = 2 * W;
    const double tol2 = D.tol * D.tol;
    double* dsc = (double*)D.dsc;
    double* alph = (double*)D.alph;
    const double fold_min = 1e-120;

    if (tid < W2) {
        const int blk = (tid < W) ? bi : bj;
        const int c = blk * W + (tid < W ? tid : tid - W);
        bool ok = (blk * W < D.n) && (c < D.n);
        if (D.filter != 0) {
            const int j0 = *(volatile const int*)D.j0;  // fixed before the launch
            if (D.filter == 1 && c < j0) ok = false;
            s.side[tid] = (unsigned char)(c < j0);
        }
        s.gidx[tid] = ok ? c : -1;
        const double dc = ok ? __ldcg(dsc + c) : 1.0;
        s.d[tid] = dc;
        s.dinv[tid] = 1.0 / dc;
        s.alpha[tid] = ok ? __ldcg(alph + c) : 0.0;
        s.fold[tid] = 1.0;
    }
    if (tid == 0) {
        s.flags[0] = 0;
        s.flags[1] = 0;
        s.mxc = 0u;
        s.mxt = 0u;
        s.cross_only = (D.filter == 2);
    }
    __syncthreads();

    double x[RPT][W2];
#pragma unroll
    for (int c = 0; c < W2; ++c) {
        const int gc = s.gidx[c];
        const double* col = X + (size_t)(gc < 0 ? 0 : gc) * D.ldX;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = rows.lo + tid + k * nthr;
            x[k][c] = (gc >= 0 && r < rows.hi) ? __ldcg(col + r) : 0.0;
        }
    }
    bool fresh = false;  // the first round's norms already in s.alpha
    if (batch) {
        // rotations have become rare: test every pair of the visit at once; a visit without a
        // rotation stores nothing but the fresh norms
        const bool quiet = first ? cl_batch_quiet<true, W, RPT, CS>(cl, x, sm, par, rank, tol2)
                                 : cl_batch_quiet<false, W, RPT, CS>(cl, x, sm, par, rank, tol2);
        if (quiet) {
            if (first && rank == 0 && tid < W2 && s.gidx[tid] >= 0) alph[s.gidx[tid]] = s.alpha[tid];
            __syncthreads();
            return 0;
        }
        fresh = first;
    }
    if (first && !fresh) cl_norms<W, RPT, CS>(cl, x, sm, par, rank);

    if (first) {
#pragma unroll
        for (int q = 0; q < W - 1; ++q) cl_inner_round<W, RPT, CS>(cl, x, true, q, q, sm, par, rank, tol2);
    }
    const int base = first ? W - 1 : 0;
#pragma unroll
    for (int q = 0; q < W; ++q) cl_inner_round<W, RPT, CS>(cl, x, false, q, base + q, sm, par, rank, tol2);

    const int nrot = s.flags[0];
    if (nrot > 0) {
        if (tid < W2 && s.gidx[tid] >= 0 && s.d[tid] < fold_min) {
            s.fold[tid] = s.d[tid];
            s.d[tid] = 1.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = s.gidx[c];
            if (gc < 0) continue;
            const double f = s.fold[c];
            double* col = X + (size_t)gc * D.ldX;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = rows.lo + tid + k * nthr;
                if (r < rows.hi) col[r] = (f == 1.0) ? x[k][c] : x[k][c] * f;
            }
        }
        if (rank == 0 && tid < W2 && s.gidx[tid] >= 0) {
            dsc[s.gidx[tid]] = s.d[tid];
            alph[s.gidx[tid]] = s.alpha[tid];
        }
    } else if (first) {
        if (rank == 0 && tid < W2 && s.gidx[tid] >= 0) alph[s.gidx[tid]] = s.alpha[tid];
    }
    __syncthreads();
    return nrot;
}

// Replay of the visit's rotation table on this CTA's rows of V (rows.lo .. rows.hi - 1).
template <int W, int RPT, int CS>
__device__ void cl_replay_v(const SweepDims& D, double* V, bool first, const ClShared<W, CS>& sm, ClRows rows)
{
    const VisitShared<double, W>& s = sm.v;
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int W2 = 2 * W;
    for (int r0 = rows.lo + tid; r0 < rows.hi; r0 += RPT * nthr) {
        double v[RPT][W2];
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = s.gidx[c];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = r0 + k * nthr;
                v[k][c] = (gc >= 0 && r < rows.hi) ? __ldcg(V + cm(r, gc, D.ldV)) : 0.0;
            }
        }
        replay_rows<W, RPT, double>(v, first, s);
#pragma unroll
        for (int c = 0; c < W2; ++c) {
            const int gc = s.gidx[c];
            if (gc < 0) continue;
            const double f = s.fold[c];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = r0 + k * nthr;
                if (r < rows.hi) V[cm(r, gc, D.ldV)] = (f == 1.0) ? v[k][c] : v[k][c] * f;
            }
        }
    }
}

// Thread 0 spins (bounded) until blocks bi and bj have version >= R. The result is this CTA's
// alone: callers agree on it over the cluster.
__device__ __forceinline__ bool cl_wait_local(const unsigned* ver, int bi, int bj, unsigned R, DevState* st)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
        unsigned spins = 0;
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

// The whole stage of Alg. 1 on X (and V) in one cooperative cluster launch (grid = whole
// clusters, one visit per cluster at a time), then the persistent scales are folded.
template <bool WITH_V, int W, int RPT, int CS>
__global__ void __launch_bounds__(kClMaxThreads, 1)
    k_sweeps_cl(SweepDims D, double* X, double* V, DevState* st, int phase, int gate_want)
{
    __shared__ ClShared<W, CS> sm;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    ClPar par;
    // The launch geometry this kernel is written for: clusters of exactly CS consecutive CTAs
    // of a one-dimensional grid, the rank equal to blockIdx.x mod CS, at most kClMaxThreads
    // threads. The same for every CTA of a cluster (so all leave together), checked before any
    // access to a peer's shared memory; a mismatch is recorded and nothing is computed.
    if (cl.num_blocks() != (unsigned)CS || gridDim.x % CS != 0 || gridDim.y != 1 || gridDim.z != 1 ||
        rank != (int)(blockIdx.x % CS) || blockDim.x > kClMaxThreads || blockDim.y != 1 || blockDim.z != 1) {
        if (tid == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
        return;
    }
    cl.sync();  // every CTA of the cluster has started before any writes a peer's shared memory
    // the gate and the failure flag: every CTA of the cluster leaves, or none
    if (!cl_agree<W, CS>(cl, sm, par, rank, !call_failed(st) && gate_open(st, gate_want), 0, nullptr)) return;
    const int ncl = (int)gridDim.x / CS, cid = (int)blockIdx.x / CS;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    double* dsc = (double*)D.dsc;
    for (int j = blockIdx.x * blockDim.x + tid; j < D.n; j += gridDim.x * blockDim.x) dsc[j] = 1.0;
    for (int b = blockIdx.x * blockDim.x + tid; b < 2 * D.k; b += gridDim.x * blockDim.x) D.ver[b] = 0u;
    if (blockIdx.x == 0)
        for (int i = tid; i < 64; i += blockDim.x) {
            st->rot_sweep[phase][i] = 0ull;
            st->mx_cos[phase][i] = 0u;
            st->mx_tan[phase][i] = 0u;
        }
    if (!cl_agree<W, CS>(cl, sm, par, rank, g.sync(), 0, nullptr)) return;

    const int rpc = (D.mX + CS - 1) / CS;
    const ClRows xr{rank * rpc, min(D.mX, (rank + 1) * rpc)};
    const int vpc = (D.nV + CS - 1) / CS;
    const ClRows vr{rank * vpc, min(D.nV, (rank + 1) * vpc)};
    const int k = D.k, half = k / 2, rounds = k - 1;
    const long long per_sweep = (long long)rounds * half;
    unsigned long long* rot_sweep = st->rot_sweep[phase];
    unsigned* mxc = st->mx_cos[phase];
    unsigned* mxt = st->mx_tan[phase];
    unsigned* vv = D.ver + k;
    int sweep = 0;
    bool conv = false;
    bool batch = false;  // the batched test (agreed with the convergence decision of the previous sweep)
    for (; sweep < D.maxsweep; ++sweep) {
        for (long long f = cid; f < per_sweep; f += ncl) {
            const int r = (int)(f / half), i = (int)(f - (long long)r * half);
            int bi, bj;
            rr_pair(k, r, i, bi, bj);
            if (bi > bj) { const int t = bi; bi = bj; bj = t; }
            const unsigned R = (unsigned)(sweep * rounds + r);
            if (!cl_agree<W, CS>(cl, sm, par, rank, cl_wait_local(D.ver, bi, bj, R, st), 0, nullptr)) return;
            const int nrot = cl_visit_x<W, RPT, CS>(cl, D, X, bi, bj, r == 0, sm, par, rank, xr, batch);
            if (nrot == 0) {
                // (the same in every CTA) nothing of X or V was stored but rank 0's norms, and every
                // rank read its rows before the visit's last exchange: rank 0 alone passes the
                // blocks on (X now; V once the previous round's replays on them are done). A wait
                // that gives up records the failure, which the sweep's grid barrier reports to all.
                if (rank == 0 && tid == 0) {
                    __threadfence();
                    st_release_u32(D.ver + bi, R + 1);
                    st_release_u32(D.ver + bj, R + 1);
                    if (WITH_V) {
                        const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
                        bool ok = true;
                        unsigned spins = 0;
                        while (ld_acquire_u32(vv + bi) < R || ld_acquire_u32(vv + bj) < R) {
                            if ((++spins & 255u) == 0 && (call_failed(st) || globaltimer_ns() - t0 > lim)) {
                                if (!call_failed(st)) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                                ok = false;
                                break;
                            }
                        }
                        if (ok) {
                            st_release_u32(vv + bi, R + 1);
                            st_release_u32(vv + bj, R + 1);
                        }
                    }
                }
                continue;
            }
            if (tid == 0) __threadfence();  // this CTA's stores before the barrier below
            // V's versions (each CTA acquires them for itself) and the release of X: after this
            // barrier every rank's X stores precede rank 0's release
            const bool okv = WITH_V ? cl_wait_local(vv, bi, bj, R, st) : true;
            const bool all = cl_agree<W, CS>(cl, sm, par, rank, okv, 0, nullptr);
            if (rank == 0 && tid == 0) {
                if (nrot) {
                    atomicAdd(&rot_sweep[sweep], (unsigned long long)nrot);
                    atomicMax(mxc + sweep, sm.v.mxc);
                    atomicMax(mxt + sweep, sm.v.mxt);
                }
                __threadfence();
                st_release_u32(D.ver + bi, R + 1);
                st_release_u32(D.ver + bj, R + 1);
            }
            if (!all) return;
            if (WITH_V) {
                if (nrot > 0) cl_replay_v<W, RPT, CS>(D, V, r == 0, sm, vr);
                __syncthreads();
                if (tid == 0) __threadfence();
                cl.sync();  // every rank's V stores precede the release
                if (rank == 0 && tid == 0) {
                    st_release_u32(vv + bi, R + 1);
                    st_release_u32(vv + bj, R + 1);
                }
            }
        }
        const bool ok = g.sync();
        int c0 = 0;
        if (rank == 0 && tid == 0) {
            c0 = (__ldcg(&rot_sweep[sweep]) == 0 || negligible_sweep(D, mxc, mxt, sweep)) ? 1 : 0;
            if (__uint_as_float(__ldcg(mxc + sweep)) < kClBatchCos) c0 |= 2;
        }
        int cdec = 0;
        if (!cl_agree<W, CS>(cl, sm, par, rank, ok, c0, &cdec)) return;
        batch = (cdec & 2) != 0;
        if (cdec & 1) {
            conv = true;
            ++sweep;
            break;
        }
    }
    fold_scales_cols<double>(g, D.mX, D.n, X, D.ldX, WITH_V ? D.nV : 0, WITH_V ? V : nullptr, D.ldV, dsc);
    if (blockIdx.x == 0 && tid == 0) {
        unsigned long long tot = 0;
        for (int s = 0; s < sweep; ++s) tot += __ldcg(&rot_sweep[s]);
        if (phase == 1) { st->sweeps_work = sweep; st->rot_work = tot; }
        else { st->sweeps_v += sweep; st->rot_v += tot; }
        if (!conv && D.filter != 2) atomicOr(&st->status, MPJSVD_STATUS_NOT_CONVERGED);
    }
    cl.sync();  // no CTA leaves while a peer could still write its shared memory
}

template <bool WITH_V, int W, int CS>
static int launch_cl(mpjsvd_ctx* h, const SweepDims& D0, double* X, double* V, DevState* st, int phase,
                     int gate_want)
{
    SweepDims D = D0;
    constexpr int RPT = cl_rpt(W);
    auto kern = k_sweeps_cl<WITH_V, W, RPT, CS>;
    const int rpc = (D.mX + CS - 1) / CS;
    int threads = (rpc + RPT - 1) / RPT;
    threads = std::max(64, std::min(kClMaxThreads, (threads + 31) & ~31));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(CS * std::max(1, D.k / 2));
    int ncl = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
    if (e != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return 1;  // not available: the caller uses the single-CTA visits
    }
    ncl = std::min(ncl, std::max(1, D.k / 2));
    cfg.gridDim = dim3(CS * ncl);
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.numAttrs = 2;
    e = cudaLaunchKernelEx(&cfg, kern, D, X, V, st, phase, gate_want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    ++h->launch_count;
    return 0;
}

// The launch for block width W and cs CTAs per visit (instantiated per W in its own file).
template <int W>
int launch_cl_w(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st, int phase, int gate_want,
                int cs)
{
    const bool wv = D.nV > 0 && V != nullptr;
    switch (cs) {
    case 2: return wv ? launch_cl<true, W, 2>(h, D, X, V, st, phase, gate_want) : launch_cl<false, W, 2>(h, D, X, V, st, phase, gate_want);
    case 4: return wv ? launch_cl<true, W, 4>(h, D, X, V, st, phase, gate_want) : launch_cl<false, W, 4>(h, D, X, V, st, phase, gate_want);
    case 8: return wv ? launch_cl<true, W, 8>(h, D, X, V, st, phase, gate_want) : launch_cl<false, W, 8>(h, D, X, V, st, phase, gate_want);
    default: return cuda_fail("cluster sweeps: cluster size", cudaErrorInvalidValue);
    }
}
extern template int launch_cl_w<2>(mpjsvd_ctx*, const SweepDims&, double*, double*, DevState*, int, int, int);
extern template int launch_cl_w<4>(mpjsvd_ctx*, const SweepDims&, double*, double*, DevState*, int, int, int);
extern template int launch_cl_w<8>(mpjsvd_ctx*, const SweepDims&, double*, double*, DevState*, int, int, int);

}  // namespace mpj
