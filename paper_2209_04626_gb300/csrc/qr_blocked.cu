// qr_blocked.cu -- blocked Householder QR and the compact-WY application of its Q
// (Section 3.1: QR preconditioning; Section 3.3: QR of B and Q of the precision switch;
// Alg. 4 last line: U = Q [U_R; 0]).
//
// Layout is LAPACK's geqrf: R on and above the diagonal, the tail of reflector j below it
// (v_j(j) = 1 implicit), tau[j]; H_j = I - tau_j v_j v_j^T. Each reflector follows the same
// convention as the unblocked kernels: beta = -sign(alpha) |x|, tail scaled by
// 1 / (alpha - beta), tau = (beta - alpha) / beta, tau = 0 when the tail is zero.
//
// Panels of NB columns (NB = 32, or 16 for tall matrices whose panel does not fit):
//   k_panel_qr   one thread-block cluster of kPanelCl CTAs factors the m_p x NB panel; the
//                panel's rows are spread over the CTAs' shared memory and each column step
//                exchanges its partial sums through distributed shared memory (two cluster
//                barriers per column), so the panel never round-trips through L2;
//   k_wy_w       W = V^T C over all SMs (tiles of rows x 32 columns, split over rows with FP64
//                atomics), plus the panel's Gram matrix V^T V; the last Gram tile to finish
//                builds the triangular factor T of the compact-WY form Q_panel = I - V T V^T
//                recursively (T = [T1, -T1 G12 T2; 0, T2]: dependency depth 2 NB, not NB^2 / 2);
//   k_wy_update  per tile W' = T^T W (QR trailing update) or T W (Q C), then C -= V W'.
// On this GPU every binary64 instruction a warp issues occupies its SM sub-partition's FP64
// unit for a full pipe cycle, so the kernels spread the FP64 work over as many SMs as the
// dependency structure allows and keep the per-warp dependency chains short.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

// Phase probes of the panel kernel: empty here; a profiling build may define them to record
// per-phase clock counts (PROBE_BEGIN declares its state, PROBE(i) closes phase i).
#ifndef MPJ_PANEL_PROBE_BEGIN
#define MPJ_PANEL_PROBE_BEGIN
#define MPJ_PANEL_PROBE(i)
#define MPJ_PANEL_PROBE_END
#endif

namespace mpj {

constexpr int kPanelCl = 8;        // CTAs per panel cluster (portable cluster size)
constexpr int kPanelThreads = 256;
constexpr int kWyRc = 128;         // rows per tile of the wide trailing updates and of Q C
constexpr int kWyRcNarrow = 32;    // rows per tile of the look-ahead's narrow (next panel) update
constexpr int kWyThreads = 256;
constexpr size_t kPanelSmemMax = 200 * 1024;

__device__ __forceinline__ bool gate_skip(const DevState* st, int gate_want)
{
    return call_failed(st) || !gate_open(st, gate_want);
}

// v_k(r) of the panel starting at column j0: 0 above row j0 + k, 1 on it, the stored tail below.
__device__ __forceinline__ double refl_at(const double* V, int ldv, int j0, int k, int r)
{
    const int dr = j0 + k;
    return (r < dr) ? 0.0 : ((r == dr) ? 1.0 : V[cm(r, dr, ldv)]);
}

// ------------------------------------------------------------------------------------------
// Panel factorization: columns j0 .. j0+nbp-1, rows j0 .. m-1 of A, nbp <= NB. CTA q of the
// cluster holds rows j0 + q*rpc .. j0 + (q+1)*rpc - 1 in shared memory (column-major, odd ld).
template <int NB>
__global__ void __cluster_dims__(kPanelCl, 1, 1) __launch_bounds__(kPanelThreads)
    k_panel_qr(int m, int j0, int nbp, double* A, int lda, double* tau, DevState* st, int gate_want)
{
    extern __shared__ double psm[];
    __shared__ double exn[2][kPanelCl][2];   // per CTA: partial |tail|^2, diagonal entry
    __shared__ double exd[2][kPanelCl][NB];  // per CTA: partial dots with the later columns
    __shared__ double part[kPanelThreads / 32][NB];
    __shared__ double wv[NB];
    __shared__ double red[kPanelThreads / 32];
    __shared__ double refl[3];               // tau, beta, 1 / (alpha - beta) of this step
    __shared__ double ex4[2][kPanelCl][4];   // per CTA: S, R(j,j+1), A(j+1,j+1), v(j+1) partials
    __shared__ double part2[1];
    __shared__ double nxt[2];                // next step's |tail|^2 and diagonal entry
    __shared__ int s_fresh;
    if (gate_skip(st, gate_want)) return;  // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    const int cr = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kPanelThreads / 32;
    static_assert(NW == kPanelCl, "the cross-warp and cross-CTA sums share one 8-lane tree");
    const int mp = m - j0;
    const int rpc = (mp + kPanelCl - 1) / kPanelCl;
    const int ldp = rpc | 1;
    const int base = j0 + cr * rpc;
    const int nr = max(0, min(rpc, m - base));

    for (int c = 0; c < NB; ++c)
        for (int r = tid; r < rpc; r += kPanelThreads)
            psm[c * ldp + r] = (c < nbp && r < nr) ? A[cm(base + r, j0 + c, lda)] : 0.0;
    __syncthreads();
    MPJ_PANEL_PROBE_BEGIN

    // Every binary64 instruction occupies the FP64 unit of the warp's SM sub-partition, so
    // scalar work (the sums over warps and CTAs, the reflector) runs in warp 0 alone and is
    // broadcast through shared memory; 8-way sums are 3-level shuffle trees.
    //
    // One exchange per column: H_j preserves the norm of column j+1 over rows >= j, so with S
    // = |A(j:, j+1)|^2 (summed in the same pass as the dot products), the new entries
    // a = R(j, j+1) and alpha' = A'(j+1, j+1), the next reflector's |tail|^2 = S - a^2 - alpha'^2.
    // It is used only when it keeps almost all of S ((S - a^2) >= S/2 and the tail >= half of
    // that: then it is as accurate as a direct sum, and never mistakes rounding noise for a
    // tail); otherwise, and at the panel's first column, the next step sums it exactly.
    bool fresh = true;
    for (int j = 0; j < nbp; ++j) {
        const int par = j & 1;
        const int lj = j0 + j - base;  // local row of the diagonal entry (may lie outside)
        const int rlo = max(0, lj + 1);
        double* colj = psm + j * ldp;
        if (fresh) {
            // ---- |tail|^2 and the diagonal entry, summed over the cluster
            double s = 0.0;
            for (int r = rlo + tid; r < nr; r += kPanelThreads) s = fma(colj[r], colj[r], s);
            s = warp_sum(s);
            if (lane == 0) red[wid] = s;
            __syncthreads();
            MPJ_PANEL_PROBE(0)
            if (wid == 0) {
                double t = (lane < NW) ? red[lane] : 0.0;
                t += __shfl_xor_sync(0xffffffffu, t, 4);
                t += __shfl_xor_sync(0xffffffffu, t, 2);
                t += __shfl_xor_sync(0xffffffffu, t, 1);
                if (lane < kPanelCl) {
                    double* peer = cl.map_shared_rank(&exn[par][cr][0], lane);
                    peer[0] = t;
                    peer[1] = (lj >= 0 && lj < nr) ? colj[lj] : 0.0;
                }
            }
            MPJ_PANEL_PROBE(1)
            cl.sync();
            MPJ_PANEL_PROBE(2)
        }
        // ---- at the same time: warp 0 the reflector's scalars, warp 1 S = |A(j:, j+1)|^2,
        // warps 2..NW-1 the dot products of the UNSCALED tail with the later columns (the
        // reflector's scale 1/(alpha - beta) is applied to the partial sums afterwards)
        const int na = nbp - j - 1;
        int cpw = 1;
        while (cpw < na) cpw <<= 1;
        const int sub = 32 / cpw;
        const int ci = lane & (cpw - 1), sg = lane / cpw;
        const bool colok = ci < na;
        double* colc = psm + (j + 1 + (colok ? ci : 0)) * ldp;
        if (wid == 0) {
            double sq, al;
            if (fresh) {
                sq = (lane < kPanelCl) ? exn[par][lane][0] : 0.0;
                al = (lane < kPanelCl) ? exn[par][lane][1] : 0.0;  // one nonzero
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    sq += __shfl_xor_sync(0xffffffffu, sq, o);
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                }
            } else {
                sq = nxt[0];
                al = nxt[1];
            }
            if (lane == 0) {
                // with y = 1/|x|: beta = -sign(alpha)|x|, tau = (beta - alpha)/beta = 1 +
                // |alpha| y, 1/(alpha - beta) = sign(alpha)/(|alpha| + |x|): one reciprocal
                // square root and one division instead of a square root and two divisions
                double tj, beta, rden;
                if (sq == 0.0) {
                    tj = 0.0;
                    beta = al;
                    rden = 0.0;
                } else {
                    const double x2 = fma(al, al, sq);
                    const double y = rsqrt(x2);
                    const double nrm = x2 * y;
                    const double aa = fabs(al);
                    beta = (al >= 0.0) ? -nrm : nrm;
                    tj = fma(aa, y, 1.0);
                    const double rd = 1.0 / (aa + nrm);
                    rden = (al >= 0.0) ? rd : -rd;
                }
                refl[0] = tj;
                refl[1] = beta;
                refl[2] = rden;
                if (cr == 0) tau[j0 + j] = tj;
            }
        } else if (wid == 1) {
            if (na > 0) {
                const double* c1 = psm + (j + 1) * ldp;
                double sacc = 0.0;
                for (int r = max(0, lj) + lane; r < nr; r += 32) sacc = fma(c1[r], c1[r], sacc);
                sacc = warp_sum(sacc);
                if (lane == 0) part2[0] = sacc;
            }
        } else {
            // every lane of the warp reaches the full-mask shuffles (acc = 0 on idle lanes)
            double acc = 0.0;
            if (colok)
                for (int r = rlo + (wid - 2) * sub + sg; r < nr; r += (NW - 2) * sub) acc = fma(colj[r], colc[r], acc);
            for (int o = cpw; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (sg == 0 && colok) part[wid - 2][ci] = acc;
        }
        __syncthreads();
        MPJ_PANEL_PROBE(3)
        const double tj = refl[0], rden = refl[2];
        if (na == 0 || tj == 0.0) {  // tj is identical in every CTA of the cluster
            for (int r = rlo + tid; r < nr; r += kPanelThreads) colj[r] *= rden;
            if (tid == 0 && lj >= 0 && lj < nr) colj[lj] = refl[1];
            __syncthreads();
            fresh = true;
            continue;
        }
        MPJ_PANEL_PROBE(4)
        if (tid < na) {
            // this CTA's share of v^T A(:, c): rden * (unscaled dots) + the diagonal row's entry
            const double d = ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid])) +
                             (part[4][tid] + part[5][tid]);
            const double a = (lj >= 0 && lj < nr) ? psm[(j + 1 + tid) * ldp + lj] : 0.0;
            const double p = fma(rden, d, a);
#pragma unroll
            for (int q = 0; q < kPanelCl; ++q) *cl.map_shared_rank(&exd[par][cr][tid], q) = p;
        } else if (tid == 32) {
            // S, R(j, j+1) before the update, A(j+1, j+1) and v(j+1): the owners contribute
            const double sp = part2[0];
            const int l1 = lj + 1;
            const double aj = (lj >= 0 && lj < nr) ? psm[(j + 1) * ldp + lj] : 0.0;
            const double aj1 = (l1 >= 0 && l1 < nr) ? psm[(j + 1) * ldp + l1] : 0.0;
            const double vj1 = (l1 >= 0 && l1 < nr) ? colj[l1] * rden : 0.0;
#pragma unroll
            for (int q = 0; q < kPanelCl; ++q) {
                double* peer = cl.map_shared_rank(&ex4[par][cr][0], q);
                peer[0] = sp;
                peer[1] = aj;
                peer[2] = aj1;
                peer[3] = vj1;
            }
        }
        MPJ_PANEL_PROBE(5)
        cl.sync();
        MPJ_PANEL_PROBE(6)
        if (tid < na) {
            const double (*e)[NB] = exd[par];
            const double w = ((e[0][tid] + e[1][tid]) + (e[2][tid] + e[3][tid])) +
                             ((e[4][tid] + e[5][tid]) + (e[6][tid] + e[7][tid]));
            wv[tid] = tj * w;
        } else if (wid == 1) {
            // the next column's reflector inputs, downdated, in one warp: lane l holds quantity
            // l / 8 (S, R(j,j+1), A(j+1,j+1), v(j+1)) of CTA l % 8, and w_{j+1}; 3-level trees
            // over CTAs in the association order of the sums above (bit-identical results)
            const int q = lane & 7, kq = lane >> 3;
            double v = ex4[par][q][kq];
            double w = exd[par][q][0];
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
            const double S = __shfl_sync(0xffffffffu, v, 0);
            const double aj = __shfl_sync(0xffffffffu, v, 8);
            const double aj1 = __shfl_sync(0xffffffffu, v, 16);
            const double vj1 = __shfl_sync(0xffffffffu, v, 24);
            if (lane == 0) {
                const double wj = tj * w;
                const double a1 = fma(-wj, 1.0, aj);
                const double alpha1 = fma(-wj, vj1, aj1);
                const double T = fma(-a1, a1, S);
                const double tail = fma(-alpha1, alpha1, T);
                const bool ok = (T >= 0.5 * S) && (tail >= 0.5 * T);
                nxt[0] = tail;
                nxt[1] = alpha1;
                s_fresh = ok ? 0 : 1;
            }
        }
        // column j becomes the reflector: scaled tail, beta on the diagonal (the same product
        // x * rden as v(j+1) above, so the downdated alpha' equals the stored update)
        for (int r = rlo + tid; r < nr; r += kPanelThreads) colj[r] *= rden;
        __syncthreads();
        if (tid == 0 && lj >= 0 && lj < nr) colj[lj] = refl[1];
        MPJ_PANEL_PROBE(7)
        fresh = s_fresh != 0;
        // ---- A(:, c) -= tau w_c v (all NW warps: each row exactly once; v(lj) = 1)
        if (colok) {
            const double wc = wv[ci];
            const int rs8 = max(0, lj) + wid * sub + sg, rstep8 = NW * sub;
            for (int r = rs8; r < nr; r += rstep8) colc[r] = fma(-wc, r == lj ? 1.0 : colj[r], colc[r]);
        }
        __syncthreads();
        MPJ_PANEL_PROBE(8)
    }
    MPJ_PANEL_PROBE_END
    for (int c = 0; c < nbp; ++c)
        for (int r = tid; r < nr; r += kPanelThreads) A[cm(base + r, j0 + c, lda)] = psm[c * ldp + r];
}

// ------------------------------------------------------------------------------------------
// T (NB x NB upper triangular, Q_panel = H_0 ... H_{nbp-1} = I - V T V^T) from the Gram matrix
// G (NB x NB, ld NB, global) and tau, recursively: for block sizes b = 1, 2, 4, .. the
// off-diagonal block of each adjacent pair of diagonal blocks is -T1 G12 T2. Ts, Gs, Ms:
// shared scratch; all threads of the CTA call it; Ts holds T on return (synchronized).
template <int NB>
__device__ void build_T(const double* G, const double* tau, int j0, int nbp, double (*Ts)[NB + 1],
                        double (*Gs)[NB + 1], double (*Ms)[NB + 1])
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int e = tid; e < NB * NB; e += nthr) {
        const int i = e % NB, j = e / NB;
        Gs[i][j] = (i < nbp && j < nbp) ? __ldcg(G + (size_t)j * NB + i) : 0.0;
        Ts[i][j] = (i == j && i < nbp) ? tau[j0 + i] : 0.0;
    }
    __syncthreads();
    for (int b = 1; b < NB; b <<= 1) {
        const int nout = (NB / (2 * b)) * b * b;
        for (int e = tid; e < nout; e += nthr) {  // M = G12 T2
            const int pr = e / (b * b), ij = e % (b * b), i = ij % b, j = ij / b;
            const int lo = pr * 2 * b, hi = lo + b;
            double s = 0.0;
            for (int l = 0; l <= j; ++l) s = fma(Gs[lo + i][hi + l], Ts[hi + l][hi + j], s);
            Ms[lo + i][hi + j] = s;
        }
        __syncthreads();
        for (int e = tid; e < nout; e += nthr) {  // T12 = -T1 M
            const int pr = e / (b * b), ij = e % (b * b), i = ij % b, j = ij / b;
            const int lo = pr * 2 * b, hi = lo + b;
            double s = 0.0;
            for (int l = i; l < b; ++l) s = fma(Ts[lo + i][lo + l], Ms[lo + l][hi + j], s);
            Ts[lo + i][hi + j] = -s;
        }
        __syncthreads();
    }
}

// One accumulator set of the compact-WY update: the final W (NB x (ncols + NB), ld NB: V^T C
// then the Gram matrix V^T V), T (NB x NB), one partial W per row chunk and column strip, and
// a counter per strip (zero between uses).
struct WySet {
    double* W;
    double* T;
    double* Wp;
    unsigned* cnt;
};
constexpr int kWyMaxChunks = 32;

// Partial W(k, c) = sum_r v_k(r) C(r, c0 + c) over row chunk blockIdx.y (spc tiles of RC
// rows) and the 32 columns of strip blockIdx.x; the strip after the last one forms the Gram
// matrix V^T V. Each CTA stores its partial; the last CTA of a strip to finish (per-strip
// counter) sums the partials in chunk order (the result does not depend on timing), and for
// the Gram strip builds T. Every CTA does RC * 32 * NB FMAs: narrow updates (on the
// factorization's critical path) use short tiles so that more SMs share them.
template <int NB, int RC>
__global__ void __launch_bounds__(kWyThreads)
    k_wy_w(int m, int j0, int nbp, const double* V, int ldv, const double* C, int ldc, int c0,
           int ncols, int spc, WySet ws, const double* tau, DevState* st, int gate_want)
{
    constexpr int kTile = NB * (RC + 1), kTsc = 3 * NB * (NB + 1);
    __shared__ double Vsb[kTile > kTsc ? kTile : kTsc];  // the V tile, later T's scratch
    double(*Vs)[RC + 1] = reinterpret_cast<double(*)[RC + 1]>(Vsb);
    __shared__ int s_last;
    if (gate_skip(st, gate_want)) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nstrips = (ncols + 31) / 32;
    const int strip = blockIdx.x;
    const bool is_gram = strip == nstrips;
    constexpr int CG = 32 / NB;                       // column groups per warp
    constexpr int CPT = 32 / (kWyThreads / 32 * CG);  // columns per thread
    const int k = lane % NB;
    const int cgrp = wid * CG + lane / NB;
    const int cl0 = cgrp * CPT;  // first local column of this thread
    const double* cp[CPT];
    bool ok[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = cl0 + i;
        ok[i] = is_gram ? (c < nbp) : (strip * 32 + c < ncols);
        cp[i] = (ok[i] && !is_gram) ? C + (size_t)(c0 + strip * 32 + c) * ldc : C;
    }
    double acc[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) acc[i] = 0.0;
    for (int sc = 0; sc < spc; ++sc) {
        const int r0 = j0 + (blockIdx.y * spc + sc) * RC;
        if (r0 >= m) break;
        __syncthreads();  // Vs of the previous tile is no longer read
        for (int e = tid; e < NB * RC; e += kWyThreads) {
            const int kk = e / RC, r = e % RC, gr = r0 + r;
            Vs[kk][r] = (kk < nbp && gr < m) ? refl_at(V, ldv, j0, kk, gr) : 0.0;
        }
        __syncthreads();
        const int rend = min(RC, m - r0);
        for (int r = 0; r < rend; ++r) {
            const double v = Vs[k][r];
            const int gr = r0 + r;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                double c;
                if (is_gram) c = ok[i] ? Vs[cl0 + i][r] : 0.0;
                else c = ok[i] ? cp[i][gr] : 0.0;
                acc[i] = fma(v, c, acc[i]);
            }
        }
    }
    double* mine = ws.Wp + ((size_t)blockIdx.y * (nstrips + 1) + strip) * (NB * 32);
#pragma unroll
    for (int i = 0; i < CPT; ++i) mine[(cl0 + i) * NB + k] = acc[i];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&ws.cnt[strip], 1u) == gridDim.y - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int ncs = is_gram ? NB : min(32, ncols - strip * 32);
    for (int e = tid; e < NB * ncs; e += kWyThreads) {
        const int kk = e % NB, c = e / NB;
        double sum = 0.0;
        for (int q = 0; q < (int)gridDim.y; ++q)
            sum += __ldcg(ws.Wp + ((size_t)q * (nstrips + 1) + strip) * (NB * 32) + c * NB + kk);
        ws.W[(size_t)(is_gram ? ncols + c : strip * 32 + c) * NB + kk] = sum;
    }
    if (tid == 0) ws.cnt[strip] = 0u;
    if (!is_gram) return;
    __syncthreads();
    double(*Ts)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(Vsb);
    double(*Gs)[NB + 1] = Ts + NB;
    double(*Ms)[NB + 1] = Ts + 2 * NB;
    build_T<NB>(ws.W + (size_t)ncols * NB, tau, j0, nbp, Ts, Gs, Ms);
    for (int e = tid; e < NB * NB; e += kWyThreads) ws.T[e] = Ts[e % NB][e / NB];
}

// C(r, c0 + c) -= sum_k v_k(r) W'(k, c), W' = op(T) W(:, strip), over a tile of RC rows x
// 32 columns; op(T) = T^T (trans: Q_panel^T C, the QR's trailing update) or T (Q_panel C).
template <int NB, int RC>
__global__ void __launch_bounds__(kWyThreads)
    k_wy_update(int m, int j0, int nbp, const double* V, int ldv, double* C, int ldc, int c0,
                int ncols, const double* W, const double* T, bool trans, DevState* st, int gate_want)
{
    static_assert(RC % 32 == 0, "rows per thread are lane + 32 i");
    __shared__ double Vs[NB][RC + 1];
    __shared__ double Ws[NB][33];
    if (gate_skip(st, gate_want)) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int r0 = j0 + blockIdx.y * RC;
    const int cs = blockIdx.x * 32;
    for (int e = tid; e < NB * RC; e += kWyThreads) {
        const int k = e / RC, r = e % RC, gr = r0 + r;
        Vs[k][r] = (k < nbp && gr < m) ? refl_at(V, ldv, j0, k, gr) : 0.0;
    }
    for (int e = tid; e < NB * 32; e += kWyThreads) {
        const int k = e % NB, c = e / NB;
        Ws[k][c] = (k < nbp && cs + c < ncols) ? W[(size_t)(cs + c) * NB + k] : 0.0;
    }
    __syncthreads();
    {
        // W' = op(T) Ws: thread (c = lane, row group wid) computes rows {g, NB/2-1-g, NB/2+g,
        // NB-1-g} (NB = 32) or {g, NB-1-g} (NB = 16): every thread runs the same number of
        // triangular terms. op(T)(k, l) = T(l, k), l <= k (trans) or T(k, l), l >= k.
        constexpr int KPT = NB / 8;
        int ks[KPT];
        if (KPT == 4) {
            ks[0] = wid; ks[1 % KPT] = NB / 2 - 1 - wid; ks[2 % KPT] = NB / 2 + wid; ks[3 % KPT] = NB - 1 - wid;
        } else {
            ks[0] = wid; ks[1 % KPT] = NB - 1 - wid;
        }
        double out[KPT];
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            const int kk = ks[q];
            double s = 0.0;
            if (trans) {
                for (int l = 0; l <= kk; ++l) s = fma(__ldg(T + (size_t)kk * NB + l), Ws[l][lane], s);
            } else {
                for (int l = kk; l < NB; ++l) s = fma(__ldg(T + (size_t)l * NB + kk), Ws[l][lane], s);
            }
            out[q] = s;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < KPT; ++q) Ws[ks[q]][lane] = out[q];
        __syncthreads();
    }
    constexpr int RI = RC / 32;                 // rows per thread (lane + 32 i)
    constexpr int CJ = 32 / (kWyThreads / 32);  // columns per thread (wid * CJ + j)
    double acc[RI][CJ];
    bool rok[RI], cok[CJ];
#pragma unroll
    for (int i = 0; i < RI; ++i) rok[i] = r0 + lane + 32 * i < m;
#pragma unroll
    for (int j = 0; j < CJ; ++j) cok[j] = cs + wid * CJ + j < ncols;
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
        const double* col = C + (size_t)(c0 + cs + wid * CJ + j) * ldc;
#pragma unroll
        for (int i = 0; i < RI; ++i) acc[i][j] = (rok[i] && cok[j]) ? col[r0 + lane + 32 * i] : 0.0;
    }
    for (int k = 0; k < nbp; ++k) {
        double vk[RI], wk[CJ];
#pragma unroll
        for (int i = 0; i < RI; ++i) vk[i] = Vs[k][lane + 32 * i];
#pragma unroll
        for (int j = 0; j < CJ; ++j) wk[j] = Ws[k][wid * CJ + j];
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < CJ; ++j) acc[i][j] = fma(-vk[i], wk[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
        if (!cok[j]) continue;
        double* col = C + (size_t)(c0 + cs + wid * CJ + j) * ldc;
#pragma unroll
        for (int i = 0; i < RI; ++i)
            if (rok[i]) col[r0 + lane + 32 * i] = acc[i][j];
    }
}

// ------------------------------------------------------------------------------------------
// host side

// Panel width for an m-row factorization: 32 when the panel's rows fit the cluster's shared
// memory, else 16; 0 when neither fits (callers then use the unblocked kernels).
int bqr_nb(int m)
{
    const int rpc = (m + kPanelCl - 1) / kPanelCl;
    const size_t ldp = (size_t)(rpc | 1);
    if (ldp * 32 * sizeof(double) <= kPanelSmemMax) return 32;
    if (ldp * 16 * sizeof(double) <= kPanelSmemMax) return 16;
    return 0;
}

// Row chunks of a step with m - j0 <= m_max rows and tiles of rc rows (at most kWyMaxChunks).
static int wy_chunks_max(int m_max, int rc) { return std::max(1, std::min(kWyMaxChunks, (m_max + rc - 1) / rc)); }

// Doubles of one accumulator set for up to ncap columns, m_max rows and tiles of rc rows
// (sized for NB = 32).
static size_t wyset_doubles(int ncap, int m_max, int rc)
{
    const size_t ns = (size_t)(ncap + 31) / 32 + 1;
    return (size_t)32 * ((size_t)ncap + 32) + 32 * 32 + (size_t)wy_chunks_max(m_max, rc) * ns * 32 * 32 + (ns + 1) / 2 + 2;
}
static WySet wyset_at(double* base, int ncap, int m_max, int rc)
{
    const size_t ns = (size_t)(ncap + 31) / 32 + 1;
    WySet w;
    w.W = base;
    w.T = w.W + (size_t)32 * ((size_t)ncap + 32);
    w.Wp = w.T + 32 * 32;
    w.cnt = (unsigned*)(w.Wp + (size_t)wy_chunks_max(m_max, rc) * ns * 32 * 32);
    return w;
}
static size_t wyset_cnt_bytes(int ncap) { return sizeof(unsigned) * ((size_t)(ncap + 31) / 32 + 1); }

// a narrow set (the next panel's columns) and a wide set (the rest / a whole apply)
size_t bqr_wbuf_doubles(int ncols_max, int m_max)
{
    return wyset_doubles(32, m_max, kWyRcNarrow) + wyset_doubles(ncols_max, m_max, kWyRc);
}

// One panel's compact-WY update C(j0:m, c0:c0+ncols) <- (I - V op(T) V^T) C with T built
// from the panel's Gram matrix: op(T) = T^T applies Q_panel^T (QR trailing update), T applies
// Q_panel (forming Q C). Rows are split into at most kWyMaxChunks chunks.
template <int NB, int RC>
static void wy_step(mpjsvd_ctx* h, cudaStream_t s, int m, int j0, int nbp, const double* V, int ldv,
                    const double* tau, double* C, int ldc, int c0, int ncols, const WySet& ws, bool trans,
                    DevState* st, int gate_want)
{
    const int nstrips = (ncols + 31) / 32;
    const int nsub = (m - j0 + RC - 1) / RC;
    const int spc = (nsub + kWyMaxChunks - 1) / kWyMaxChunks;
    const int nchunks = (nsub + spc - 1) / spc;
    k_wy_w<NB, RC><<<dim3(nstrips + 1, nchunks), kWyThreads, 0, s>>>(m, j0, nbp, V, ldv, C, ldc, c0, ncols, spc,
                                                                     ws, tau, st, gate_want);
    k_wy_update<NB, RC><<<dim3(std::max(1, nstrips), nsub), kWyThreads, 0, s>>>(m, j0, nbp, V, ldv, C, ldc, c0,
                                                                                ncols, ws.W, ws.T, trans, st,
                                                                                gate_want);
    h->launch_count += 2;
}

// Look-ahead: the panel after p needs only its own columns updated by panel p (the "narrow"
// update), so the update of the columns beyond it (the "wide" update) overlaps the
// factorization of the next panel. Panels and narrow updates form the critical chain and run
// on the handle's high-priority stream, the wide updates on its low-priority stream: the
// wide updates fill the GPU, and without the priorities the narrow update's CTAs queue
// behind theirs (measured on 1024 x 1024: narrow 137 us per panel instead of ~10 us). Column
// ranges: panel p = [j0, j0 + nbp), next panel = [cn0, cn0 + nbn), wide = [cw0, n). Panel
// p's columns have received every earlier update once wide(p-2) and narrow(p-1) (in order
// on the critical stream) are done; the narrow update of p needs wide(p-1). The narrow and
// wide updates use separate accumulator sets; successive wide updates run in order.
template <int NB>
static int bqr_factor_nb(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau, double* W,
                         DevState* st, int gate_want)
{
    cudaStream_t s = h->stream;
    const size_t smax = sizeof(double) * NB * (size_t)(((m + kPanelCl - 1) / kPanelCl) | 1);
    cudaError_t e = cudaFuncSetAttribute(k_panel_qr<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    if (e != cudaSuccess) return cuda_fail("panel smem attribute", e);
    const WySet wn = wyset_at(W, 32, m, kWyRcNarrow), ww = wyset_at(W + wyset_doubles(32, m, kWyRcNarrow), n, m, kWyRc);
    if ((e = cudaMemsetAsync(wn.cnt, 0, wyset_cnt_bytes(32), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(ww.cnt, 0, wyset_cnt_bytes(n), s)) != cudaSuccess)
        return cuda_fail("wy counters", e);
    const bool la = h->have_side;
    const cudaStream_t c = la ? h->crit : s;
    if (la && ((e = cudaEventRecord(h->qev[5], s)) != cudaSuccess || (e = cudaStreamWaitEvent(c, h->qev[5], 0)) != cudaSuccess ||
               (e = cudaStreamWaitEvent(h->side, h->qev[5], 0)) != cudaSuccess))
        return cuda_fail("blocked QR fork", e);
    int p = 0;
    for (int j0 = 0; j0 < n; j0 += NB, ++p) {
        const int nbp = std::min(NB, n - j0);
        const int cn0 = j0 + nbp, nbn = std::min(NB, n - cn0);
        const int cw0 = cn0 + nbn, ncw = n - cw0;
        const size_t psmem = sizeof(double) * NB * (size_t)(((m - j0 + kPanelCl - 1) / kPanelCl) | 1);
        if (!la) {  // one stream: the whole trailing matrix at once
            const int nt = n - cn0;
            k_panel_qr<NB><<<kPanelCl, kPanelThreads, psmem, s>>>(m, j0, nbp, A, lda, tau, st, gate_want);
            ++h->launch_count;
            if (nt > 0) wy_step<NB, kWyRc>(h, s, m, j0, nbp, A, lda, tau, A, lda, cn0, nt, ww, true, st, gate_want);
        } else {
            if (p >= 2 && (e = cudaStreamWaitEvent(c, h->qev[1 + (p - 2) % 3], 0)) != cudaSuccess) break;
            k_panel_qr<NB><<<kPanelCl, kPanelThreads, psmem, c>>>(m, j0, nbp, A, lda, tau, st, gate_want);
            ++h->launch_count;
            if ((e = cudaEventRecord(h->qev[0], c)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(h->side, h->qev[0], 0)) != cudaSuccess) break;
            if (ncw > 0)
                wy_step<NB, kWyRc>(h, h->side, m, j0, nbp, A, lda, tau, A, lda, cw0, ncw, ww, true, st, gate_want);
            if ((e = cudaEventRecord(h->qev[1 + p % 3], h->side)) != cudaSuccess) break;
            if (nbn > 0) {
                if (p >= 1 && (e = cudaStreamWaitEvent(c, h->qev[1 + (p - 1) % 3], 0)) != cudaSuccess) break;
                wy_step<NB, kWyRcNarrow>(h, c, m, j0, nbp, A, lda, tau, A, lda, cn0, nbn, wn, true, st, gate_want);
            }
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
    }
    if (la) {  // join: later work on the handle's stream sees both chains
        cudaError_t e2 = cudaEventRecord(h->qev[4], h->side);
        if (e2 == cudaSuccess) e2 = cudaEventRecord(h->qev[6], c);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, h->qev[4], 0);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, h->qev[6], 0);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail("blocked QR kernels", e);
    return 0;
}

// Scratch bytes of bqr_factor / bqr_apply for m rows and n columns (or reflectors).
size_t bqr_ws_bytes(const mpjsvd_ctx* h, int m, int n)
{
    const size_t one = sizeof(double) * bqr_wbuf_doubles(n, m);
    bool any = false;
    for (int site = kQrSitePrecond; site <= kQrSiteCall; ++site) any = any || bqr_outer_used(h, m, n, site);
    return any ? std::max(one, bqr_outer_ws_bytes(m, n)) : one;
}

// Householder QR of the m x n (m >= n) column-major A in place (geqrf layout) with tau[n].
// W: bqr_ws_bytes(h, m, n) bytes of scratch. Requires bqr_nb(m) > 0.
int bqr_factor(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau, double* W, DevState* st,
               int gate_want, int site)
{
    if (bqr_outer_used(h, m, n, site)) return bqr_factor_outer(h, m, n, A, lda, tau, W, st, gate_want);
    const int nb = bqr_nb(m);
    if (nb == 32) return bqr_factor_nb<32>(h, m, n, A, lda, tau, W, st, gate_want);
    if (nb == 16) return bqr_factor_nb<16>(h, m, n, A, lda, tau, W, st, gate_want);
    return cuda_fail("blocked QR: panel does not fit", cudaErrorInvalidValue);
}

// C (m x ncols, leading rows of a matrix with ld ldc) <- Q C, Q = H_0 ... H_{k-1} from the k
// reflectors stored in V (m x k, geqrf layout). ident: C holds the identity's first ncols
// columns on entry, so panel p only touches columns >= its first (the structure of forming Q).
// W: bqr_wbuf_doubles(ncols, m) doubles of scratch, or bqr_outer_ws_bytes(m, max(ncols, k))
// bytes when bqr_outer_used(h, m, k).
int bqr_apply(mpjsvd_ctx* h, int m, int ncols, int k, const double* V, int ldv, const double* tau,
              double* C, int ldc, bool ident, double* W, DevState* st, int gate_want, int site)
{
    if (bqr_outer_used(h, m, k, site))
        return bqr_apply_outer(h, m, ncols, k, V, ldv, tau, C, ldc, ident, W, st, gate_want);
    constexpr int NB = 32;
    const WySet ws = wyset_at(W + wyset_doubles(32, m, kWyRcNarrow), ncols, m, kWyRc);
    cudaError_t e = cudaMemsetAsync(ws.cnt, 0, wyset_cnt_bytes(ncols), h->stream);
    if (e != cudaSuccess) return cuda_fail("wy counters", e);
    for (int j0 = ((k - 1) / NB) * NB; j0 >= 0; j0 -= NB) {
        const int nbp = std::min(NB, k - j0);
        const int cstart = ident ? j0 : 0;
        const int nc = ncols - cstart;
        if (nc <= 0) continue;
        wy_step<NB, kWyRc>(h, h->stream, m, j0, nbp, V, ldv, tau, C, ldc, cstart, nc, ws, false, st, gate_want);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail("blocked apply kernels", e);
    }
    return 0;
}

int qr_call(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau)
{
    const size_t wbytes = bqr_ws_bytes(h, m, n);
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, wbytes);
    if (rc) return rc;
    DevState* st = (DevState*)h->dstate;
    h->launch_count = 0;
    rc = state_reset(h, st);
    if (rc) return rc;
    return bqr_factor(h, m, n, A, lda, tau, (double*)h->ws, st, -1);
}

int apply_q_call(mpjsvd_ctx* h, int m, int ncols, int k, const double* A, int lda, const double* tau,
                 double* C, int ldc)
{
    size_t wbytes = sizeof(double) * bqr_wbuf_doubles(ncols, m);
    if (bqr_outer_used(h, m, k, kQrSiteCall)) wbytes = std::max(wbytes, bqr_outer_ws_bytes(m, std::max(ncols, k)));
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, wbytes);
    if (rc) return rc;
    DevState* st = (DevState*)h->dstate;
    h->launch_count = 0;
    rc = state_reset(h, st);
    if (rc) return rc;
    return bqr_apply(h, m, ncols, k, A, lda, tau, C, ldc, false, (double*)h->ws, st, -1);
}

}  // namespace mpj
