// qr.cuh -- Householder QR and QR with column pivoting (Section 3.1 of the paper; the
// QRCP is the Businger-Golub RRQR the paper takes from DGEQP3), and the application of
// the resulting orthogonal factor.
//
// Parallel form: physical column c of the m x n matrix is owned by CTA c % g.size; every
// CTA recomputes the step's Householder vector from the pivot column (identical
// arithmetic in every CTA, so no broadcast is needed) and updates only its own columns.
// One group barrier per step (before the pivot is chosen). Pivoting is logical: columns never move; perm[j] names
// the physical column eliminated at step j, and a final gather puts R and the reflectors
// in logical order.
#pragma once

#include "common.cuh"

namespace mpj {

constexpr int kQrColBatch = 4;     // owned columns reduced together per pass
constexpr int kQrSlotStride = 256; // pivot-candidate slots per step parity (max CTAs)
constexpr int kApplyBatch = 8;     // columns of C updated per pass of apply_q_cols

// Pivot candidates of the column-distributed QRCP: CTA r publishes (largest remaining norm,
// physical column) of its own columns in slot par * kQrSlotStride + r (one 16-byte store;
// column -1 = none). The parity of the step double-buffers the slots.
__device__ __forceinline__ void put_candidate(DevState* st, int par, int rank, double v, int idx)
{
    st->cand[par * kQrSlotStride + rank] = make_double2(v, (double)idx);
}

// Warp-wide argmax over the `size` published candidates: largest norm, lowest column on ties,
// entries without a column skipped. All loads are issued before any is used (one L2 round
// trip). Every lane returns the winner.
__device__ __forceinline__ int pivot_argmax(const DevState* st, int par, int size, int lane)
{
    constexpr int K = kQrSlotStride / 32;
    double2 c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = lane + 32 * k;
        c[k] = (r < size) ? __ldcg(&st->cand[par * kQrSlotStride + r]) : make_double2(0.0, -1.0);
    }
    int best = -1;
    double bv = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int idx = (int)c[k].y;
        const double v = c[k].x;
        if (idx >= 0 && (best < 0 || v > bv || (v == bv && idx < best))) { bv = v; best = idx; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, best, o);
        if (oi >= 0 && (best < 0 || ov > bv || (ov == bv && oi < best))) { bv = ov; best = oi; }
    }
    return best;
}

// Householder reflector of x = A(j:m-1, p) (Section 3.1): H = I - tau v v^T with
// v = [1; x(1:) * rden], rden = 1 / (x_0 - beta), beta = -sign(x_0) |x|, H x = beta e_1.
// vs[j+1..m-1] receives the UNSCALED tail x(1:); the scale rden is applied to the two
// scalars of each column update instead of to every element (an FP64 division or
// multiply per element would be repeated by every CTA).
__device__ __forceinline__ void house_vector(int m, int j, const double* __restrict__ col,
                                             double* vs, double* red, double& tau, double& beta,
                                             double& rden)
{
    // the pivot column was last written by another CTA: read through L2 (__ldcg), never from a
    // possibly stale L1 line; four independent loads in flight per thread
    const double alpha = __ldcg(col + j);
    const int nt = blockDim.x;
    double s = 0.0, s2 = 0.0;
    int i = j + 1 + threadIdx.x;
    for (; i + 3 * nt < m; i += 4 * nt) {
        double x0 = __ldcg(col + i), x1 = __ldcg(col + i + nt);
        double x2 = __ldcg(col + i + 2 * nt), x3 = __ldcg(col + i + 3 * nt);
        vs[i] = x0;
        vs[i + nt] = x1;
        vs[i + 2 * nt] = x2;
        vs[i + 3 * nt] = x3;
        s = fma(x0, x0, s);
        s2 = fma(x1, x1, s2);
        s = fma(x2, x2, s);
        s2 = fma(x3, x3, s2);
    }
    for (; i < m; i += nt) {
        double x = __ldcg(col + i);
        vs[i] = x;
        s = fma(x, x, s);
    }
    s = block_sum(s + s2, red);
    if (s == 0.0) {
        tau = 0.0;
        beta = alpha;
        rden = 0.0;
    } else {
        double nrm = sqrt(fma(alpha, alpha, s));
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        rden = 1.0 / (alpha - beta);
    }
    __syncthreads();
}

// Partial dot products of the unscaled tail (rows j+1..m-1) with up to kQrColBatch
// columns, reduced over the CTA. red must hold >= kQrColBatch * 32 doubles. Result in w[]
// (all threads).
__device__ __forceinline__ void batch_dots(int m, int j, const double* vs, double* const* cols,
                                           int nb, double* red, double* w)
{
    double acc[kQrColBatch];
#pragma unroll
    for (int b = 0; b < kQrColBatch; ++b) acc[b] = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
        double vi = vs[i];
#pragma unroll
        for (int b = 0; b < kQrColBatch; ++b)
            if (b < nb) acc[b] = fma(vi, cols[b][i], acc[b]);
    }
    double out[kQrColBatch];
    block_sum_multi<kQrColBatch>(acc, red, out);
#pragma unroll
    for (int b = 0; b < kQrColBatch; ++b) w[b] = out[b];
}

// Column-distributed Householder QR (PIVOT = false) or QR with column pivoting
// (PIVOT = true) of the m x n matrix A (m >= n), in place.
// Outputs: tau[j]; perm[j] = physical column eliminated at step j (identity if !PIVOT);
// physical column perm[j] holds R(0..j, j) in rows 0..j and the reflector tail in rows
// j+1..m-1. Per-column metadata of the CTA's own columns (active flag, norms, new row-j
// entry) lives in shared memory. Dynamic shared memory: vs[m] doubles followed by
// own_max * (3 doubles + 1 int), own_max = ceil(n / g.size) (see hh_qr_smem_bytes).
// Returns false if a group barrier failed (the caller must exit).
__host__ __device__ inline size_t hh_qr_smem_bytes(int m, int n, int gsize)
{
    int own = (n + gsize - 1) / gsize;
    return sizeof(double) * ((size_t)m + 3 * (size_t)own) + sizeof(int) * (size_t)own + 64;
}

template <bool PIVOT>
__device__ bool hh_qr(const Group& g, int m, int n, double* A, int lda, double* tau, int* perm,
                      double* smem)
{
    __shared__ double red[kQrColBatch * 33];
    __shared__ int s_piv;
    __shared__ int s_recompute;
    const double tol3z = 1.0536712127723509e-08;  // sqrt(2^-53)
    DevState* st = g.st;
    const int own = (n - g.rank + g.size - 1) / g.size;  // columns c = rank + t * size
    double* vs = smem;
    double* vn1 = vs + m;
    double* vn2 = vn1 + own;
    double* rowj = vn2 + own;
    int* act = (int*)(rowj + own);
    const int lane = threadIdx.x & 31;

    for (int t = threadIdx.x; t < own; t += blockDim.x) act[t] = 1;
    if (PIVOT) {
        // initial norms of the CTA's columns
        for (int t = 0; t < own; ++t) {
            const double* col = A + cm(0, g.rank + t * g.size, lda);
            double s = 0.0;
            for (int i = threadIdx.x; i < m; i += blockDim.x) s = fma(col[i], col[i], s);
            s = block_sum(s, red);
            if (threadIdx.x == 0) {
                vn1[t] = sqrt(s);
                vn2[t] = vn1[t];
            }
        }
    }
    __syncthreads();

    int prev_p = -1;       // pivot column of the previous step (its store is deferred)
    double prev_beta = 0.0, prev_rden = 0.0;
    for (int j = 0; j < n; ++j) {
        // ---- pivot column of this step
        if (PIVOT) {
            // this CTA's candidate (warp 0): largest norm among active columns, first
            // active column if every comparison fails (NaN norms)
            if (threadIdx.x < 32) {
                int best = -1;
                double bv = 0.0;
                for (int t = lane; t < own; t += 32) {
                    if (!act[t]) continue;
                    double v = vn1[t];
                    if (best < 0 || v > bv) { bv = v; best = t; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    int ob = __shfl_xor_sync(0xffffffffu, best, o);
                    if (ob >= 0 && (best < 0 || ov > bv || (ov == bv && ob < best))) { bv = ov; best = ob; }
                }
                // slots alternate with the step's parity, so a CTA that runs ahead writes
                // step j+1's candidate while slower CTAs still read step j's
                if (lane == 0)
                    put_candidate(st, j & 1, g.rank, bv, best >= 0 ? g.rank + best * g.size : -1);
            }
            if (!g.sync()) return false;
            if (threadIdx.x < 32) {
                const int best = pivot_argmax(st, j & 1, g.size, lane);
                if (lane == 0) s_piv = best;
            }
            __syncthreads();
        } else {
            if (j > 0 && !g.sync()) return false;
            if (threadIdx.x == 0) s_piv = j;
            __syncthreads();
        }
        const int p = s_piv;
        if (p < 0 || p >= n) {  // cannot happen: n - j >= 1 columns are active
            if (threadIdx.x == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
            return false;
        }
        double* colp = A + cm(0, p, lda);

        // ---- store of the previous step's reflector, deferred past the barrier because
        //      every CTA reads the pivot column during its own step
        if (prev_p >= 0 && prev_p % g.size == g.rank) {
            double* cq = A + cm(0, prev_p, lda);
            for (int i = j + threadIdx.x; i < m; i += blockDim.x) cq[i] = vs[i] * prev_rden;
            if (threadIdx.x == 0) cq[j - 1] = prev_beta;
        }
        __syncthreads();

        // ---- Householder vector, computed redundantly by every CTA
        double tj, beta, rden;
        house_vector(m, j, colp, vs, red, tj, beta, rden);

        if (p % g.size == g.rank) {
            if (threadIdx.x == 0) {
                tau[j] = tj;
                perm[j] = p;
                act[(p - g.rank) / g.size] = 0;
            }
        }
        prev_p = p;
        prev_beta = beta;
        prev_rden = rden;
        __syncthreads();

        // ---- apply H_j to this CTA's active columns, kQrColBatch at a time
        int t = 0;
        while (true) {
            double* cols[kQrColBatch];
            int tix[kQrColBatch];
            int nb = 0;
            for (; t < own && nb < kQrColBatch; ++t) {
                int c = g.rank + t * g.size;
                bool active = PIVOT ? (act[t] != 0) : (c > j);
                if (active) {
                    tix[nb] = t;
                    cols[nb] = A + cm(0, c, lda);
                    ++nb;
                }
            }
            if (nb == 0) break;
            for (int b = nb; b < kQrColBatch; ++b) { cols[b] = cols[0]; tix[b] = tix[0]; }
            if (tj != 0.0) {
                // w = tau (c_j + rden x^T c_tail); c_j -= w; c_tail -= (w rden) x
                double w[kQrColBatch], f[kQrColBatch];
                batch_dots(m, j, vs, cols, nb, red, w);
#pragma unroll
                for (int b = 0; b < kQrColBatch; ++b) {
                    w[b] = tj * fma(rden, w[b], cols[b][j]);
                    f[b] = w[b] * rden;
                }
                __syncthreads();  // every thread has read c_j before it changes
                if (threadIdx.x == 0) {
                    for (int b = 0; b < nb; ++b) {
                        double nv = cols[b][j] - w[b];
                        cols[b][j] = nv;
                        if (PIVOT) rowj[tix[b]] = nv;
                    }
                }
                for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
                    double xi = vs[i];
#pragma unroll
                    for (int b = 0; b < kQrColBatch; ++b)
                        if (b < nb) cols[b][i] = fma(-f[b], xi, cols[b][i]);
                }
            } else if (PIVOT && threadIdx.x == 0) {
                for (int b = 0; b < nb; ++b) rowj[tix[b]] = cols[b][j];
            }
            __syncthreads();
            if (PIVOT) {
                // downdate the norms by the new row-j entries, one thread per column;
                // recompute from the data when cancellation is severe
                if (threadIdx.x == 0) s_recompute = 0;
                __syncthreads();
                if (threadIdx.x < nb) {
                    int tt = tix[threadIdx.x];
                    double v1 = vn1[tt];
                    if (v1 != 0.0) {
                        double r = fabs(rowj[tt]) / v1;
                        double q = 1.0 - r * r;
                        q = q < 0.0 ? 0.0 : q;
                        double ratio = v1 / vn2[tt];
                        if (q * ratio * ratio <= tol3z) {
                            atomicOr(&s_recompute, 1 << threadIdx.x);
                        } else {
                            vn1[tt] = v1 * sqrt(q);
                        }
                    }
                }
                __syncthreads();
                int mask = s_recompute;
                for (int b = 0; b < nb; ++b) {
                    if (!(mask & (1 << b))) continue;
                    double s = 0.0;
                    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x)
                        s = fma(cols[b][i], cols[b][i], s);
                    s = block_sum(s, red);
                    if (threadIdx.x == 0) {
                        vn1[tix[b]] = sqrt(s);
                        vn2[tix[b]] = vn1[tix[b]];
                    }
                }
                __syncthreads();
            }
        }
    }
    if (!PIVOT && !g.sync()) return false;
    if (prev_p >= 0 && prev_p % g.size == g.rank) {
        double* cq = A + cm(0, prev_p, lda);
        for (int i = n + threadIdx.x; i < m; i += blockDim.x) cq[i] = vs[i] * prev_rden;
        if (threadIdx.x == 0) cq[n - 1] = prev_beta;
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------------------
// Shared-memory-resident variant. Each CTA keeps its own columns (c = rank + t * size) in
// shared memory for the whole factorization, so the per-step updates never touch global
// memory; only the column that defines the step's reflector travels through a global
// broadcast buffer.
//   QRCP (PIVOT): after its updates every CTA publishes its candidate column (largest
//     remaining norm) in a parity-double-buffered slot; one grid barrier per step; every
//     CTA then reads the winner's slot.
//   QR (!PIVOT): no grid barrier. The owner of column j+1 updates that column first
//     (lookahead), publishes it in bcast[j+1] and raises flag[j+1]; the other CTAs wait
//     for the flag (bounded) before step j+1.
// Output in global memory as hh_qr: physical column c holds R and the reflector tail.
// ---------------------------------------------------------------------------------------

// Dynamic shared memory of hh_qr_res: own columns of ldc doubles, the step vector, and the
// per-column metadata.
__host__ __device__ inline int hh_res_ldc(int m) { return (m + 1) & ~1; }
__host__ __device__ inline size_t hh_qr_res_smem_bytes(int m, int n, int gsize)
{
    size_t own = (size_t)((n + gsize - 1) / gsize);
    return sizeof(double) * (own * (size_t)hh_res_ldc(m) + (size_t)m + 3 * own) +
           sizeof(int) * own + 64;
}

// Bounded wait until *flag != 0 (thread 0), then a CTA barrier. Returns false on timeout.
__device__ __forceinline__ bool wait_flag(const int* flag, DevState* st)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
        unsigned int spins = 0;
        while (*(volatile const int*)flag == 0) {
            if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > lim) {
                atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// bcast: PIVOT: 2 * g.size * m doubles; !PIVOT: n * m doubles. flags: n ints, zeroed
// (used when !PIVOT).
template <bool PIVOT>
__device__ bool hh_qr_res(const Group& g, int m, int n, double* A, int lda, double* tau, int* perm,
                          double* smem, double* bcast, int* flags)
{
    __shared__ double red[kQrColBatch * 33];
    __shared__ int s_piv, s_src;
    __shared__ int s_recompute;
    const double tol3z = 1.0536712127723509e-08;  // sqrt(2^-53)
    DevState* st = g.st;
    const int own = (n - g.rank + g.size - 1) / g.size;
    const int ldc = hh_res_ldc(m);
    double* C = smem;                       // own x ldc
    double* vs = C + (size_t)own * ldc;     // m
    double* vn1 = vs + m;
    double* vn2 = vn1 + own;
    double* rowj = vn2 + own;
    int* act = (int*)(rowj + own);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;

    // ---- load own columns, norms
    for (int t = 0; t < own; ++t) {
        const double* src = A + cm(0, g.rank + t * g.size, lda);
        double* dst = C + (size_t)t * ldc;
        for (int i = tid; i < m; i += nthr) dst[i] = src[i];
    }
    for (int t = tid; t < own; t += nthr) act[t] = 1;
    __syncthreads();
    if (PIVOT) {
        for (int t = 0; t < own; ++t) {
            const double* col = C + (size_t)t * ldc;
            double s = 0.0;
            for (int i = tid; i < m; i += nthr) s = fma(col[i], col[i], s);
            s = block_sum(s, red);
            if (tid == 0) { vn1[t] = s > 0.0 ? sqrt(s) : 0.0; vn2[t] = vn1[t]; }
        }
        __syncthreads();
    } else if (g.rank == 0 && n > 0) {
        // column 0 is ready as loaded: publish it
        for (int i = tid; i < m; i += nthr) bcast[i] = C[i];
        __syncthreads();
        if (tid == 0) { __threadfence(); atomicExch(&flags[0], 1); }
    }

    for (int j = 0; j < n; ++j) {
        const double* src;  // the step's column, rows j..m-1
        int p;
        if (PIVOT) {
            // candidate of this CTA: largest norm among its active columns (the first active
            // column if every comparison fails, NaN norms); publish its rows j..m-1
            if (tid < 32) {
                int best = -1;
                double bv = 0.0;
                for (int t = lane; t < own; t += 32) {
                    if (!act[t]) continue;
                    if (best < 0 || vn1[t] > bv) { bv = vn1[t]; best = t; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    int ob = __shfl_xor_sync(0xffffffffu, best, o);
                    if (ob >= 0 && (best < 0 || ov > bv || (ov == bv && ob < best))) { bv = ov; best = ob; }
                }
                if (lane == 0) {
                    put_candidate(st, j & 1, g.rank, bv, best >= 0 ? g.rank + best * g.size : -1);
                    s_src = best;
                }
            }
            __syncthreads();
            if (s_src >= 0) {
                const double* c = C + (size_t)s_src * ldc;
                double* slot = bcast + ((size_t)(j & 1) * g.size + g.rank) * m;
                for (int i = j + tid; i < m; i += nthr) slot[i] = c[i];
            }
            if (!g.sync()) return false;
            if (tid < 32) {
                const int best = pivot_argmax(st, j & 1, g.size, lane);
                if (lane == 0) s_piv = best;
            }
            __syncthreads();
            p = s_piv;
            if (p < 0 || p >= n) {
                if (tid == 0) atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                return false;
            }
            src = bcast + ((size_t)(j & 1) * g.size + (p % g.size)) * m;
        } else {
            p = j;
            if (!wait_flag(&flags[j], st)) return false;
            src = bcast + (size_t)j * m;
        }

        // ---- Householder vector from the published column (every CTA)
        double tj, beta, rden;
        house_vector(m, j, src, vs, red, tj, beta, rden);
        const bool mine = (p % g.size == g.rank);
        const int tp = (p - g.rank) / g.size;

        // ---- apply H_j: lookahead column first (plain QR), then the rest in batches
        const int la = (!PIVOT && j + 1 < n && (j + 1) % g.size == g.rank) ? (j + 1 - g.rank) / g.size : -1;
        for (int pass = (la >= 0 ? 0 : 1); pass < 2; ++pass) {
            int t = 0;
            while (true) {
                double* cols[kQrColBatch];
                int tix[kQrColBatch];
                int nb = 0;
                if (pass == 0) {
                    if (t == 0) { tix[0] = la; cols[0] = C + (size_t)la * ldc; nb = 1; t = own; }
                } else {
                    for (; t < own && nb < kQrColBatch; ++t) {
                        int c = g.rank + t * g.size;
                        bool active = PIVOT ? (act[t] != 0 && t != (mine ? tp : -1)) : (c > j && t != la);
                        if (active) { tix[nb] = t; cols[nb] = C + (size_t)t * ldc; ++nb; }
                    }
                }
                if (nb == 0) break;
                for (int b = nb; b < kQrColBatch; ++b) { cols[b] = cols[0]; tix[b] = tix[0]; }
                if (tj != 0.0) {
                    double w[kQrColBatch], f[kQrColBatch];
                    batch_dots(m, j, vs, cols, nb, red, w);
#pragma unroll
                    for (int b = 0; b < kQrColBatch; ++b) {
                        w[b] = tj * fma(rden, w[b], cols[b][j]);
                        f[b] = w[b] * rden;
                    }
                    __syncthreads();  // every thread has read c_j before it changes
                    if (tid == 0) {
                        for (int b = 0; b < nb; ++b) {
                            double nv = cols[b][j] - w[b];
                            cols[b][j] = nv;
                            if (PIVOT) rowj[tix[b]] = nv;
                        }
                    }
                    for (int i = j + 1 + tid; i < m; i += nthr) {
                        double xi = vs[i];
#pragma unroll
                        for (int b = 0; b < kQrColBatch; ++b)
                            if (b < nb) cols[b][i] = fma(-f[b], xi, cols[b][i]);
                    }
                } else if (PIVOT && tid == 0) {
                    for (int b = 0; b < nb; ++b) rowj[tix[b]] = cols[b][j];
                }
                __syncthreads();
                if (PIVOT) {
                    if (tid == 0) s_recompute = 0;
                    __syncthreads();
                    if (tid < nb) {
                        int tt = tix[tid];
                        double v1 = vn1[tt];
                        if (v1 != 0.0) {
                            double r = fabs(rowj[tt]) / v1;
                            double q = 1.0 - r * r;
                            q = q < 0.0 ? 0.0 : q;
                            double ratio = v1 / vn2[tt];
                            if (q * ratio * ratio <= tol3z) atomicOr(&s_recompute, 1 << tid);
                            else vn1[tt] = v1 * sqrt(q);
                        }
                    }
                    __syncthreads();
                    int mask = s_recompute;
                    for (int b = 0; b < nb; ++b) {
                        if (!(mask & (1 << b))) continue;
                        double s = 0.0;
                        for (int i = j + 1 + tid; i < m; i += nthr) s = fma(cols[b][i], cols[b][i], s);
                        s = block_sum(s, red);
                        if (tid == 0) { vn1[tix[b]] = sqrt(s); vn2[tix[b]] = vn1[tix[b]]; }
                    }
                    __syncthreads();
                }
            }
            if (pass == 0) {
                // publish the lookahead column for step j+1 and raise its flag
                const double* c = C + (size_t)la * ldc;
                double* dst = bcast + (size_t)(j + 1) * m;
                for (int i = j + 1 + tid; i < m; i += nthr) dst[i] = c[i];
                __syncthreads();
                if (tid == 0) { __threadfence(); atomicExch(&flags[j + 1], 1); }
            }
        }

        // ---- the owner finalizes column p: R entries above, beta, the scaled tail
        if (mine) {
            double* c = C + (size_t)tp * ldc;
            for (int i = j + 1 + tid; i < m; i += nthr) c[i] = vs[i] * rden;
            if (tid == 0) {
                c[j] = beta;
                tau[j] = tj;
                perm[j] = p;
                act[tp] = 0;
            }
        }
        __syncthreads();
    }

    // ---- write the own columns back
    for (int t = 0; t < own; ++t) {
        const double* s = C + (size_t)t * ldc;
        double* d = A + cm(0, g.rank + t * g.size, lda);
        for (int i = tid; i < m; i += nthr) d[i] = s[i];
    }
    __syncthreads();
    return true;
}

// C <- Q C (trans = false) or Q^T C (trans = true) for the rows 0..mrows-1 of the columns
// [c0, c1) of C, where Q = H_0 H_1 ... H_{k-1} and H_j = I - tau[j] v_j v_j^T,
// v_j = [0 (j entries); 1; Vr(j+1:mrows-1, j)]. Columns are independent, so any set of
// CTAs can split them without synchronizing. If c_ident >= 0 the block [c0, c1) of C holds
// columns c_ident.. of the identity, which H_j leaves untouched for j > column index:
// those reflectors are skipped (valid for trans = false only, where H_{k-1} acts first).
__device__ inline void apply_q_cols(bool trans, int mrows, int k, const double* Vr, int ldv,
                             const double* tau, double* C, int ldc, int c0, int c1, int c_ident)
{
    __shared__ double red[kApplyBatch * 33];
    for (int cb = c0; cb < c1; cb += kApplyBatch) {
        int nb = min(kApplyBatch, c1 - cb);
        double* cols[kApplyBatch];
#pragma unroll
        for (int b = 0; b < kApplyBatch; ++b) cols[b] = C + cm(0, cb + (b < nb ? b : 0), ldc);
        int jmax = k - 1;
        if (c_ident >= 0) jmax = min(jmax, c_ident + (cb - c0) + nb - 1);
        for (int s = 0; s < k; ++s) {
            int j = trans ? s : (k - 1 - s);
            if (j > jmax) continue;
            double tj = tau[j];
            if (tj == 0.0) continue;
            const double* v = Vr + cm(0, j, ldv);
            double acc[kApplyBatch];
#pragma unroll
            for (int b = 0; b < kApplyBatch; ++b) acc[b] = 0.0;
            for (int i = j + threadIdx.x; i < mrows; i += blockDim.x) {
                double vi = (i == j) ? 1.0 : v[i];
#pragma unroll
                for (int b = 0; b < kApplyBatch; ++b)
                    if (b < nb) acc[b] = fma(vi, cols[b][i], acc[b]);
            }
            double w[kApplyBatch];
            block_sum_multi<kApplyBatch>(acc, red, w);
#pragma unroll
            for (int b = 0; b < kApplyBatch; ++b) w[b] *= tj;
            for (int i = j + threadIdx.x; i < mrows; i += blockDim.x) {
                double vi = (i == j) ? 1.0 : v[i];
#pragma unroll
                for (int b = 0; b < kApplyBatch; ++b)
                    if (b < nb) cols[b][i] = fma(-w[b], vi, cols[b][i]);
            }
            __syncthreads();
        }
    }
}

}  // namespace mpj
