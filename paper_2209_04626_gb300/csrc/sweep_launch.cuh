// sweep_launch.cuh -- the persistent cooperative sweep kernel and its host launcher,
// instantiated for binary32 (sweep_f32.cu) and binary64 (sweep_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"

namespace mpj {

// Internal return code: the variant needs fewer threads (more rows per thread).
constexpr int kSweepTooManyThreads = 1;

// Stage of Alg. 1 on X (rows mX, n columns, ld mX) and optionally V (n x n): all sweeps in one
// cooperative launch, then the persistent column scales are folded into X and V. Returns
// immediately if the call already failed or the gate says the stage is skipped.
template <typename T, bool WITH_V, int W, int RPT>
__global__ void k_sweeps(SweepDims D, T* X, double* V, DevState* st, int phase, int gate_want)
{
    __shared__ VisitShared<T, W> sm;
    if (call_failed(st)) return;
    if (!gate_open(st, gate_want)) return;
    Group g{(int)blockIdx.x, (int)gridDim.x, st};
    // persistent scales start at 1, block versions at 0, the phase's per-sweep records at 0 (a
    // phase may run more than once in a call)
    T* dsc = (T*)D.dsc;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += gridDim.x * blockDim.x) dsc[j] = T(1);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < 2 * D.k; b += gridDim.x * blockDim.x) D.ver[b] = 0u;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 64; i += blockDim.x) {
            st->rot_sweep[phase][i] = 0ull;
            st->mx_cos[phase][i] = 0u;
            st->mx_tan[phase][i] = 0u;
        }
    if (!g.sync()) return;
    bool conv = false;
    int sweeps = jacobi_sweeps_flow<T, WITH_V, W, RPT>(g, D, X, V, st->rot_sweep[phase], st->mx_cos[phase],
                                                       st->mx_tan[phase], D.ver, sm, &conv);
    if (sweeps < 0) return;
    fold_scales_cols<T>(g, D.mX, D.n, X, D.ldX, WITH_V ? D.nV : 0, WITH_V ? V : nullptr, D.ldV, dsc);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int s = 0; s < sweeps; ++s) tot += __ldcg(&st->rot_sweep[phase][s]);
        if (phase == 0) { st->sweeps_low = sweeps; st->rot_low = tot; }
        else if (phase == 1) { st->sweeps_work = sweeps; st->rot_work = tot; }
        else { st->sweeps_v += sweeps; st->rot_v += tot; }
        // a one-pass launch (the safeguard's pass over the Y1 x Y2 pairs) is complete by design
        if (!conv && D.filter != 2) atomicOr(&st->status, MPJSVD_STATUS_NOT_CONVERGED);
    }
}

template <typename T, bool WITH_V, int W, int RPT>
static int launch_sweeps_wr(mpjsvd_ctx* h, const SweepDims& D0, T* X, double* V, DevState* st,
                            int phase, int gate_want, int threads)
{
    SweepDims D = D0;
    auto kern = k_sweeps<T, WITH_V, W, RPT>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return cuda_fail("sweep attributes", e);
    if (threads > fa.maxThreadsPerBlock) return kSweepTooManyThreads;  // caller retries
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail("sweep occupancy", e);
    if (occ < 1) return cuda_fail("sweep occupancy (0 blocks fit)", cudaErrorInvalidConfiguration);
    // up to two CTAs per visit of a round: consecutive rounds of a visit index go to different
    // CTAs, so a CTA's replay on V overlaps the next round's work on X
    int grid = std::min(D.k, occ * h->num_sms);
    grid = std::max(1, std::min(grid, 1024));
    void* args[] = {&D, &X, &V, &st, &phase, &gate_want};
    e = cudaLaunchCooperativeKernel((void*)kern, grid, threads, args, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail("sweep launch", e);
    ++h->launch_count;
    return 0;
}

// Rows per thread for a register-resident visit: the smallest power of two >= 2 that keeps
// the block at <= 1024 threads and near the target per thread.
inline int sweep_rpt(int mX, int target)
{
    int rpt = std::max(2, target);
    while ((mX + rpt - 1) / rpt > 1024) rpt *= 2;
    return rpt;
}

inline int sweep_threads(int mX, int rpt)
{
    int t = (mX + rpt - 1) / rpt;
    t = (t + 31) & ~31;
    return std::max(64, std::min(1024, t));
}

}  // namespace mpj
