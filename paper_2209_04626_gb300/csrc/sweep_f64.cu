// sweep_f64.cu -- binary64 refinement sweeps with V (Section 3.4): kernel instantiations
// and the launcher used by the single-matrix path.
#include "sweep_launch.cuh"

namespace mpj {

static int try_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                   int phase, int gate_want, int w, int rpt, int threads)
{
#define MPJ_L(WW, RR) \
    if (w == WW && rpt == RR) return launch_sweeps_wr<double, true, WW, RR>(h, D, X, V, st, phase, gate_want, threads)
    MPJ_L(1, 2); MPJ_L(1, 4); MPJ_L(1, 8); MPJ_L(1, 16);
    MPJ_L(2, 2); MPJ_L(2, 4); MPJ_L(2, 8); MPJ_L(2, 16);
    MPJ_L(4, 2); MPJ_L(4, 4); MPJ_L(4, 8);
    MPJ_L(8, 2); MPJ_L(8, 4);
#undef MPJ_L
    return -1;
}

// Block width w in {1, 2, 4, 8}; rows per thread chosen so that the visit's 2w columns fit
// in registers (w * rpt <= 32 doubles per thread), doubled while a variant's register use
// does not allow the thread count.
int launch_sweeps_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                      int phase, int gate_want, int* threads_out)
{
    const int w = D.w;
    int rpt = sweep_rpt(D.mX, w >= 8 ? 4 : 8);
    while (w * rpt > 32 && rpt > 2) rpt /= 2;
    for (; rpt <= 16 && w * rpt <= 32; rpt *= 2) {
        if ((D.mX + rpt - 1) / rpt > 1024) continue;
        const int threads = sweep_threads(D.mX, rpt);
        int rc = try_f64(h, D, X, V, st, phase, gate_want, w, rpt, threads);
        if (rc == kSweepTooManyThreads) continue;
        if (rc == -1) break;
        if (threads_out) *threads_out = threads;
        return rc;
    }
    return cuda_fail("sweep: no binary64 variant fits (block width, rows)", cudaErrorInvalidValue);
}

}  // namespace mpj
