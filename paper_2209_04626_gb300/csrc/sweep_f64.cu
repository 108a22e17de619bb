// sweep_f64.cu -- binary64 refinement sweeps with V (Section 3.4): kernel instantiations
// and the launcher used by the single-matrix path.
#include "sweep_launch.cuh"

namespace mpj {

static int try_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                   int phase, int gate_want, int w, int rpt, int threads)
{
#define MPJ_L(WW, RR) \
    if (w == WW && rpt == RR) return launch_sweeps_wr<double, true, WW, RR>(h, D, X, V, st, phase, gate_want, threads)
    MPJ_L(1, 2); MPJ_L(1, 4); MPJ_L(1, 8); MPJ_L(1, 16); MPJ_L(1, 32);
    MPJ_L(2, 2); MPJ_L(2, 4); MPJ_L(2, 8); MPJ_L(2, 16);
    MPJ_L(4, 2); MPJ_L(4, 4); MPJ_L(4, 8);
    MPJ_L(8, 2); MPJ_L(8, 4);
#undef MPJ_L
    return -1;
}

// Register-limited thread count of variant (w, rpt), 0 if it is not instantiated.
static int max_threads_f64(int w, int rpt)
{
    cudaFuncAttributes fa;
#define MPJ_Q(WW, RR) \
    if (w == WW && rpt == RR) return cudaFuncGetAttributes(&fa, k_sweeps<double, true, WW, RR>) == cudaSuccess ? fa.maxThreadsPerBlock : 0
    MPJ_Q(1, 2); MPJ_Q(1, 4); MPJ_Q(1, 8); MPJ_Q(1, 16); MPJ_Q(1, 32);
    MPJ_Q(2, 2); MPJ_Q(2, 4); MPJ_Q(2, 8); MPJ_Q(2, 16);
    MPJ_Q(4, 2); MPJ_Q(4, 4); MPJ_Q(4, 8);
    MPJ_Q(8, 2); MPJ_Q(8, 4);
#undef MPJ_Q
    return 0;
}

// Largest block width <= w_want (a power of two) with a variant whose register-resident
// visit holds mX rows (w * rpt <= 32 doubles per thread). 0: none.
int sweep_fit_w_f64(int mX, int w_want)
{
    for (int w = w_want; w >= 1; w /= 2)
        for (int rpt = 2; rpt <= 32 && w * rpt <= 32; rpt *= 2) {
            const int need = (mX + rpt - 1) / rpt;
            if (need > 1024) continue;
            const int mt = max_threads_f64(w, rpt);
            if (mt > 0 && sweep_threads(mX, rpt) <= mt) return w;
        }
    return 0;
}

// Block width w in {1, 2, 4, 8}; rows per thread chosen so that the visit's 2w columns fit
// in registers (w * rpt <= 32 doubles per thread), doubled while a variant's register use
// does not allow the thread count. Four rows per thread from w = 4 up (measured on the
// 1024-column refinement: w = 4 with 256 threads 25.6 ms, with 128 threads 27.9 ms, with 512
// threads 29.3 ms; w = 2 with 128 threads 27.6 ms).
int launch_sweeps_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                      int phase, int gate_want, int* threads_out)
{
    const int w = D.w;
    int rpt = sweep_rpt(D.mX, w >= 4 ? 4 : 8);
    while (w * rpt > 32 && rpt > 2) rpt /= 2;
    for (; rpt <= 32 && w * rpt <= 32; rpt *= 2) {
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
