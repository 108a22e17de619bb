// sweep_f32.cu -- binary32 sweeps on low(X), no V (Section 3.2): kernel instantiations and
// the launcher used by the single-matrix path.
#include "sweep_launch.cuh"

namespace mpj {

static int try_f32(mpjsvd_ctx* h, const SweepDims& D, float* X, DevState* st, int phase,
                   int gate_want, int w, int rpt, int threads)
{
#define MPJ_L(WW, RR) \
    if (w == WW && rpt == RR) return launch_sweeps_wr<float, false, WW, RR>(h, D, X, nullptr, st, phase, gate_want, threads)
    MPJ_L(1, 2); MPJ_L(1, 4); MPJ_L(1, 8); MPJ_L(1, 16);
    MPJ_L(2, 2); MPJ_L(2, 4); MPJ_L(2, 8); MPJ_L(2, 16);
    MPJ_L(4, 2); MPJ_L(4, 4); MPJ_L(4, 8);
    MPJ_L(8, 2); MPJ_L(8, 4); MPJ_L(8, 8);
    MPJ_L(16, 2); MPJ_L(16, 4);
#undef MPJ_L
    return -1;
}

// Register-limited thread count of variant (w, rpt), 0 if it is not instantiated.
static int max_threads_f32(int w, int rpt)
{
    cudaFuncAttributes fa;
#define MPJ_Q(WW, RR) \
    if (w == WW && rpt == RR) return cudaFuncGetAttributes(&fa, k_sweeps<float, false, WW, RR>) == cudaSuccess ? fa.maxThreadsPerBlock : 0
    MPJ_Q(1, 2); MPJ_Q(1, 4); MPJ_Q(1, 8); MPJ_Q(1, 16);
    MPJ_Q(2, 2); MPJ_Q(2, 4); MPJ_Q(2, 8); MPJ_Q(2, 16);
    MPJ_Q(4, 2); MPJ_Q(4, 4); MPJ_Q(4, 8);
    MPJ_Q(8, 2); MPJ_Q(8, 4); MPJ_Q(8, 8);
    MPJ_Q(16, 2); MPJ_Q(16, 4);
#undef MPJ_Q
    return 0;
}

// Largest block width <= w_want (a power of two) with a variant whose register-resident
// visit holds mX rows: some rpt with w * rpt <= 64 and ceil(mX / rpt) threads allowed by the
// variant's register use. 0: none.
int sweep_fit_w_f32(int mX, int w_want)
{
    for (int w = w_want; w >= 1; w /= 2)
        for (int rpt = 2; rpt <= 16 && w * rpt <= 64; rpt *= 2) {
            const int need = (mX + rpt - 1) / rpt;
            if (need > 1024) continue;
            const int mt = max_threads_f32(w, rpt);
            if (mt > 0 && sweep_threads(mX, rpt) <= mt) return w;
        }
    return 0;
}

// Block width w in {1, 2, 4, 8, 16}; w * rpt <= 64 floats per thread.
int launch_sweeps_f32(mpjsvd_ctx* h, const SweepDims& D, float* X, DevState* st, int phase,
                      int gate_want, int* threads_out)
{
    const int w = D.w;
    int rpt = sweep_rpt(D.mX, 2);  // 512 threads at 1024 rows: 12.4 ms vs 12.9 ms with 256
    while (w * rpt > 64 && rpt > 2) rpt /= 2;
    for (; rpt <= 16 && w * rpt <= 64; rpt *= 2) {
        if ((D.mX + rpt - 1) / rpt > 1024) continue;
        const int threads = sweep_threads(D.mX, rpt);
        int rc = try_f32(h, D, X, st, phase, gate_want, w, rpt, threads);
        if (rc == kSweepTooManyThreads) continue;
        if (rc == -1) break;
        if (threads_out) *threads_out = threads;
        return rc;
    }
    return cuda_fail("sweep: no binary32 variant fits (block width, rows)", cudaErrorInvalidValue);
}

// The binary32 stage that also accumulates its rotations into V (binary64, n rows; the
// alternative switch of Section 3.3 takes the QR of that V). Block widths 4 and 8.
int launch_sweeps_f32v(mpjsvd_ctx* h, const SweepDims& D, float* X, double* V, DevState* st, int phase,
                       int gate_want)
{
    const int w = D.w >= 8 ? 8 : 4;
    SweepDims Dv = D;
    Dv.w = w;
    Dv.k = std::max(2, (D.n + w - 1) / w + (((D.n + w - 1) / w) & 1));
    for (int rpt = 2; rpt <= 8; rpt *= 2) {
        if ((D.mX + rpt - 1) / rpt > 1024) continue;
        const int threads = sweep_threads(D.mX, rpt);
        int rc = -1;
#define MPJ_V(WW, RR) \
        if (w == WW && rpt == RR) rc = launch_sweeps_wr<float, true, WW, RR>(h, Dv, X, V, st, phase, gate_want, threads)
        MPJ_V(4, 2); MPJ_V(4, 4); MPJ_V(4, 8);
        MPJ_V(8, 2); MPJ_V(8, 4); MPJ_V(8, 8);
#undef MPJ_V
        if (rc == kSweepTooManyThreads) continue;
        return rc;
    }
    return cuda_fail("sweep: no binary32 variant with V fits", cudaErrorInvalidValue);
}

}  // namespace mpj
