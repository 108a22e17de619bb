// sweep_cl.cu -- cluster-split binary64 sweeps (sweep_cl.cuh): the choice of the cluster size
// and block width, the dispatch, and the block-width-4 kernels (widths 2 and 8 in
// sweep_cl_w2.cu, sweep_cl_w8.cu).
#include "sweep_cl.cuh"

namespace mpj {

template int launch_cl_w<4>(mpjsvd_ctx*, const SweepDims&, double*, double*, DevState*, int, int, int);

// CTAs per visit for mX rows at block width w (2, 4 or 8 CTAs; at least min_cs), 0 when the
// single-CTA visits are to be used. The preferred split leaves about kClPrefRows rows per CTA
// (at w = 4, 128 threads: two CTAs of different visits share an SM and hide each other's
// exchange and reduction latencies); measured on the large recipe (binary64 sweeps, w = 4):
// n = 4096 single-CTA visits (w = 2) 1032 ms, 2 CTAs per visit 907 ms, 4 CTAs 867 ms; n = 8192
// single-CTA (w = 1) 11843 ms, 4 CTAs 9042 ms, 8 CTAs 8852 ms; n = 2048 equal (104 / 102 ms),
// n = 1024 slower (18.6 ms single-CTA, 27.7 ms on 2 CTAs).
constexpr int kClPrefRows = 1024;

int sweep_cl_width(int block_w)
{
    return (block_w == 2 || block_w == 8) ? block_w : 4;
}

int sweep_cl_size(int mX, int work_kernel, int min_cs, int w)
{
    if (work_kernel == MPJSVD_WORKK_CTA) return 0;
    if (work_kernel == MPJSVD_WORKK_AUTO && mX <= cl_rows_per_cta(4)) return 0;
    const int lo = std::max(2, min_cs);
    for (int cs = lo; cs <= 8; cs *= 2)
        if ((mX + cs - 1) / cs <= kClPrefRows) return cs;
    for (int cs = lo; cs <= 8; cs *= 2)
        if ((mX + cs - 1) / cs <= cl_rows_per_cta(w)) return cs;
    return 0;
}

int launch_sweeps_f64_cl(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st, int phase,
                         int gate_want, int cs)
{
    if (phase == 0) return cuda_fail("cluster sweeps: binary64 stages only", cudaErrorInvalidValue);
    switch (D.w) {
    case 2: return launch_cl_w<2>(h, D, X, V, st, phase, gate_want, cs);
    case 4: return launch_cl_w<4>(h, D, X, V, st, phase, gate_want, cs);
    case 8: return launch_cl_w<8>(h, D, X, V, st, phase, gate_want, cs);
    default: return cuda_fail("cluster sweeps: block width", cudaErrorInvalidValue);
    }
}

}  // namespace mpj
