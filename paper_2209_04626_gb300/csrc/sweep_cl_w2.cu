// sweep_cl_w2.cu -- the cluster-split binary64 sweep kernels of block width 2 (sweep_cl.cuh).
#include "sweep_cl.cuh"

namespace mpj {

template int launch_cl_w<2>(mpjsvd_ctx*, const SweepDims&, double*, double*, DevState*, int, int, int);

}  // namespace mpj
