// svd_batched.cu -- placeholder until the persistent batched kernel lands.
#include "internal.h"

namespace mpj {

int svd_batched(mpjsvd_ctx*, int, const int*, const int*, const int*, const double* const*,
                double* const*, double* const*, double* const*, double, int*)
{
    set_last_error("mpjsvd_svd_batched", cudaErrorNotSupported);
    return MPJSVD_ERR_CUDA;
}

}  // namespace mpj
