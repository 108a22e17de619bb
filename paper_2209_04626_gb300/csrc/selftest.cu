// selftest.cu -- a check of the failure detection of the bounded device waits (not part of
// the paper's method): every cross-CTA wait of the library gives up after the call's limit
// (params.wait_limit_ms), records MPJSVD_STATUS_TIMEOUT and returns, so the kernel exits and
// the context stays usable. This entry point makes such a wait run out on purpose, on a
// counter that nothing releases, with no fault and no unbounded spin.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"

namespace mpj {

// Two CTAs of one cooperative launch. CTA 0 waits (the sweeps' block hand-off, wait_blocks)
// for block 0 to reach version 1: ver[0] is 0 and nothing releases it, so the wait gives up
// after the limit and records the timeout. CTA 1 waits at the grid barrier (grid_sync) for
// CTA 0, which never arrives: it sees the timeout in the status word and leaves.
static __global__ void k_stalled_wait(unsigned* ver, DevState* st)
{
    const Group g{(int)blockIdx.x, (int)gridDim.x, st};
    if (blockIdx.x == 0 && !wait_blocks(ver, 0, 0, 1u, st)) return;
    g.sync();
}

static int selftest_timeout(mpjsvd_ctx* h)
{
    int rc = ensure_buffer(&h->ws, &h->ws_bytes, 256);
    if (rc) return rc;
    h->launch_count = 0;
    if ((rc = state_reset(h, h->dstate))) return rc;
    cudaError_t e = cudaMemsetAsync(h->ws, 0, 256, h->stream);
    if (e != cudaSuccess) return cuda_fail("selftest: memset", e);
    unsigned* ver = (unsigned*)h->ws;
    DevState* st = (DevState*)h->dstate;
    void* args[] = {&ver, &st};
    e = cudaLaunchCooperativeKernel((void*)k_stalled_wait, 2, 32, args, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail("selftest: launch", e);
    ++h->launch_count;
    return 0;
}

}  // namespace mpj

extern "C" int mpjsvd_selftest_timeout(mpjsvd_handle h)
{
    if (!h) return -1;
    return mpj::selftest_timeout(h);
}
