// api.cu -- the extern "C" entry points declared in include/mpjsvd.h: argument validation,
// the handle and its workspace; the work itself is in svd_single.cu, svd_batched.cu and
// adjoint.cu.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.h"

namespace mpj {

static thread_local char g_last_error[256] = "no error";

void set_last_error(const char* where, cudaError_t e)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}

int cuda_fail(const char* where, cudaError_t e)
{
    set_last_error(where, e);
    return MPJSVD_ERR_CUDA;
}

// Zero the per-call state block and store the call's wait limit in it (one small kernel).
static __global__ void k_state_reset(DevState* st, unsigned long long spin_ns)
{
    for (size_t i = threadIdx.x; i < sizeof(DevState) / 4; i += blockDim.x) ((int*)st)[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) st->spin_ns = spin_ns;
}

int state_reset(mpjsvd_ctx* h, void* st)
{
    const unsigned long long ns = (unsigned long long)h->params.wait_limit_ms * 1000000ull;
    k_state_reset<<<1, 256, 0, h->stream>>>((DevState*)st, ns);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("state reset", e);
    ++h->launch_count;
    return 0;
}

int ensure_buffer(void** buf, size_t* cur, size_t bytes)
{
    if (*buf && *cur >= bytes) return 0;
    if (*buf) {
        cudaError_t e = cudaFree(*buf);
        *buf = nullptr;
        *cur = 0;
        if (e != cudaSuccess) return cuda_fail("workspace free", e);
    }
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        *buf = nullptr;
        set_last_error("workspace cudaMalloc", e);
        cudaGetLastError();
        return MPJSVD_ERR_NOMEM;
    }
    *cur = bytes;
    return 0;
}

}  // namespace mpj

using namespace mpj;

extern "C" {

int mpjsvd_default_params(mpjsvd_params* p)
{
    if (!p) return -1;
    p->tol_alg = 1e-2;
    p->tol_orth = 1e-5;
    p->tol_cond_coef = 1.5;
    p->trailing_frac = 0.25;
    p->maxsweep = 30;
    p->block_w = 0;
    p->mode = MPJSVD_MODE_AUTO;
    p->precond = MPJSVD_PRECOND_RT;
    p->qr_first = 0;
    p->timing = 0;
    p->qrcp = MPJSVD_QRCP_MIXED;
    p->stop = MPJSVD_STOP_XGESVJ;
    p->wait_limit_ms = 4000;
    p->low_kernel = MPJSVD_LOWK_AUTO;
    p->v_by_qr = 0;
    p->switch_method = MPJSVD_SWITCH_U;
    p->gemm_kernel = MPJSVD_GEMMK_AUTO;
    p->y_tol = 0.0;
    p->work_kernel = MPJSVD_WORKK_AUTO;
    p->work_cluster = 0;
    p->qr_update = MPJSVD_QRU_AUTO;
    return 0;
}

static int check_params(const mpjsvd_params* p)
{
    if (p->maxsweep < 1 || p->maxsweep > 64) return 1;
    if (p->block_w < 0 || p->block_w > 16) return 1;
    if (p->mode < 0 || p->mode > 2) return 1;
    if (p->precond < 0 || p->precond > 3) return 1;
    if (p->qrcp < 0 || p->qrcp > 1) return 1;
    if (p->stop < 0 || p->stop > 1) return 1;
    if (!(p->trailing_frac >= 0.0 && p->trailing_frac <= 1.0)) return 1;
    if (p->wait_limit_ms < 1 || p->wait_limit_ms > 600000) return 1;
    if (p->low_kernel < 0 || p->low_kernel > 2) return 1;
    if (p->v_by_qr < 0 || p->v_by_qr > 1) return 1;
    if (p->switch_method < 0 || p->switch_method > 1) return 1;
    if (p->gemm_kernel < 0 || p->gemm_kernel > 2) return 1;
    if (!(p->y_tol >= 0.0 && p->y_tol < 1.0)) return 1;
    if (p->work_kernel < 0 || p->work_kernel > 2) return 1;
    if (p->work_cluster != 0 && p->work_cluster != 2 && p->work_cluster != 4 && p->work_cluster != 8) return 1;
    if (p->qr_update < 0 || p->qr_update > 2) return 1;
    return 0;
}

int mpjsvd_create(mpjsvd_handle* h, const mpjsvd_params* p, void* cuda_stream)
{
    if (!h) return -1;
    *h = nullptr;
    mpjsvd_params prm;
    if (p) prm = *p;
    else mpjsvd_default_params(&prm);
    if (check_params(&prm)) return -2;
    mpjsvd_ctx* c = new (std::nothrow) mpjsvd_ctx();
    if (!c) return MPJSVD_ERR_NOMEM;
    memset(c, 0, sizeof(*c));
    c->params = prm;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { delete c; return cuda_fail("cudaGetDevice", e); }
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) { delete c; return cuda_fail("SM count", e); }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (!coop) { delete c; return cuda_fail("cooperative launch unsupported", cudaErrorNotSupported); }
    e = cudaMalloc(&c->dstate, sizeof(DevState));
    if (e != cudaSuccess) { delete c; set_last_error("state cudaMalloc", e); return MPJSVD_ERR_NOMEM; }
    c->have_events = true;
    for (int i = 0; i < 8 && c->have_events; ++i)
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(c->ev[k]);
            c->have_events = false;
        }
    // look-ahead streams: when both CTAs of the critical chain and of a wide update are
    // waiting for an SM, the critical chain's go first
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    c->have_side = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_lo) == cudaSuccess;
    if (c->have_side && cudaStreamCreateWithPriority(&c->crit, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
        cudaStreamDestroy(c->side);
        c->have_side = false;
    }
    for (int i = 0; i < 7 && c->have_side; ++i)
        if (cudaEventCreateWithFlags(&c->qev[i], cudaEventDisableTiming) != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(c->qev[k]);
            cudaStreamDestroy(c->side);
            cudaStreamDestroy(c->crit);
            c->have_side = false;
        }
    cudaGetLastError();  // a failed optional resource leaves no sticky error behind
    *h = c;
    return 0;
}

int mpjsvd_set_stream(mpjsvd_handle h, void* cuda_stream)
{
    if (!h) return -1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (s == h->stream) return 0;
    // the workspace is shared by all calls of the handle: the new stream waits (on the device)
    // for the work already queued on the previous one before a call reuses it
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);  // released once the wait has been satisfied
    if (e != cudaSuccess) return cuda_fail("set_stream: order after the previous stream", e);
    h->stream = s;
    return 0;
}

int mpjsvd_set_params(mpjsvd_handle h, const mpjsvd_params* p)
{
    if (!h) return -1;
    if (!p || check_params(p)) return -2;
    h->params = *p;
    return 0;
}

int mpjsvd_svd(mpjsvd_handle h, int m, int n, const double* A, int lda, double* U, double* S,
               double* V, double tol)
{
    if (!h) return -1;
    if (m < 1 || m < n || m > 24576) return -2;
    if (n < 1 || n > 8192) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (!U) return -6;
    if (!S) return -7;
    if (!V) return -8;
    if (!(tol <= 0.0 || (tol > 0.0 && tol < 1.0))) return -9;
    int d = -1;
    cudaGetDevice(&d);
    if (d != h->device) return cuda_fail("mpjsvd_svd: current device differs from the handle's", cudaErrorInvalidDevice);
    int rc = svd_single(h, m, n, A, lda, U, S, V, tol);
    h->last_valid = (rc == 0);
    return rc;
}

int mpjsvd_svd_batched(mpjsvd_handle h, int batch, const int* m, const int* n, const int* lda,
                       const double* const* A, double* const* U, double* const* S,
                       double* const* V, double tol, int* info)
{
    if (!h) return -1;
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    if (!m) return -3;
    if (!n) return -4;
    if (!lda) return -5;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 512) return -4;
        if (m[i] < n[i] || m[i] > 1024) return -3;
        if (lda[i] < m[i]) return -5;
    }
    if (!A) return -6;
    if (!U) return -7;
    if (!S) return -8;
    if (!V) return -9;
    if (!(tol <= 0.0 || (tol > 0.0 && tol < 1.0))) return -10;
    if (!info) return -11;
    if (h->params.precond > MPJSVD_PRECOND_R) {
        set_last_error("mpjsvd_svd_batched: params.precond L and AUTO are single-matrix only",
                       cudaErrorInvalidValue);
        return -1;
    }
    return svd_batched(h, batch, m, n, lda, A, U, S, V, tol, info);
}

int mpjsvd_svd_batched_dev(mpjsvd_handle h, int batch, int max_m, int max_n, const int* m, const int* n,
                           const int* lda, const double* const* A, double* const* U, double* const* S,
                           double* const* V, double tol, int* info)
{
    if (!h) return -1;
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    if (max_m < 1 || max_m > 1024) return -3;
    if (max_n < 1 || max_n > 512 || max_n > max_m) return -4;
    if (!m) return -5;
    if (!n) return -6;
    if (!lda) return -7;
    if (!A) return -8;
    if (!U) return -9;
    if (!S) return -10;
    if (!V) return -11;
    if (!(tol <= 0.0 || (tol > 0.0 && tol < 1.0))) return -12;
    if (!info) return -13;
    if (h->params.precond > MPJSVD_PRECOND_R) {
        set_last_error("mpjsvd_svd_batched_dev: params.precond L and AUTO are single-matrix only",
                       cudaErrorInvalidValue);
        return -1;
    }
    return svd_batched_dev(h, batch, max_m, max_n, m, n, lda, A, U, S, V, tol, info);
}

int mpjsvd_get_batched_tuning(mpjsvd_handle h, int* w_low, int* w_work, float* ms)
{
    if (!h) return -1;
    batched_tuning(h, w_low, w_work, ms);
    return 0;
}

int mpjsvd_svd_backward(mpjsvd_handle h, int m, int n, const double* U, const double* S,
                        const double* V, const double* gU, const double* gS, const double* gV,
                        double* gA, double gap_tol, int* n_flagged)
{
    if (!h) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1 || n > 16384) return -3;
    if (!U) return -4;
    if (!S) return -5;
    if (!V) return -6;
    if (!gA) return -10;
    if (!(gap_tol >= 0.0)) return -11;
    return svd_backward(h, m, n, U, S, V, gU, gS, gV, gA, gap_tol, n_flagged);
}

int mpjsvd_svd_backward_batched(mpjsvd_handle h, int batch, const int* m, const int* n,
                                const double* const* U, const double* const* S,
                                const double* const* V, const double* const* gU,
                                const double* const* gS, const double* const* gV,
                                double* const* gA, double gap_tol, int* n_flagged)
{
    if (!h) return -1;
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    if (!m) return -3;
    if (!n) return -4;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 512) return -4;
        if (m[i] < n[i] || m[i] > 4096) return -3;
    }
    if (!U) return -5;
    if (!S) return -6;
    if (!V) return -7;
    if (!gA) return -11;
    if (!(gap_tol >= 0.0)) return -12;
    if (!n_flagged) return -13;
    return svd_backward_batched(h, batch, m, n, U, S, V, gU, gS, gV, gA, gap_tol, n_flagged);
}

int mpjsvd_geqrf(mpjsvd_handle h, int m, int n, double* A, int lda, double* tau)
{
    if (!h) return -1;
    if (m < 1 || m < n || m > 12480 || mpj::bqr_nb(m) == 0) return -2;
    if (n < 1 || n > 12288) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (!tau) return -6;
    return mpj::qr_call(h, m, n, A, lda, tau);
}

int mpjsvd_geqp3(mpjsvd_handle h, int m, int n, double* A, int lda, int* jpvt, double* tau)
{
    if (!h) return -1;
    if (m < 1 || m < n || m > 24576) return -2;
    if (n < 1 || n > 12288) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (!jpvt) return -6;
    if (!tau) return -7;
    return mpj::geqp3_call(h, m, n, A, lda, jpvt, tau);
}

int mpjsvd_apply_q(mpjsvd_handle h, int m, int ncols, int k, const double* A, int lda,
                   const double* tau, double* C, int ldc)
{
    if (!h) return -1;
    if (m < 1 || m > 12480) return -2;
    if (ncols < 1 || ncols > 12288) return -3;
    if (k < 1 || k > m) return -4;
    if (!A) return -5;
    if (lda < m) return -6;
    if (!tau) return -7;
    if (!C) return -8;
    if (ldc < m) return -9;
    return mpj::apply_q_call(h, m, ncols, k, A, lda, tau, C, ldc);
}

int mpjsvd_get_stats(mpjsvd_handle h, mpjsvd_stats* st)
{
    if (!h) return -1;
    if (!st) return -2;
    return read_stats(h, st);
}

int mpjsvd_destroy(mpjsvd_handle h)
{
    if (!h) return -1;
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->bws) cudaFree(h->bws);
    if (h->aws) cudaFree(h->aws);
    if (h->dstate) cudaFree(h->dstate);
    if (h->have_side) {
        cudaStreamSynchronize(h->side);
        cudaStreamSynchronize(h->crit);
        for (int i = 0; i < 7; ++i) cudaEventDestroy(h->qev[i]);
        cudaStreamDestroy(h->side);
        cudaStreamDestroy(h->crit);
    }
    if (h->have_events)
        for (int i = 0; i < 8; ++i) cudaEventDestroy(h->ev[i]);
    delete h;
    return 0;
}

const char* mpjsvd_last_error(void) { return g_last_error; }

}  // extern "C"
