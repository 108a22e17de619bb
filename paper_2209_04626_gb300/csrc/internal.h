// internal.h -- host-side definitions shared by the translation units of libmpjsvd.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "mpjsvd.h"

struct mpjsvd_ctx {
    int device;
    int num_sms;
    cudaStream_t stream;
    mpjsvd_params params;
    // workspace (device), grown on demand
    void* ws;
    size_t ws_bytes;
    // per-call device state (mpj::DevState), separate allocation
    void* dstate;
    // batched path workspace
    void* bws;
    size_t bws_bytes;
    // backward path workspace
    void* aws;
    size_t aws_bytes;
    // timing events
    cudaEvent_t ev[8];
    bool have_events;
    // last call's stats with the phase times filled in on the host
    mpjsvd_stats last;
    bool last_valid;
    int last_block_w_low, last_block_w_work;
    int launch_count;  // kernels launched by the last call
};

namespace mpj {

// error bookkeeping (thread-local text of the last CUDA error)
void set_last_error(const char* where, cudaError_t e);
int cuda_fail(const char* where, cudaError_t e);

// grow a device buffer to at least `bytes`
int ensure_buffer(void** buf, size_t* cur, size_t bytes);

struct SweepDims;
struct DevState;

// sweep stages (sweep_f32.cu, sweep_f64.cu): one cooperative launch each
int launch_sweeps_f32(mpjsvd_ctx* h, const SweepDims& D, float* X, DevState* st, int phase,
                      int gate_want, int* threads_out);
int launch_sweeps_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                      int phase, int gate_want, int* threads_out);

// single-matrix pipeline (svd_single.cu)
int svd_single(mpjsvd_ctx* h, int m, int n, const double* A, int lda, double* U, double* S,
               double* V, double tol);
int read_stats(mpjsvd_ctx* h, mpjsvd_stats* st);

// batched pipeline (svd_batched.cu)
int svd_batched(mpjsvd_ctx* h, int batch, const int* m, const int* n, const int* lda,
                const double* const* A, double* const* U, double* const* S, double* const* V,
                double tol, int* info);

// adjoint (adjoint.cu)
int svd_backward(mpjsvd_ctx* h, int m, int n, const double* U, const double* S, const double* V,
                 const double* gU, const double* gS, const double* gV, double* gA, double gap_tol,
                 int* n_flagged);

}  // namespace mpj
