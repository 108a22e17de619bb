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
    int last_work_cs;  // CTAs per visit of the last call's binary64 sweeps
    int launch_count;  // kernels launched by the last call
    int last_qrcp;     // MPJSVD_QRCP_* that the last call ran
    int last_precond;  // MPJSVD_PRECOND_* of the last call (AUTO resolved from the device)
    int* last_flag_dev;  // device count of near-degenerate flags of the last svd_backward
    // batched autotuner: per size class of n (<= 32, 64, 128, 256, 512), the kernel variant
    // (block widths of the two Jacobi stages) picked by timing, and its sample time
    bool bt_tuned[5];
    int bt_variant[5];
    float bt_ms[5];
    // the blocked QR's look-ahead: the critical chain (panels and the updates of the next
    // panel) on a high-priority stream, the wide trailing updates on a low-priority one;
    // both fork from and join back into `stream` through events
    cudaStream_t side;   // lowest priority: wide updates
    cudaStream_t crit;   // highest priority: panels and narrow updates
    cudaEvent_t qev[7];  // [0] panel done, [1..3] wide updates (ring), [4] side join,
                         // [5] fork, [6] critical-chain join
    bool have_side;
};

namespace mpj {

// error bookkeeping (thread-local text of the last CUDA error)
void set_last_error(const char* where, cudaError_t e);
int cuda_fail(const char* where, cudaError_t e);

// zero the per-call state block (DevState) on the handle's stream and store the call's wait
// limit in it
int state_reset(mpjsvd_ctx* h, void* st);

// grow a device buffer to at least `bytes`
int ensure_buffer(void** buf, size_t* cur, size_t bytes);

struct SweepDims;
struct DevState;

// sweep stages (sweep_f32.cu, sweep_f64.cu): one cooperative launch each
int launch_sweeps_f32(mpjsvd_ctx* h, const SweepDims& D, float* X, DevState* st, int phase,
                      int gate_want, int* threads_out);
int launch_sweeps_f64(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st,
                      int phase, int gate_want, int* threads_out);
int launch_sweeps_f32v(mpjsvd_ctx* h, const SweepDims& D, float* X, double* V, DevState* st, int phase,
                       int gate_want);
// the binary32 stage in blocked form on the tensor cores (bsweep_tc.cu): block width 64
int launch_bsweeps_tf32(mpjsvd_ctx* h, const SweepDims& D, float* X, DevState* st, int phase,
                        int gate_want);
// its building blocks as a standalone call: G = Z^T Z and / or Z <- Z W for a 128-column Z
int tc_block_call(mpjsvd_ctx* h, int m, float* Z, int ldz, float* G, const float* W);
// largest block width <= w_want whose register-resident visit holds mX rows (0: none)
int sweep_fit_w_f32(int mX, int w_want);
int sweep_fit_w_f64(int mX, int w_want);
// binary64 sweeps with every visit split by rows over a cluster of cs CTAs (sweep_cl.cu):
// cs for mX rows under params.work_kernel (0: one CTA per visit), the block width, and the
// launch (1 = cluster launch unavailable here, nothing launched)
int sweep_cl_width(int block_w);
int sweep_cl_size(int mX, int work_kernel, int min_cs, int w);
int launch_sweeps_f64_cl(mpjsvd_ctx* h, const SweepDims& D, double* X, double* V, DevState* st, int phase,
                         int gate_want, int cs);

// blocked Householder QR and compact-WY application of Q (qr_blocked.cu)
int bqr_nb(int m);                       // panel width for m rows; 0: use the unblocked kernels
size_t bqr_wbuf_doubles(int ncols_max, int m_max);  // scratch of the one-level bqr_factor / bqr_apply
// two-level form (qr_outer.cu): 256-column outer blocks, their trailing updates and the
// applications of Q on the tensor cores; used by bqr_factor / bqr_apply when bqr_outer_used
// Where a QR or an application of Q sits in the pipeline: the automatic choice takes the
// tensor cores only where the operands are scaled column by column (the preconditioner's A P,
// U = Q [U_R; 0]); the switch's QR of B (rows graded like X) stays on the FP64 pipe.
enum QrSite { kQrSitePrecond = 0, kQrSiteSwitch = 1, kQrSiteFinal = 2, kQrSiteCall = 3 };
constexpr int kQrOuterMinNFactor = 6144;  // automatic choice: preconditioner QR from this n on
constexpr int kQrOuterMinNApply = 4096;   // automatic choice: U assembly / standalone from this n on
bool bqr_outer_used(const mpjsvd_ctx* h, int m, int n, int site);
size_t bqr_outer_ws_bytes(int m, int n);           // its scratch (bytes)
// scratch bytes bqr_factor / bqr_apply need for m rows and n columns (or reflectors), any site
size_t bqr_ws_bytes(const mpjsvd_ctx* h, int m, int n);
int bqr_factor_outer(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau, void* W, DevState* st,
                     int gate_want);
int bqr_apply_outer(mpjsvd_ctx* h, int m, int ncols, int k, const double* V, int ldv, const double* tau, double* C,
                    int ldc, bool ident, void* W, DevState* st, int gate_want);
struct GemmArgs;
int launch_gemm_d(mpjsvd_ctx* h, const GemmArgs& g, const int* gate, int want);  // binary64 SIMT product
int bqr_factor(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau, double* W, DevState* st,
               int gate_want, int site = kQrSiteCall);
int bqr_apply(mpjsvd_ctx* h, int m, int ncols, int k, const double* V, int ldv, const double* tau,
              double* C, int ldc, bool ident, double* W, DevState* st, int gate_want, int site = kQrSiteCall);
// binary32 pivot search of Alg. 5 (qrcp_low.cu); 1 = does not fit, nothing launched
int launch_qrcp_low(mpjsvd_ctx* h, int m, int n, const double* A, int lda, int* perm, float* bcast,
                    size_t bcast_bytes, DevState* st);
size_t qrcp_low_bcast_bytes(int m, int n, int sms);  // what its global-column variant needs

// standalone calls behind mpjsvd_geqrf / mpjsvd_apply_q (workspace and state of the handle)
int qr_call(mpjsvd_ctx* h, int m, int n, double* A, int lda, double* tau);
int apply_q_call(mpjsvd_ctx* h, int m, int ncols, int k, const double* A, int lda, const double* tau,
                 double* C, int ldc);

// single-matrix pipeline (svd_single.cu)
int svd_single(mpjsvd_ctx* h, int m, int n, const double* A, int lda, double* U, double* S,
               double* V, double tol);
int read_stats(mpjsvd_ctx* h, mpjsvd_stats* st);
int geqp3_call(mpjsvd_ctx* h, int m, int n, double* A, int lda, int* jpvt, double* tau);

// batched pipeline (svd_batched.cu)
int svd_batched(mpjsvd_ctx* h, int batch, const int* m, const int* n, const int* lda,
                const double* const* A, double* const* U, double* const* S, double* const* V,
                double tol, int* info);

int svd_batched_dev(mpjsvd_ctx* h, int batch, int max_m, int max_n, const int* m, const int* n, const int* lda,
                    const double* const* A, double* const* U, double* const* S, double* const* V, double tol,
                    int* info);
void batched_tuning(const mpjsvd_ctx* h, int* w_low, int* w_work, float* ms);

// binary64 products on the bf16 tensor cores by operand splitting (ozaki.cu)
struct GemmArgs;
size_t ozaki_ws_bytes(int M, int N, int K);
int ozaki_dgemm(mpjsvd_ctx* h, const GemmArgs& g, void* ws, const int* gate, int want, DevState* st);

// adjoint (adjoint.cu)
int svd_backward(mpjsvd_ctx* h, int m, int n, const double* U, const double* S, const double* V,
                 const double* gU, const double* gS, const double* gV, double* gA, double gap_tol,
                 int* n_flagged);
int svd_backward_batched(mpjsvd_ctx* h, int batch, const int* m, const int* n,
                         const double* const* U, const double* const* S, const double* const* V,
                         const double* const* gU, const double* const* gS, const double* const* gV,
                         double* const* gA, double gap_tol, int* n_flagged);

}  // namespace mpj
