// common.cuh -- device helpers shared by the mpjsvd kernels (sm_103a).
//
// Matrices are column-major FP64 (LAPACK convention) unless a name says otherwise.
// Every wait in device code is bounded in time: a grid barrier gives up after the call's
// limit (params.wait_limit_ms, stored in DevState::spin_ns; kSpinLimitNs when unset),
// records MPJSVD_STATUS_TIMEOUT in the call's status word and returns false, so the kernel
// can exit and the context stays usable.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpjsvd.h"

namespace mpj {

constexpr int kWarp = 32;
constexpr uint64_t kSpinLimitNs = 4000000000ull;  // 4 s: the limit when none is set

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-call device state: barrier words, the status word and counters. Zeroed by the
// host at the start of every call (one cudaMemsetAsync).
struct DevState {
    unsigned int bar_count;
    unsigned int bar_gen;
    int status;            // MPJSVD_STATUS_* bits set by device code (atomicOr)
    int gate_low;          // 1: run the lower-precision stage (Alg. 4 branch decision)
    int branch;            // mpjsvd_stats.branch
    int sweeps_low;
    int sweeps_work;
    int pad0;
    unsigned long long rot_low;
    unsigned long long rot_work;
    double cond_r;
    double orth;
    double maxnorm;        // max column norm of X (branch test)
    unsigned long long rot_sweep[3][64];   // rotations per sweep, [phase][sweep]
    double2 cand[512];                     // QRCP: per-CTA candidate (norm, column) x parity
    unsigned long long amax_bits;          // Alg. 5: max |a_ij| (bits of a non-negative double)
    unsigned long long cand_rec[512];      // Alg. 5: per-CTA step records (tag, column, norm) x parity
    unsigned mx_cos[3][64];                // binary32 bits: largest cosine among the rotated pairs, [phase][sweep]
    unsigned mx_tan[3][64];                // binary32 bits: largest |tan| of the rotations, [phase][sweep]
    unsigned long long spin_ns;            // limit of every bounded wait of the call (0: kSpinLimitNs)
    int gate_lq;                           // 1: the Jacobi input is X = L (second preconditioning)
    int gate_y2;                           // 1: the Y1/Y2 safeguard found columns to treat first
    int y_j0;                              // first column of Y2 (n: none)
    int y2_cols_n;                         // n of the safeguard's partition
    int sweeps_v;                          // phase 2 (safeguard passes, final pass of V from QR)
    unsigned long long rot_v;
};

// The call's wait limit in nanoseconds.
__device__ __forceinline__ uint64_t spin_limit_ns(const DevState* st)
{
    const uint64_t v = *(volatile const unsigned long long*)&st->spin_ns;
    return v ? v : kSpinLimitNs;
}

// Gates of stages whose execution is decided on the device. gate_want: -1 always; 0 / 1 run
// only when gate_low (the lower-precision stage of Alg. 4) has that value; kGateLq + 0 / 1: by
// gate_lq (the second preconditioning of Alg. 2); kGateY2 + 0 / 1: by gate_y2 (the Y1/Y2
// safeguard).
constexpr int kGateLq = 2;
constexpr int kGateY2 = 4;
__device__ __forceinline__ bool gate_open(const DevState* st, int gate_want)
{
    if (gate_want < 0) return true;
    if (gate_want >= kGateY2) return *(volatile const int*)&st->gate_y2 == gate_want - kGateY2;
    if (gate_want >= kGateLq) return *(volatile const int*)&st->gate_lq == gate_want - kGateLq;
    return *(volatile const int*)&st->gate_low == gate_want;
}

// True once the call cannot produce meaningful output: a non-finite input, or a cooperative
// stage that gave up on a bounded wait. Later stages then return at once.
__device__ __forceinline__ bool call_failed(const DevState* st)
{
    return (*(volatile const int*)&st->status &
            (MPJSVD_STATUS_NONFINITE | MPJSVD_STATUS_TIMEOUT)) != 0;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier for a cooperative launch (all CTAs co-resident). Returns false
// if the wait timed out or another CTA reported an error; callers then exit.
// Thread 0 arrives with an acq_rel atomic (after the CTA barrier, so the release covers every
// thread's earlier writes); the last arrival resets the count and releases the next
// generation; the others spin on an acquire load of the generation (no sleep: the wait is
// usually well under a microsecond), checking the time limit every 1024 polls.
__device__ __forceinline__ bool grid_sync(DevState* st)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_gpu(&st->bar_gen);
        unsigned arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&st->bar_count) : "memory");
        if (arrived == gridDim.x - 1) {
            st->bar_count = 0;
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&st->bar_gen), "r"(gen + 1) : "memory");
        } else {
            const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
            unsigned spins = 0;
            while (ld_acquire_gpu(&st->bar_gen) == gen) {
                if ((++spins & 1023u) == 0) {
                    if (globaltimer_ns() - t0 > lim) {
                        atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (*(volatile int*)&st->status & MPJSVD_STATUS_TIMEOUT) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (*(volatile int*)&st->status & MPJSVD_STATUS_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// A "group" is the set of CTAs that cooperate on one matrix: all CTAs of a cooperative
// launch (single-matrix path) or one CTA (batched path, where sync is __syncthreads).
struct Group {
    int rank;        // this CTA's index in the group
    int size;        // number of CTAs in the group
    DevState* st;    // barrier/status state (single-matrix path), may be null if size == 1
    __device__ __forceinline__ bool sync() const
    {
        if (size == 1) {
            __syncthreads();
            return true;
        }
        return grid_sync(st);
    }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; every thread gets the result. scratch: >= 32 elements of T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T r = (lane < nw) ? scratch[lane] : T(0);
    r = warp_sum(r);
    return r;
}

__device__ __forceinline__ size_t cm(int i, int j, int ld) { return (size_t)j * (size_t)ld + (size_t)i; }

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// Warp reduction of N values per lane (N a power of two <= 32). Afterwards v[0] of lane l
// holds the warp-wide sum of value index (l >> (5 - log2 N)) (index 0 for N = 1). Costs
// N - 1 + 5 - log2 N additions per lane instead of 5 N for N separate butterflies, which
// matters where every FP64 addition occupies the scarce FP64 pipe.
template <int N, typename T>
__device__ __forceinline__ void warp_reduce_multi(T (&v)[N], int lane)
{
    constexpr int L = ilog2c(N);
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int o = 16 >> k;
        const int half = N >> (k + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            T send = upper ? v[i] : v[i + half];
            T keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> L; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

// Sum N values (N a power of two <= 32) over the CTA; every thread receives the N sums in
// out[]. red: shared scratch of >= 33 * N elements.
template <int N, typename T>
__device__ __forceinline__ void block_sum_multi(T (&v)[N], T* red, T (&out)[N])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int sh = 5 - ilog2c(N);
    warp_reduce_multi<N>(v, lane);
    __syncthreads();
    if ((lane & ((1 << sh) - 1)) == 0) red[(lane >> sh) * 32 + wid] = v[0];
    __syncthreads();
    if (threadIdx.x < N) {
        T s = T(0);
        for (int k = 0; k < nw; ++k) s += red[threadIdx.x * 32 + k];
        red[N * 32 + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < N; ++b) out[b] = red[N * 32 + b];
}

}  // namespace mpj
