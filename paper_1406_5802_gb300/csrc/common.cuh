// common.cuh -- shared definitions of the librmge CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/rmge.h"

namespace rmge {

// ------------------------------------------------------------------------------------------
// Device control block, at the start of every workspace.  Zeroed/initialised by the host-side
// driver of each call with one small kernel; kernels communicate through it (breakdown step,
// stop flags, reductions) so that no call has to synchronise the stream.
// ------------------------------------------------------------------------------------------
struct DevState {
    int info;            // first breakdown step (1-based), INT32_MAX while none
    int halt;            // nonzero: factorization steps skip their work (set on breakdown)
    int stop;            // nonzero: refinement has stopped; sweep kernels skip their work
    int sweeps;          // refinement sweeps performed
    int error;           // RMGE_ERR_TIMEOUT etc. from bounded device waits, 0 if none
    int pad0;
    unsigned long long maxabs_m;   // bits of max |M| (non-negative doubles order like integers)
    unsigned long long maxabs_u;   // bits of max |U|
    double norm_a;                 // ||A||_inf
    double berr_prev;              // backward error two sweeps back (stagnation test)
    double berr_last;              // latest backward error
    unsigned int ticket;           // dynamic block-order ticket of the running triangular solve
    unsigned int done;             // CTAs of the running triangular solve that have finished
    long long spin_limit;          // polls of a bounded wait before it gives up (set by state_init)
    // reduced-precision refinement: classical sweeps until one fails to halve the backward error,
    // then FGMRES cycles; the two corrections of a sweep read these as their skip flags
    int krylov;        // nonzero once the sweeps have switched to FGMRES cycles
    int krylov_start;  // the sweep at which they switched
    int skip_cls;      // stop || krylov
    int skip_kry;      // stop || !krylov
    int nonfinite;     // nonzero once a scanned result held an Inf or NaN
    int status;        // the call's outcome as an rmge_status, written by its last kernel
};
static_assert(sizeof(DevState) <= 256, "the control block fits its 256-byte slot");

// Triangular-solve tiling (rows per block, right-hand sides per block column).
constexpr int kTrsvRows = 64;
constexpr int kTrsvCols = 2;
constexpr int kLowRankMaxL = 64;  // columns of the low-rank basis (Algorithm 6.1's l)
// Refinement sweeps one rmge_refine call may run.
constexpr int kMaxSweeps = 64;
// Restart length of the FGMRES cycles used as refinement sweeps for reduced-precision factors
// (default; rmge_options.gmres_m chooses another, up to kMaxGmresM).
constexpr int kGmresM = 16;
constexpr int kMaxGmresM = 256;
// Default spin limit of the bounded device waits of the triangular solves and the batched solve (about
// a second at their back-off); rmge_options.spin_limit overrides it.
constexpr long long kSpinLimit = 1LL << 22;

// Pivot block width of the blocked GENP.
constexpr int kNb = 64;

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout (byte offsets from ws).
struct WsLayout {
    size_t state;     // DevState
    size_t flags;     // int per (row block, column block): triangular-solve completion epochs
    size_t rowsum;    // n doubles
    size_t colred;    // 4 * nrhs doubles (max|r|, max|x|, max|b|, spare) as ull bits
    size_t R;         // n * nrhs doubles (residual / FP64 work)
    size_t Y;         // n * nrhs doubles (FP64 work) or floats
    size_t D;         // n * nrhs doubles
    size_t fft;       // circulant work: twiddle table
    size_t tcmx;      // FP16 operand-scaling slots (tensor-core precisions)
    size_t tc;        // 16-bit operand buffers (tensor-core precisions)
    size_t gm;        // FGMRES work (reduced precisions)
    size_t oz;        // digit planes of the emulated FP64 products
    size_t total;
};

WsLayout ws_layout(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec, int gmres_m = kGmresM);

// ------------------------------------------------------------------------------------------
// Small device helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Kernel launches enqueued by this process (reported by rmge_kernel_launches).
extern std::atomic<unsigned long long> g_launches;

}  // namespace rmge

// Host-side launch check, placed after every kernel launch: counts the launch and turns a failed
// launch into RMGE_ERR_CUDA.
#define RMGE_LAUNCH_CHECK()                                         \
    do {                                                            \
        rmge::g_launches.fetch_add(1, std::memory_order_relaxed);   \
        if (cudaPeekAtLastError() != cudaSuccess) {                 \
            (void)cudaGetLastError();                               \
            return RMGE_ERR_CUDA;                                   \
        }                                                           \
    } while (0)

#define RMGE_TRY(...)                           \
    do {                                        \
        rmge_status _s = (__VA_ARGS__);         \
        if (_s != RMGE_OK) return _s;           \
    } while (0)
