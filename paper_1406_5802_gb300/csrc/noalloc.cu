// noalloc.cu -- rmge_solve_noalloc: rmge_solve with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the point where they solve: code that must not
// touch the device allocator after start-up (a latency-bound serving loop, where cudaMalloc can
// synchronise the device), or a plugin whose host process owns every allocation and hands it
// only the inputs and outputs.  This entry point serves them: the workspace rmge_solve needs comes
// from a file-scope __device__ array of RMGE_NOALLOC_WS_BYTES, which every GPU that has made a call
// holds until the process exits.  The entry point itself calls no cudaMalloc, cudaFree
// or other allocating routine.
//
// The array's name is, in host code, only a host-side stand-in for the symbol; its device address is
// looked up with cudaGetSymbolAddress, with the calling device current, on every call (a cheap lookup
// once the module is loaded, and never stale: a cached address would outlive a cudaDeviceReset or a
// re-created primary context).  The module holding the array loads lazily (CUDA's default module
// loading): the first call on each device loads it, which allocates the array and may synchronise the
// device, so callers make one call at start-up, before any stream capture or latency-bound loop.  All
// calls share the one array: rmge_solve clears the parts that must start at zero (the control block and
// the solve flags) at the start of each call, in stream order, and calls that overlap on the GPU
// (different streams, or different host threads) race on it.
#include "kernels.cuh"

#define RMGE_NOALLOC_WS_BYTES ((size_t)16 << 20)

namespace {

__device__ __align__(256) unsigned char g_noalloc_ws[RMGE_NOALLOC_WS_BYTES];

// Device address of g_noalloc_ws on the current device; NULL on failure.
void* noalloc_ws_address() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

}  // namespace

extern "C" {

size_t rmge_noalloc_capacity(void) { return RMGE_NOALLOC_WS_BYTES; }

rmge_status rmge_solve_noalloc(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu,
                               const void* G, const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                               rmge_stream_t stream) {
    const size_t need = rmge_solve_workspace_size(n, nrhs, kind, prec);
    if (need == 0) return RMGE_ERR_INVALID_ARG;
    if (need > RMGE_NOALLOC_WS_BYTES) return RMGE_ERR_WORKSPACE;
    void* ws = noalloc_ws_address();
    if (ws == nullptr) return RMGE_ERR_CUDA;
    return rmge_solve(kind, n, nrhs, LU, ldlu, G, B, ldb, X, ldx, prec, ws, RMGE_NOALLOC_WS_BYTES, stream);
}

}  // extern "C"
