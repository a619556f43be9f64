// launch_timing.cu -- CUDA event pairs around the emulated Schur-update launches (rmge_launch_timing).
//
// GENP's Schur updates (Sec. 3) are launched inside rmge_factor*, so a caller's own events can only bracket
// the whole factorization.  While recording is on, each update launch records an event pair on its own
// stream; rmge_launch_timing_read sums their elapsed times per launch class.  Host code only.
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace rmge {

namespace {

struct Record {
    int kernel;
    cudaEvent_t begin, end;
    double flops;
    bool ended;
};

constexpr size_t kMaxRecords = 65536;
constexpr int kTimedKernels = 2;

std::mutex g_mu;
bool g_on = false;
uint32_t g_generation = 0;           // bumped by every reset, so that stale tokens record nothing
std::vector<Record> g_records;       // launches recorded since the last reset
std::vector<cudaEvent_t> g_spare;    // created events kept for reuse

cudaEvent_t take_event() {
    if (!g_spare.empty()) {
        cudaEvent_t e = g_spare.back();
        g_spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

void give_back(cudaEvent_t e) {
    if (e != nullptr) g_spare.push_back(e);
}

}  // namespace

int64_t timing_begin(int kernel, cudaStream_t s, double mma_flops) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on || g_records.size() >= kMaxRecords) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    if (cs != cudaStreamCaptureStatusNone) return -1;
    Record r{kernel, take_event(), take_event(), mma_flops, false};
    if (r.begin == nullptr || r.end == nullptr || cudaEventRecord(r.begin, s) != cudaSuccess) {
        (void)cudaGetLastError();
        give_back(r.begin);
        give_back(r.end);
        return -1;
    }
    g_records.push_back(r);
    return ((int64_t)g_generation << 32) | (int64_t)(g_records.size() - 1);
}

void timing_end(int64_t token, cudaStream_t s) {
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    const uint32_t gen = (uint32_t)(token >> 32);
    const size_t slot = (size_t)(token & 0xffffffffll);
    if (gen != g_generation || slot >= g_records.size()) return;
    Record& r = g_records[slot];
    if (cudaEventRecord(r.end, s) == cudaSuccess)
        r.ended = true;
    else
        (void)cudaGetLastError();
}

}  // namespace rmge

using namespace rmge;

extern "C" {

rmge_status rmge_launch_timing(int32_t enable) {
    if (enable != 0 && enable != 1) return RMGE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable) {
        // destroyed rather than kept: the next events are created on the device current now
        for (const Record& r : g_records) {
            (void)cudaEventDestroy(r.begin);
            (void)cudaEventDestroy(r.end);
        }
        for (cudaEvent_t e : g_spare) (void)cudaEventDestroy(e);
        if (!g_records.empty() || !g_spare.empty()) (void)cudaGetLastError();
        g_records.clear();
        g_spare.clear();
        ++g_generation;
    }
    g_on = enable != 0;
    return RMGE_OK;
}

rmge_status rmge_launch_timing_read(int32_t kernel, int64_t* launches, double* ms, double* mma_flops) {
    if (kernel < 0 || kernel >= kTimedKernels || launches == nullptr || ms == nullptr || mma_flops == nullptr)
        return RMGE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t count = 0;
    double total = 0.0, flops = 0.0;
    for (const Record& r : g_records) {
        if (r.kernel != kernel || !r.ended) continue;
        float t = 0.f;
        if (cudaEventSynchronize(r.end) != cudaSuccess || cudaEventElapsedTime(&t, r.begin, r.end) != cudaSuccess) {
            (void)cudaGetLastError();
            return RMGE_ERR_CUDA;
        }
        ++count;
        total += (double)t;
        flops += r.flops;
    }
    *launches = count;
    *ms = total;
    *mma_flops = flops;
    return RMGE_OK;
}

}  // extern "C"
