// k_match_noalloc.cu — a variant of the match stage that allocates nothing.
//
// rfr_stage_match needs a device workspace from its caller.  Some callers
// cannot provide one: code that runs under a host framework which owns all
// device memory and forbids side allocations, or a latency-critical loop in
// which a cudaMalloc (which may synchronise the device) is not allowed.  For
// them rfr_stage_match_noalloc takes its workspace from a fixed array in
// device memory that is part of this library: every GPU that loads the
// library holds RFR_NOALLOC_SCRATCH_BYTES of it until the process exits.
//
// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device with cudaGetSymbolAddress (on the
// first call made with that device current) and cached.  All calls on a
// device share the array, so calls that overlap on the GPU (two streams, or
// two host threads) race on it and must be serialised by the caller.  The
// match zeroes the parts of the workspace that must start at zero (its
// counters and halo counts) on every call, so results do not depend on what
// an earlier call left behind.  The cached address is not looked up again:
// after a cudaDeviceReset of a device it is stale, and the header says not to
// call this entry point on a device that has been reset.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rfr_stages.h"

namespace {

__device__ __align__(256) unsigned char g_match_scratch[RFR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
void* scratch_for_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_match_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

}  // namespace

extern "C" int rfr_stage_match_noalloc(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                                       const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                                       uint64_t window, uint64_t window2,
                                       uint64_t* cand, uint64_t cap, uint64_t* counters,
                                       void* stream) {
    const size_t need = rfr_stage_match_workspace(n_a, n_b);
    if (need == 0) return RFR_E_INVALID;
    if (need > (size_t)RFR_NOALLOC_SCRATCH_BYTES) return RFR_E_BUDGET;
    void* ws = scratch_for_current_device();
    if (!ws) return RFR_E_CUDA;
    return rfr_stage_match(w_a, w2_a, n_a, w_b, w2_b, n_b, window, window2, ws,
                           (size_t)RFR_NOALLOC_SCRATCH_BYTES, cand, cap, counters, stream);
}
