// vr_noalloc.cu -- vr_render_batch for callers that cannot allocate memory.
//
// vr_render_batch needs a small device workspace for its work counter and
// per-request tile counters, and asks the caller for it.  Some callers cannot
// provide one: code that runs where allocating device memory is not allowed
// or not possible (inside a real-time or embedded loop with a fixed memory
// budget, a plugin given no allocator, a process that must not grow its
// footprint after start-up).  This file gives them the same batched render
// with its counters in a fixed array that lives in the library's own device
// memory image instead: nothing is allocated by the call, the library or any
// library it uses.
//
// The array is a file-scope __device__ variable.  Its name, used in host
// code, is only a host-side stand-in: handing it to a kernel would be wrong.
// Its device address is obtained once per device with cudaGetSymbolAddress,
// with that device current, and passed to the kernel like any buffer.
#include <mutex>

#include "vr_internal.h"

namespace vr {
namespace {

// The counters of one launch: the work counter and a tile counter per request
// (kBatchWords words, 260 bytes).  Every GPU that loads the library holds
// these bytes until the process exits.
constexpr int kStaticRequests = VR_BATCH_MAX;
static __device__ __align__(256) unsigned g_batch_counters[kBatchWords];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned* g_counters_addr[kMaxDevices];   // device address of the array, per device

}  // namespace
}  // namespace vr

extern "C" int vr_render_batch_noalloc(const vr_request* reqs, int n, void* stream)
{
    if (n < 0) return vr::record_error(VR_ERR_ARG, "n must not be negative");
    if (n > vr::kStaticRequests)
        return vr::record_error(VR_ERR_ARG,
                                "vr_render_batch_noalloc takes at most VR_BATCH_MAX (64) "
                                "requests per call; use vr_render_batch for more");
    if (n == 0) return VR_OK;
    if (!reqs) return vr::record_error(VR_ERR_ARG, "reqs is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= vr::kMaxDevices)
        return vr::record_error(VR_ERR_CUDA, "no usable current device");
    unsigned* counters = nullptr;
    {
        std::lock_guard<std::mutex> guard(vr::g_lock);
        if (!vr::g_counters_addr[dev]) {
            // first call on this device (which is current): look up where the
            // array lives in this device's memory
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, vr::g_batch_counters);
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                return vr::record_error(VR_ERR_CUDA, "cannot resolve the static counter array");
            }
            vr::g_counters_addr[dev] = static_cast<unsigned*>(addr);
        }
        counters = vr::g_counters_addr[dev];
    }
    // the counters keep the previous call's values: every launch below zeroes
    // them on the stream before its kernel runs
    return vr::batch_with_counters(reqs, n, counters, static_cast<cudaStream_t>(stream));
}
