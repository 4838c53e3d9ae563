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
// Its device address is looked up with cudaGetSymbolAddress, with the device
// current, at the first call in each CUDA context, and passed to the kernel
// like any buffer.  The cache is keyed on the context's unique ID (not the
// device number, nor the context handle, which a reset may hand out again):
// after a device reset, or with another context current on the same device,
// the old address would be stale, so a new context looks it up again.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "vr_internal.h"

namespace vr {
namespace {

// The counters of one launch: the work counter and a tile counter per request
// (kBatchWords words, 260 bytes).  Every GPU that loads the library holds
// these bytes until the process exits.
constexpr int kStaticRequests = VR_BATCH_MAX;
static __device__ __align__(256) unsigned g_batch_counters[kBatchWords];

// Address of the array per context ID (a few contexts at most in practice;
// a full table is refilled from the start).
constexpr int kMaxContexts = 64;
std::mutex g_lock;
struct CtxAddr {
    unsigned long long ctx_id;
    unsigned* addr;
};
CtxAddr g_addr[kMaxContexts];
int g_n_addr = 0;

// The two driver calls this file needs, reached through the runtime (the
// library does not link the driver library itself).
struct DriverCalls {
    PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    PFN_cuCtxGetId_v12000 get_id = nullptr;
    bool ok = false;
};

const DriverCalls& driver_calls()
{
    static const DriverCalls calls = [] {
        DriverCalls c;
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                             &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            c.get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
            c.get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
            c.ok = true;
        }
        cudaGetLastError();
        return c;
    }();
    return calls;
}

unsigned* lookup_counters()
{
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_batch_counters);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned*>(addr);
}

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
    // the context the launch will use: the one current on this thread (none
    // yet if the runtime has not touched the device on this thread: the
    // symbol lookup then initialises the device's primary context)
    const vr::DriverCalls& drv = vr::driver_calls();
    if (!drv.ok) return vr::record_error(VR_ERR_CUDA, "CUDA driver entry points unavailable");
    CUcontext ctx = nullptr;
    unsigned* fresh = nullptr;
    if (drv.get_current(&ctx) != CUDA_SUCCESS || !ctx) {
        fresh = vr::lookup_counters();
        if (!fresh || drv.get_current(&ctx) != CUDA_SUCCESS || !ctx)
            return vr::record_error(VR_ERR_CUDA, "no usable current device");
    }
    unsigned long long id = 0;
    if (drv.get_id(ctx, &id) != CUDA_SUCCESS)
        return vr::record_error(VR_ERR_CUDA, "cannot identify the current context");
    unsigned* counters = nullptr;
    {
        std::lock_guard<std::mutex> guard(vr::g_lock);
        for (int i = 0; i < vr::g_n_addr; ++i)
            if (vr::g_addr[i].ctx_id == id) counters = vr::g_addr[i].addr;
        if (!counters) {
            // first call in this context: look up where the array lives in
            // this device's memory
            counters = fresh ? fresh : vr::lookup_counters();
            if (!counters)
                return vr::record_error(VR_ERR_CUDA, "cannot resolve the static counter array");
            if (vr::g_n_addr == vr::kMaxContexts) vr::g_n_addr = 0;
            vr::g_addr[vr::g_n_addr++] = {id, counters};
        }
    }
    // the counters keep the previous call's values: every launch below zeroes
    // them on the stream before its kernel runs
    return vr::batch_with_counters(reqs, n, counters, static_cast<cudaStream_t>(stream));
}
