// rtgd_noalloc.cu -- device scratch for rt_trace_device_noalloc.
//
// Some callers cannot allocate device memory while they trace: code running
// under an allocator that must not be re-entered, graph-building or
// real-time paths with a fixed memory budget, or hosts whose device memory is
// owned by another runtime.  For them the trace scratch -- the persistent
// kernel's ray counter and the fan tables -- lives in this file-scope array,
// which every GPU that loads the library holds until the process exits.  All
// calls share it: work queued by one call must finish before another call's
// work starts on the GPU (calls that overlap on the GPU race on it).
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "rtgd_internal.h"

namespace rtgd {

// 16 bytes of ray counter followed by the fan's tables: at most
// 3 x kNoallocMaxTable doubles (about 96 KiB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static std::map<int, void *> g_noalloc_ptr;

// Device address of the scratch on `device`, which must be the current
// device.  The first call per device looks the symbol up (host code cannot use
// the array's name as a device address); later calls return the cached value.
cudaError_t noalloc_scratch(int device, void **ptr, size_t *bytes) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_ptr.find(device);
    if (it == g_noalloc_ptr.end()) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        it = g_noalloc_ptr.emplace(device, p).first;
    }
    *ptr = it->second;
    *bytes = sizeof(g_noalloc_scratch);
    return cudaSuccess;
}

}  // namespace rtgd
