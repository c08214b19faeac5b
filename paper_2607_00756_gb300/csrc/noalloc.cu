// Static device scratch for bip_build_s1_noalloc, the entry point for
// callers that cannot allocate device memory themselves.
//
// The array lives in this library's module: every GPU that loads the
// library holds it (kNoallocScratchBytes) until the process exits.  Host
// code cannot use `bip_noalloc_scratch` as a device address -- the name
// is a host-side stand-in -- so the address is looked up once per device
// with cudaGetSymbolAddress and handed to the kernels as a plain pointer.
#include <map>
#include <mutex>

#include "bip_internal.h"

static __device__ __align__(256) unsigned char bip_noalloc_scratch[kNoallocScratchBytes];

cudaError_t bip_noalloc_scratch_ptr(void** ptr) {
    static std::mutex mu;
    static std::map<int, void*> addr;   // device -> address of the array
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = addr.find(dev);
    if (it != addr.end()) {
        *ptr = it->second;
        return cudaSuccess;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, bip_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
    *ptr = p;
    return cudaSuccess;
}
