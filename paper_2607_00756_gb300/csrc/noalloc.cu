// Static device scratch for bip_build_s1_noalloc, the entry point for
// callers that cannot allocate device memory themselves.
//
// The array lives in this library's module: every GPU that loads the
// library holds it (kNoallocScratchBytes) until the process exits.  Host
// code cannot use `bip_noalloc_scratch` as a device address -- the name
// is a host-side stand-in -- so the address is looked up with
// cudaGetSymbolAddress on every call (cheap), in whatever device context
// is current, and handed to the kernels as a plain pointer.  (The library
// serves one GPU per process: its kernels' launch attributes are set once.)
#include "bip_internal.h"

static __device__ __align__(256) unsigned char bip_noalloc_scratch[kNoallocScratchBytes];

cudaError_t bip_noalloc_scratch_ptr(void** ptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, bip_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *ptr = p;
    return cudaSuccess;
}
