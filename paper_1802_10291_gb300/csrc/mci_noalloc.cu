// Scratch of mci_interp_1d_noalloc: a file-scope device array, so that the entry
// point needs no device allocation.  Every GPU that loads the library holds it
// (about 1.5 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "mci_internal.h"

namespace mci {

struct NoAllocScratch {
    int64_t sorted[MCI_NOALLOC_MAX_BATCH];    // signals grouped by size class
    int64_t in_pref[MCI_NOALLOC_MAX_BATCH];   // packed input offsets when the caller gives none
    int64_t out_pref[MCI_NOALLOC_MAX_BATCH];  // packed output offsets
    Sched1D sched;                            // per-class start and count
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
NoAllocScratch* noalloc_scratch(cudaError_t* err)
{
    static std::mutex mu;
    static void* addr[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        *err = e != cudaSuccess ? e : cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        addr[dev] = p;
    }
    *err = cudaSuccess;
    return static_cast<NoAllocScratch*>(addr[dev]);
}

int64_t* noalloc_sorted(NoAllocScratch* s) { return s->sorted; }
int64_t* noalloc_in_pref(NoAllocScratch* s) { return s->in_pref; }
int64_t* noalloc_out_pref(NoAllocScratch* s) { return s->out_pref; }
Sched1D* noalloc_sched(NoAllocScratch* s) { return &s->sched; }

}  // namespace mci
