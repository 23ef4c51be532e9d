// bp_propagate_noalloc: bound propagation whose per-call scratch is a fixed array in static
// device memory instead of buffers allocated for the handle.
//
// The paper has no counterpart.  Some callers cannot allocate device memory while they run:
// a solver process that reserves its whole device budget at start-up and treats any later
// allocation as a failure, or a host framework whose caching allocator already holds the free
// memory, where a cudaMalloc or cudaFree issued by this library could fail, or would stall
// every stream on the device in the middle of a search.  For them this entry point takes its
// scratch from one file-scope array, reserved when the module that holds it is loaded, and calls
// no allocation routine of any kind.  The propagation itself is the persistent engine of
// bp_propagate, launched unchanged on the carved scratch.
#include <mutex>

#include "bp_host.h"

// The scratch: one array per device, in the module's static device memory.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BP_NOALLOC_SCRATCH_BYTES];

namespace gpubp {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device

// Once per device, with that device current: the device address of the scratch array.  The
// first lookup loads the module that holds the array (CUDA loads modules lazily), which reserves
// the array's memory on the device; handle creation makes that first lookup (noalloc_prepare), so
// that bp_propagate_noalloc itself never causes it.
int scratch_base(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        unsigned char* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress of the static scratch");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return BP_OK;
}

// Carves the engine's buffers out of the scratch, each on a 256-byte boundary and at least one
// element long (as the handle's own buffers are).  Nothing is dereferenced on the host.
struct Carve {
    uintptr_t base;   // 0 when only sizing
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * (count ? count : 1);
        return p;
    }
};

// Lays out the scratch of one single-instance propagation.  The buffers that must start at
// zero come first, so that one memset clears them: the stamp word, the control block and the
// row and variable stamps.  Returns the bytes of that prefix; c.off is the total.
size_t layout(const mip_problem* p, Carve& c, Work& w) {
    const size_t n = (size_t)p->n, m = (size_t)p->m;
    const size_t npieces = (size_t)p->dp.npieces;   // a round holds at most every piece once
    w.stamp = c.take<int>(1);
    w.ctl = c.take<Ctl>(1);
    w.vstamp = c.take<int>(n);
    w.rstamp = c.take<int>(m);
    const size_t zero_bytes = c.off;
    w.bkey[0] = c.take<longlong2>(n);
    w.bkey[1] = c.take<longlong2>(n);
    w.list[0] = c.take<int>(m);
    w.list[1] = c.take<int>(m);
    w.chg[0] = c.take<int>(n);
    w.chg[1] = c.take<int>(n);
    w.task[0] = c.take<int4>(npieces);
    w.task[1] = c.take<int4>(npieces);
    w.hpart = c.take<double>(npieces);
    w.hpinf = c.take<int2>(npieces);
    w.dres = c.take<bp_result>(1);
    w.inst = c.take<InstState>(1);
    w.i_nnz = c.take<unsigned long long>(kPhaseSlots);
    w.i_rowinf = c.take<int>(kPhaseSlots);
    w.i_cross = c.take<int>(kPhaseSlots);
    w.i_chg = c.take<int>(kPhaseSlots);
    w.inst_cap = 1;
    return zero_bytes;
}

}  // namespace

int noalloc_prepare(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return BP_OK;   // the entry point rejects such devices itself
    unsigned char* base = nullptr;
    return scratch_base(dev, &base);
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int bp_propagate_noalloc(mip_problem* p, double* lb, double* ub, const bp_params* params,
                                    bp_result* result, void* stream) {
    if (!p || (p->n && (!lb || !ub))) {
        set_error("bp_propagate_noalloc: null argument");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) {
        prm = *params;
    } else {
        bp_params_default(&prm);
    }
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 || prm.bounds_mem != BP_MEM_DEVICE) {
        set_error("bp_propagate_noalloc: invalid parameters (theta >= 0, max_rounds >= 0, device bounds only)");
        return BP_ERR_INVALID;
    }
    int dev = -1;
    BP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device || dev < 0 || dev >= kMaxDevices) {
        set_error("bp_propagate_noalloc: the handle's device %d must be current (current: %d, at most %d devices)",
                  p->device, dev, kMaxDevices);
        return BP_ERR_INVALID;
    }
    // size check on the host, before anything is enqueued
    Work w;
    Carve sizing{0};
    layout(p, sizing, w);
    if (sizing.off > (size_t)BP_NOALLOC_SCRATCH_BYTES) {
        set_error("bp_propagate_noalloc: this problem (m=%d, n=%d) needs %zu bytes of scratch, above the fixed "
                  "limit of %zu bytes; use bp_propagate",
                  p->m, p->n, sizing.off, (size_t)BP_NOALLOC_SCRATCH_BYTES);
        return BP_ERR_CAPACITY;
    }
    unsigned char* base = nullptr;
    BP_TRY(scratch_base(dev, &base));
    Carve c{reinterpret_cast<uintptr_t>(base)};
    const size_t zero_bytes = layout(p, c, w);
    w.ctl_host = p->w.ctl_host;   // the handle's constant control-block template
    cudaStream_t s = (cudaStream_t)stream;
    // fresh state, as a newly prepared handle has it: zeros, and the stamp word at 1 (one byte
    // of value 1 in the low-order position of a zeroed little-endian int)
    BP_CUDA_TRY(cudaMemsetAsync(base, 0, zero_bytes, s));
    BP_CUDA_TRY(cudaMemsetAsync(w.stamp, 1, 1, s));
    // the engine's launch reads its scratch from the handle: point it at the carved scratch
    // for the launch, then give the handle its own buffers back
    const Work own = p->w;
    p->w = w;
    const int rc = launch_propagate(p, lb, ub, nullptr, 0, prm.theta, prm.max_rounds, prm.trace, s);
    p->w = own;
    if (rc != BP_OK) return rc;
    if (result) BP_CUDA_TRY(cudaMemcpyAsync(result, w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s));
    return BP_OK;
}
