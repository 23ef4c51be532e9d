// Batches of independent instances (the batched form of Section 2.1): mip_set_instances and
// bp_propagate_batch.  The instances share one block-diagonal layout and one persistent
// launch; the engine keeps a state per instance (bp_engine.cu).
#include <vector>

#include "bp_host.h"

namespace gpubp {

// every nonzero of row k lies in the column range of k's instance
__global__ void k_check_blocks(int m, int ninst, const int* rp, const int* col, const int* roff, const int* coff,
                               int* bad) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m; k += (gridDim.x * blockDim.x) >> 5) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (roff[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const int c0 = coff[lo], c1 = coff[lo + 1];
        bool b = false;
        for (int q = rp[k] + lane; q < rp[k + 1]; q += 32) b |= col[q] < c0 || col[q] >= c1;
        if (__any_sync(0xffffffffu, b) && lane == 0) atomicMin(bad, k);
    }
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int mip_set_instances(mip_problem* p, int32_t ninst, const int32_t* row_off, const int32_t* col_off,
                                 int32_t mem_kind, void* stream) {
    if (!p || !row_off || !col_off || ninst < 1 || ninst > kMaxInstances ||
        (mem_kind != BP_MEM_HOST && mem_kind != BP_MEM_DEVICE)) {
        set_error("mip_set_instances: invalid arguments (1 <= ninst <= %d)", kMaxInstances);
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> ro((size_t)ninst + 1), co((size_t)ninst + 1);
    const cudaMemcpyKind kind = mem_kind == BP_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    BP_CUDA_TRY(cudaMemcpyAsync(ro.data(), row_off, sizeof(int32_t) * (ninst + 1), kind, s));
    BP_CUDA_TRY(cudaMemcpyAsync(co.data(), col_off, sizeof(int32_t) * (ninst + 1), kind, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (ro[0] != 0 || co[0] != 0 || ro[ninst] != p->m || co[ninst] != p->n) {
        set_error("instance offsets must start at 0 and end at m, n");
        return BP_ERR_INVALID;
    }
    for (int i = 0; i < ninst; ++i)
        if (ro[i + 1] < ro[i] || co[i + 1] < co[i]) {
            set_error("instance offsets must be nondecreasing (instance %d)", i);
            return BP_ERR_INVALID;
        }
    int *d_ro = nullptr, *d_co = nullptr, *bad = nullptr;
    BP_TRY(dalloc(p, &d_ro, (size_t)ninst + 1));
    BP_TRY(dalloc(p, &d_co, (size_t)ninst + 1));
    BP_TRY(dalloc(p, &bad, 1));
    BP_CUDA_TRY(cudaMemcpyAsync(d_ro, ro.data(), sizeof(int32_t) * (ninst + 1), cudaMemcpyHostToDevice, s));
    BP_CUDA_TRY(cudaMemcpyAsync(d_co, co.data(), sizeof(int32_t) * (ninst + 1), cudaMemcpyHostToDevice, s));
    BP_CUDA_TRY(cudaMemsetAsync(bad, 0x7f, sizeof(int), s));
    if (p->m) {
        long long b = ((long long)p->m * 32 + 255) / 256;
        k_check_blocks<<<(int)(b > 1216 ? 1216 : b), 256, 0, s>>>(p->m, ninst, p->dp.row_ptr, p->dp.col, d_ro, d_co, bad);
        BP_CUDA_TRY(cudaGetLastError());
    }
    int hbad = 0;
    BP_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad != 0x7f7f7f7f) {
        set_error("row %d has a nonzero outside its instance's variables", hbad);
        return BP_ERR_INVALID;
    }
    p->ninst = ninst;
    p->inst_row_off = d_ro;
    p->inst_col_off = d_co;
    return BP_OK;
}

extern "C" int bp_propagate_batch(mip_problem* p, double* lb, double* ub, const bp_params* params,
                                  bp_result* results, void* stream) {
    if (!p || !results || (p->n && (!lb || !ub))) {
        set_error("bp_propagate_batch: null argument");
        return BP_ERR_INVALID;
    }
    if (p->ninst < 1 || !p->inst_row_off) {
        set_error("bp_propagate_batch: no instance batch declared (mip_set_instances)");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) prm = *params;
    else bp_params_default(&prm);
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 || prm.bounds_mem != BP_MEM_DEVICE) {
        set_error("bp_propagate_batch: invalid parameters (device bounds only)");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BP_TRY(launch_propagate(p, lb, ub, nullptr, 0, prm.theta, prm.max_rounds, prm.trace, s, nullptr, nullptr,
                            p->ninst, p->inst_row_off, p->inst_col_off));
    BP_CUDA_TRY(cudaMemcpyAsync(results, p->w.dres, sizeof(bp_result) * p->ninst, cudaMemcpyDeviceToDevice, s));
    return BP_OK;
}
