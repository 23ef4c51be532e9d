// Autotuning of the propagation engine's row-class split points and grid shape:
// bp_get_tuning, bp_set_tuning, bp_autotune.
//
// The paper bins rows by length so that each bin gets a suitable amount of parallelism
// (Section 2.1) and runs many problems concurrently (Section 2.2); where the bins split and how
// many blocks the persistent grid keeps per SM are machine- and instance-dependent choices.
// bp_autotune times a small grid of them on the caller's start bounds and keeps the fastest
// whose results equal the defaults' (same status, rounds, work and changed-variable counts for
// every instance): the split points change which code path sums a row, never what it computes.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bp_host.h"

using namespace gpubp;

namespace {

bool chunk_len_valid(int c) { return c == 32 || c == 64 || c == 128 || c == kPieceMax; }

bool tuning_valid(const mip_problem* p, const bp_tuning* t) {
    return t->warp_min >= 2 && t->warp_min <= kThreadMax + 1 && t->block_min >= t->warp_min &&
           t->block_min <= kWarpMax + 1 && t->blocks_per_sm >= 1 && t->blocks_per_sm <= p->occ_max &&
           chunk_len_valid(t->chunk_len);
}

int apply(mip_problem* p, const bp_tuning* t, cudaStream_t s) {
    const bool rechunk = t->chunk_len != p->dp.chunk_len;
    const bool reclass = rechunk || t->warp_min != p->tune_warp_min || t->block_min != p->tune_block_min;
    p->tune_warp_min = t->warp_min;
    p->tune_block_min = t->block_min;
    p->dp.chunk_len = t->chunk_len;
    p->grid_blocks = p->sms * t->blocks_per_sm;
    if (reclass) {
        BP_TRY(classify_rows(p, s));   // row classes and piece counts per row
        BP_TRY(plan_chunks(p, s));     // the round-0 piece list (block_min decides the piece rows)
    }
    return BP_OK;
}

bool same_results(const std::vector<bp_result>& a, const std::vector<bp_result>& b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].status != b[i].status || a[i].rounds != b[i].rounds || a[i].nnz_updates != b[i].nnz_updates ||
            a[i].n_changed != b[i].n_changed || a[i].error != b[i].error ||
            a[i].first_infeasible_row != b[i].first_infeasible_row ||
            a[i].first_infeasible_var != b[i].first_infeasible_var)
            return false;
    return true;
}

}  // namespace

extern "C" int bp_get_tuning(const mip_problem* p, bp_tuning* out) {
    if (!p || !out) {
        set_error("bp_get_tuning: null argument");
        return BP_ERR_INVALID;
    }
    out->warp_min = p->tune_warp_min;
    out->block_min = p->tune_block_min;
    out->blocks_per_sm = p->sms ? p->grid_blocks / p->sms : 0;
    out->chunk_len = p->dp.chunk_len;
    return BP_OK;
}

extern "C" int bp_set_tuning(mip_problem* p, const bp_tuning* t, void* stream) {
    if (!p || !t) {
        set_error("bp_set_tuning: null argument");
        return BP_ERR_INVALID;
    }
    if (!tuning_valid(p, t)) {
        set_error("bp_set_tuning: need 2 <= warp_min <= %d, warp_min <= block_min <= %d, 1 <= blocks_per_sm <= %d, "
                  "chunk_len in {32, 64, 128, %d} (got %d, %d, %d, %d)",
                  kThreadMax + 1, kWarpMax + 1, p->occ_max, kPieceMax, t->warp_min, t->block_min, t->blocks_per_sm,
                  t->chunk_len);
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BP_TRY(apply(p, t, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    return BP_OK;
}

extern "C" int bp_autotune(mip_problem* p, const double* lb, const double* ub, const bp_params* params, int32_t reps,
                           bp_tune_report* report, void* stream) {
    if (!p || (p->n && (!lb || !ub))) {
        set_error("bp_autotune: null argument");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) prm = *params;
    else bp_params_default(&prm);
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 || prm.bounds_mem != BP_MEM_DEVICE) {
        set_error("bp_autotune: invalid parameters (device bounds only)");
        return BP_ERR_INVALID;
    }
    if (reps <= 0) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    const bool batch = p->ninst > 1;
    const int ninst = batch ? p->ninst : 1;
    const size_t bytes = sizeof(double) * (size_t)p->n;
    double* wl = p->w.stage_lb;
    double* wu = p->w.stage_ub;
    cudaEvent_t e0, e1;
    BP_CUDA_TRY(cudaEventCreate(&e0));
    BP_CUDA_TRY(cudaEventCreate(&e1));

    // one configuration: a warm-up and `reps` timed propagations from lb/ub; median time
    auto measure = [&](const bp_tuning& t, float* ms, std::vector<bp_result>* res) -> int {
        BP_TRY(apply(p, &t, s));
        std::vector<float> times;
        for (int r = 0; r <= reps; ++r) {
            if (p->n) {
                BP_CUDA_TRY(cudaMemcpyAsync(wl, lb, bytes, cudaMemcpyDeviceToDevice, s));
                BP_CUDA_TRY(cudaMemcpyAsync(wu, ub, bytes, cudaMemcpyDeviceToDevice, s));
            }
            BP_CUDA_TRY(cudaEventRecord(e0, s));
            if (batch) {
                BP_TRY(launch_propagate(p, wl, wu, nullptr, 0, prm.theta, prm.max_rounds, nullptr, s, nullptr, nullptr,
                                        p->ninst, p->inst_row_off, p->inst_col_off));
            } else {
                BP_TRY(launch_propagate(p, wl, wu, nullptr, 0, prm.theta, prm.max_rounds, nullptr, s));
            }
            BP_CUDA_TRY(cudaEventRecord(e1, s));
            BP_CUDA_TRY(cudaEventSynchronize(e1));
            float t_ms = 0.f;
            BP_CUDA_TRY(cudaEventElapsedTime(&t_ms, e0, e1));
            if (r > 0) times.push_back(t_ms);
        }
        res->resize(ninst);
        BP_CUDA_TRY(cudaMemcpyAsync(res->data(), p->w.dres, sizeof(bp_result) * ninst, cudaMemcpyDeviceToHost, s));
        BP_CUDA_TRY(cudaStreamSynchronize(s));
        std::sort(times.begin(), times.end());
        *ms = times[times.size() / 2];
        return BP_OK;
    };

    bp_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    const bp_tuning defaults{kDefaultWarpMin, kWarpMax + 1, p->occ_max, kDefaultChunkLen};
    std::vector<bp_result> ref, cur;
    int rc = measure(defaults, &rep.default_ms, &ref);
    rep.best = defaults;
    rep.best_ms = rep.default_ms;
    rep.tried = 1;
    static const int kWarpMins[] = {2, kThreadMax + 1};
    static const int kBlockMins[] = {65, kWarpMax + 1};
    static const int kChunkLens[] = {64, 128, kPieceMax};
    for (int bps = 1; rc == BP_OK && bps <= p->occ_max; ++bps)
        for (int wm : kWarpMins)
            for (int bm : kBlockMins)
                for (int cl : kChunkLens) {
                    if (rc != BP_OK) break;
                    const bp_tuning t{wm, bm, bps, cl};
                    if (wm == defaults.warp_min && bm == defaults.block_min && bps == defaults.blocks_per_sm &&
                        cl == defaults.chunk_len)
                        continue;
                    float ms = 0.f;
                    rc = measure(t, &ms, &cur);
                    if (rc != BP_OK) break;
                    ++rep.tried;
                    if (!same_results(ref, cur)) {
                        ++rep.rejected;
                        continue;
                    }
                    if (ms < rep.best_ms) {
                        rep.best_ms = ms;
                        rep.best = t;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BP_OK) {
        apply(p, &defaults, s);
        return rc;
    }
    BP_TRY(apply(p, &rep.best, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (report) *report = rep;
    return BP_OK;
}
