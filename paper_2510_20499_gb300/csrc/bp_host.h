// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "bp_device.cuh"
#include "gpubp.h"

namespace gpubp {

// Control block of one propagation launch (device memory).  Every counter that many blocks
// update or poll sits on its own 128-byte line so that the blocks do not contend for one L2
// line.  The layout is private to the library; it is reset from a constant template before
// each launch.
template <class T>
struct alignas(128) Pad {
    T v;
};

// Per-round counters rotate over kPhaseSlots slots: round t reads the counts of its worklist
// from slot t % 3 and appends the next round's into slot (t + 1) % 3; its changed variables,
// nonzeros and per-instance verdicts go to slot t % 3.  A slot is cleared two rounds after its
// last reader, so no clearing races a reader or an append.
constexpr int kPhaseSlots = 3;

struct alignas(128) Ctl {
    Pad<unsigned> bar_count;                  // grid barrier arrivals, monotonic within a launch
    Pad<int> cnt[kPhaseSlots][kNumClass];     // worklist rows of a round, per class
    Pad<int> ntask[kPhaseSlots];              // pieces of a round
    Pad<int> nchg[kPhaseSlots];               // variables changed in a round
    Pad<unsigned long long> nnz[kPhaseSlots]; // nonzeros processed in a round
    Pad<unsigned> done;
    int error;
    int phases;                               // phases run (advances the stamp base at exit)
};

// State of one instance of a (possibly batched) propagation.
struct InstState {
    int status, rounds, result_par, first_row, first_var;
    int alive, pending, entry_cross;
    int start_rows;              // variables of the start list (w0v) with rows, in this instance
    unsigned long long nnz_total, n_changed;
};

void ctl_template(Ctl* c);

// Per-launch scratch of the propagation engine.
struct Work {
    longlong2* bkey[2] = {nullptr, nullptr};   // bounds as ordered keys, double-buffered
    int* vstamp = nullptr;                     // n: last round stamp a variable changed
    int* rstamp = nullptr;                     // m: last round stamp a row was queued
    int* list[2] = {nullptr, nullptr};         // m each: worklist rows by class segment
    int* chg[2] = {nullptr, nullptr};          // n each: changed variables
    int4* task[2] = {nullptr, nullptr};        // pieces of the piece rows of a round (piece_desc)
    double* hpart = nullptr;                   // partial activity per piece slot
    int2* hpinf = nullptr;                     // {ninf, infj} per piece slot
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;                   // pinned constant template
    bp_result* dres = nullptr;                 // device result slots (one per instance)
    InstState* inst = nullptr;                 // per-instance state
    unsigned long long* i_nnz = nullptr;       // [kPhaseSlots][ninst]
    int* i_rowinf = nullptr;                   // [kPhaseSlots][ninst]
    int* i_cross = nullptr;                    // [kPhaseSlots][ninst]
    int* i_chg = nullptr;                      // [kPhaseSlots][ninst]
    int inst_cap = 0;
    double* stage_lb = nullptr;                // device staging for host bounds
    double* stage_ub = nullptr;
    int* stamp = nullptr;                      // device: stamp of the next launch's round 0
    int* nvars_dev = nullptr;                  // device word: variable count of bp_propagate_from
    long long* aux = nullptr;                  // 4 device words: probe_cache_apply's result, the
                                               // entry total and index check of bp_probe_batch
};

}  // namespace gpubp

struct mip_problem {
    int device = 0;
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    gpubp::DevProblem dp{};
    double* def_lb = nullptr;
    double* def_ub = nullptr;
    double* obj = nullptr;
    gpubp::Work w;
    int grid_blocks = 0;                       // persistent grid size
    std::vector<void*> allocs;                 // every device allocation of the handle
    std::vector<void*> host_allocs;            // pinned host allocations
    cudaStream_t last_stream = nullptr;
    void* probe_work = nullptr;                // probing scratch (created on first use)
    int ninst = 0;                             // instance batch (mip_set_instances)
    int* inst_row_off = nullptr;
    int* inst_col_off = nullptr;
    void* prio_work = nullptr;                 // priority / sort scratch (created on first use)
    mip_problem* twin = nullptr;               // two copies of this problem as an instance pair
                                               // (fix_and_propagate's candidates; first use)
    // row-class split points and grid shape (bp_set_tuning / bp_autotune)
    int tune_warp_min = gpubp::kDefaultWarpMin;
    int tune_block_min = gpubp::kWarpMax + 1;
    int sms = 0, occ_max = 0;                  // SMs and resident blocks per SM of bp_kernel
    int chunk_cap = 0;                         // capacity of piece-indexed arrays (any piece length)
    void (*free_hooks[4])(mip_problem*) = {nullptr, nullptr, nullptr, nullptr};
};

namespace gpubp {

// thread-local error text
void set_error(const char* fmt, ...);
int fail_cuda(cudaError_t e, const char* what);

// allocation helpers (record on the handle, zero-initialised)
template <class T>
int dalloc(mip_problem* p, T** out, size_t count) {
    void* ptr = nullptr;
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return BP_ERR_OOM;
    }
    p->allocs.push_back(ptr);
    e = cudaMemset(ptr, 0, bytes);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemset");
    *out = static_cast<T*>(ptr);
    return BP_OK;
}

// exclusive scan of n ints on the device; writes the total to *total_dev if non-null.
int scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t s);

int engine_prepare(mip_problem* p);     // allocates Work
// resolves the static scratch of bp_propagate_noalloc on device `dev` (current), loading the
// module that holds it; called when a handle is prepared
int noalloc_prepare(int dev);

// row classes and class lists (rclass, rinfo, static_list, class_off, nlong) from the row lengths
// and the handle's split points
int classify_rows(mip_problem* p, cudaStream_t s);
// piece plan of the piece rows at dp.chunk_len (static_tasks, npieces)
int plan_chunks(mip_problem* p, cudaStream_t s);

// normalised bound keys of caller bounds (device arrays of n doubles)
int root_keys(mip_problem* p, const double* lb, const double* ub, longlong2* out, cudaStream_t s);

// stable LSD radix sort of (key, value) pairs on bits [begin_bit, end_bit)
// The values of the first k pairs of the stable ascending sort of (keys, vals)[0..n), into
// out[0..k), for 1 <= k <= min(n, kSelectMax) (one block; keys and vals unchanged).
constexpr int kSelectMax = 2048;
int select_smallest(const unsigned long long* keys, const int* vals, int n, int k, int* out, cudaStream_t s);
int radix_sort_pairs(unsigned long long* keys, int* vals, unsigned long long* tmp_keys, int* tmp_vals, int n,
                     int begin_bit, int end_bit, cudaStream_t s);
// one propagation on device bounds lb/ub (modified in place); round 0 holds every row, or the
// rows w0[0..w0_len), or the rows of the variables w0v[0..*w0v_len) (count read on the device)
int launch_propagate(mip_problem* p, double* lb, double* ub, const int* w0, int w0_len,
                     double theta, int max_rounds, int64_t* trace, cudaStream_t s,
                     const int* w0v = nullptr, const int* w0v_len = nullptr, int ninst = 1,
                     const int* row_off = nullptr, const int* col_off = nullptr);
// Device-driven one-variable fixings of fix_and_propagate over the instance pair `tw` (two
// copies of a problem with n0 variables): for each variable of queue[0..qlen) still unfixed in
// cur (ordered keys, updated in place), the two candidates propagate and the first feasible
// one becomes cur; stops after the first variable whose candidates are both infeasible.  The
// pair's key buffers must hold [cur, cur] on entry and hold it again on exit.  vdirty (2 n0,
// zero or older stamps), dirty (2 n0) and words (4) are scratch; out is device memory.
// On a stop (infeasible = 1) stop_q is the queue index of the variable that failed, j that
// variable and v0 its drawn value.  chosen / cval (both NULL, or device arrays of n0): every kept
// fixing is recorded there (the repair's fixings by choice).
struct FpSingleOut {
    long long bulks, bp_runs, nnz_updates, fixed;
    int infeasible, error, stop_q, j;
    double v0;
};
int launch_fp_single(mip_problem* tw, int n0, longlong2* cur, const int* queue, int qlen, const double* x,
                     const double* up_prob, unsigned long long seed, unsigned long long bulk0, double theta,
                     int max_rounds, int* vdirty, int* dirty, int* words, FpSingleOut* out, unsigned char* chosen,
                     double* cval, cudaStream_t s);
constexpr int kMaxInstances = 1024;

}  // namespace gpubp

#define BP_CUDA_TRY(expr)                                           \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return gpubp::fail_cuda(_e, #expr);  \
    } while (0)
#define BP_TRY(expr)                 \
    do {                             \
        int _r = (expr);             \
        if (_r != BP_OK) return _r;  \
    } while (0)
